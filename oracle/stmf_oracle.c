/*
 * Oracle for FastSTMF (Omanovic, Oblak, Curk: "FastSTMF: Efficient tropical
 * matrix factorization algorithm for sparse data", arXiv 2205.06619).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow CPU restatement of
 * the method, written from the paper's definitions and algorithms.  The
 * loops over independent rows or columns may run on several host threads
 * (OpenMP); every sum runs in a fixed order, so the results do not depend on
 * the number of threads.  Only the tests, the package's smoke() check and the CPU
 * baseline leg of bench.py may load it.  It shares no code, header, table or
 * helper with the CUDA library, and the CUDA library never calls it.
 *
 * Arithmetic modes
 *   mode 0 (ORC_FP64): every value and every operation in IEEE double.
 *   mode 1 (ORC_FP32): values are floats held in doubles; every elementary
 *     add / sub / div result is rounded to float.  For one operation on two
 *     floats, rounding the double result to float gives the correctly rounded
 *     float result (double has more than 2*24+2 significand bits), so this
 *     mode reproduces IEEE fp32 arithmetic bit for bit.  max / min / abs are
 *     exact in both modes.  Error sums (b-norm) are always accumulated in
 *     double, in row-major order, from terms rounded in the mode's precision.
 *
 * Layouts: row-major doubles.  R is m x n, M is an m x n byte mask (1 = the
 * entry of R is given/observed), U is m x r, V is r x n.
 *
 * Readings of places where the paper is silent or ambiguous are marked
 * "Reading:" below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_FP64 0
#define ORC_FP32 1

/* selections of (j, k) within a row (Section "The ByRow strategy") */
#define ORC_SEL_TD_A 0
#define ORC_SEL_TD_B 1
#define ORC_SEL_TD 2
#define ORC_SEL_SEQ 3

static double rnd(int mode, double x) { return mode == ORC_FP32 ? (double)(float)x : x; }
static double add_(int mode, double a, double b) { return rnd(mode, a + b); }
static double sub_(int mode, double a, double b) { return rnd(mode, a - b); }
static double div_(int mode, double a, double b) { return rnd(mode, a / b); }

int orc_version(void) { return 2; }

#ifdef _OPENMP
#include <omp.h>
#endif

/* Host threads of the parallel loops (0 or less: all the host's cores). */
void orc_set_threads(int nthreads)
{
#ifdef _OPENMP
    omp_set_num_threads(nthreads > 0 ? nthreads : omp_get_num_procs());
#else
    (void)nthreads;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Random draws.  SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) used as a
 * counter-based generator: draw(key, c) is the output of a SplitMix64 whose
 * state was key and which has advanced c+1 times.                          */
uint64_t orc_splitmix64(uint64_t key, uint64_t c)
{
    uint64_t z = key + (c + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Random permutation of 0..m-1 (Algorithm 3, "perm <- random permutation"):
 * Fisher-Yates from the top: for a = m-1 .. 1, b = draw(seed, m-1-a) mod
 * (a+1), swap perm[a] and perm[b].                                          */
void orc_randperm(int m, uint64_t seed, int32_t *perm)
{
    for (int s = 0; s < m; ++s) perm[s] = s;
    for (int a = m - 1; a >= 1; --a) {
        uint64_t x = orc_splitmix64(seed, (uint64_t)(m - 1 - a));
        int b = (int)(x % (uint64_t)(a + 1));
        int32_t t = perm[a]; perm[a] = perm[b]; perm[b] = t;
    }
}

/* Random Acol picks (Section "Comparison of strategies": U initialised by
 * averaging randomly chosen columns of R).  For component l, p distinct
 * columns of 0..n-1 by a partial Fisher-Yates on a fresh identity array:
 * for q = 0..p-1, b = q + draw(seed ^ 0xA5A5..., l*p+q) mod (n-q).          */
void orc_acol_picks(int n, int r, int p, uint64_t seed, int32_t *picks)
{
    int32_t *arr = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    uint64_t key = seed ^ 0xA5A5A5A5A5A5A5A5ull;
    for (int l = 0; l < r; ++l) {
        for (int t = 0; t < n; ++t) arr[t] = t;
        for (int q = 0; q < p; ++q) {
            uint64_t x = orc_splitmix64(key, (uint64_t)l * (uint64_t)p + (uint64_t)q);
            int b = q + (int)(x % (uint64_t)(n - q));
            int32_t t = arr[q]; arr[q] = arr[b]; arr[b] = t;
            picks[l * p + q] = arr[q];
        }
    }
    free(arr);
}

/* ------------------------------------------------------------------------ */
/* Tropical product (Section "Related work", matrix multiplication):
 * (U (x) V)_ij = max_l (U_il + V_lj).  Also returns, per entry, the argmax
 * f(i,j) with ties going to the smaller l (Section "The ByRow strategy",
 * definition of f(i,j)), and the runner-up P2_ij = max over l != f(i,j).
 * P2 is -inf when r == 1.  A or P2 may be NULL.                             */
void orc_maxplus(int mode, int m, int n, int r, const double *U, const double *V,
                 double *P1, int32_t *A, double *P2)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) {
            double best = -INFINITY, second = -INFINITY;
            int arg = 0;
            for (int l = 0; l < r; ++l) {
                double s = add_(mode, U[(size_t)i * r + l], V[(size_t)l * n + j]);
                if (s > best) { second = best; best = s; arg = l; }
                else if (s > second) { second = s; }
            }
            P1[(size_t)i * n + j] = best;
            if (A) A[(size_t)i * n + j] = arg;
            if (P2) P2[(size_t)i * n + j] = second;
        }
}

/* Min-plus residuation (Section "Related work", the (min,+) operation over
 * given entries) in the two shapes the factor updates use:
 *   residuate_v:  v = (-u)^T (x)* R,  v_t = min over given s of (R_st - u_s)
 *   residuate_u:  u = R (x)* (-v)^T,  u_s = min over given t of (R_st - v_t)
 * A row/column with no given entry yields +inf; the return value counts
 * them (the method needs every row and column to have a given entry).      */
int orc_residuate_v(int mode, int m, int n, const double *R, const uint8_t *M,
                    const double *u, double *v)
{
    int empty = 0;
#pragma omp parallel for schedule(static) reduction(+ : empty)
    for (int t = 0; t < n; ++t) {
        double best = INFINITY;
        int any = 0;
        for (int s = 0; s < m; ++s) {
            if (!M[(size_t)s * n + t]) continue;
            double d = sub_(mode, R[(size_t)s * n + t], u[s]);
            if (!any || d < best) best = d;
            any = 1;
        }
        v[t] = best;
        empty += !any;
    }
    return empty;
}

int orc_residuate_u(int mode, int m, int n, const double *R, const uint8_t *M,
                    const double *v, double *u)
{
    int empty = 0;
#pragma omp parallel for schedule(static) reduction(+ : empty)
    for (int s = 0; s < m; ++s) {
        double best = INFINITY;
        int any = 0;
        for (int t = 0; t < n; ++t) {
            if (!M[(size_t)s * n + t]) continue;
            double d = sub_(mode, R[(size_t)s * n + t], v[t]);
            if (!any || d < best) best = d;
            any = 1;
        }
        u[s] = best;
        empty += !any;
    }
    return empty;
}

/* Approximation error in the b-norm over the given entries (Section
 * "Evaluation metrics", b-norm = sum of absolute values):
 * f = sum over given (s,t) of |R_st - (U (x) V)_st|, recomputed from
 * scratch, summed in double: each row in column order, then the rows in row
 * order.                                                                    */
double orc_error(int mode, int m, int n, int r, const double *R, const uint8_t *M,
                 const double *U, const double *V)
{
    double *rowsum = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
#pragma omp parallel for schedule(static)
    for (int s = 0; s < m; ++s) {
        double fs = 0.0;
        for (int t = 0; t < n; ++t) {
            if (!M[(size_t)s * n + t]) continue;
            double best = -INFINITY;
            for (int l = 0; l < r; ++l) {
                double x = add_(mode, U[(size_t)s * r + l], V[(size_t)l * n + t]);
                if (x > best) best = x;
            }
            fs += fabs(sub_(mode, R[(size_t)s * n + t], best));
        }
        rowsum[s] = fs;
    }
    double f = 0.0;
    for (int s = 0; s < m; ++s) f += rowsum[s];
    free(rowsum);
    return f;
}

/* Root-mean-square errors of the approximation (Section "Evaluation
 * metrics": RMSE of the training data, RMSE-A, and of the test data of the
 * prediction task, RMSE-P; Section "Evaluation": 20% of the entries are
 * masked uniformly at random and used as the test set):
 *   RMSE_S = sqrt( (1/|S|) * sum over (s,t) in S of (R_st - (U (x) V)_st)^2 )
 * with S_A = the given entries (M = 1) and S_P = the held-out entries (M = 0)
 * whose true value is known (R_st is a number; a NaN marks an entry with no
 * truth).  The product entries and the difference are rounded in the mode's
 * precision like every other add / sub; squares and sums are in double,
 * each row in column order, then the rows in row order.
 * out = {RMSE-A, RMSE-P, |S_A|, |S_P|}; an empty set gives NaN.              */
void orc_rmse(int mode, int m, int n, int r, const double *R, const uint8_t *M, const double *U,
              const double *V, double *out)
{
    double *acc = (double *)malloc(sizeof(double) * 4 * (size_t)(m > 0 ? m : 1));
#pragma omp parallel for schedule(static)
    for (int s = 0; s < m; ++s) {
        double sa = 0.0, sp = 0.0, na = 0.0, np = 0.0;
        for (int t = 0; t < n; ++t) {
            const double x = R[(size_t)s * n + t];
            const int given = M[(size_t)s * n + t] != 0;
            if (!given && x != x) continue;
            double best = -INFINITY;
            for (int l = 0; l < r; ++l) {
                double y = add_(mode, U[(size_t)s * r + l], V[(size_t)l * n + t]);
                if (y > best) best = y;
            }
            const double d = sub_(mode, x, best);
            if (given) { sa += d * d; na += 1.0; }
            else { sp += d * d; np += 1.0; }
        }
        acc[4 * (size_t)s + 0] = sa; acc[4 * (size_t)s + 1] = sp;
        acc[4 * (size_t)s + 2] = na; acc[4 * (size_t)s + 3] = np;
    }
    double sa = 0.0, sp = 0.0, na = 0.0, np = 0.0;
    for (int s = 0; s < m; ++s) {
        sa += acc[4 * (size_t)s + 0]; sp += acc[4 * (size_t)s + 1];
        na += acc[4 * (size_t)s + 2]; np += acc[4 * (size_t)s + 3];
    }
    free(acc);
    out[0] = na > 0.0 ? sqrt(sa / na) : NAN;
    out[1] = np > 0.0 ? sqrt(sp / np) : NAN;
    out[2] = na;
    out[3] = np;
}

static void get_col(int m, int r, const double *U, int k, double *u)
{
    for (int s = 0; s < m; ++s) u[s] = U[(size_t)s * r + k];
}
static void set_col(int m, int r, double *U, int k, const double *u)
{
    for (int s = 0; s < m; ++s) U[(size_t)s * r + k] = u[s];
}

/* F-ULF (Algorithm 1), in place on U and V; returns the new error.
 * 1. U_ik <- R_ij - V_kj
 * 2. V_k. <- (-U_.k)^T (x)* R
 * 3. U_.k <- R (x)* (-V_k.)^T
 * 4. f <- ||R - U (x) V||_b
 * The caller keeps the old U_.k, V_k. for the revert.                      */
double orc_fulf(int mode, int m, int n, int r, const double *R, const uint8_t *M,
                double *U, double *V, int i, int j, int k)
{
    double *u = (double *)malloc(sizeof(double) * (size_t)m);
    U[(size_t)i * r + k] = sub_(mode, R[(size_t)i * n + j], V[(size_t)k * n + j]);
    get_col(m, r, U, k, u);
    orc_residuate_v(mode, m, n, R, M, u, V + (size_t)k * n);
    orc_residuate_u(mode, m, n, R, M, V + (size_t)k * n, u);
    set_col(m, r, U, k, u);
    free(u);
    return orc_error(mode, m, n, r, R, M, U, V);
}

/* F-URF (Algorithm 2), in place; returns the new error.
 * 1. V_kj <- R_ij - U_ik
 * 2. U_.k <- R (x)* (-V_k.)^T
 * 3. V_k. <- (-U_.k)^T (x)* R
 * 4. f <- ||R - U (x) V||_b                                                 */
double orc_furf(int mode, int m, int n, int r, const double *R, const uint8_t *M,
                double *U, double *V, int i, int j, int k)
{
    double *u = (double *)malloc(sizeof(double) * (size_t)m);
    V[(size_t)k * n + j] = sub_(mode, R[(size_t)i * n + j], U[(size_t)i * r + k]);
    orc_residuate_u(mode, m, n, R, M, V + (size_t)k * n, u);
    set_col(m, r, U, k, u);
    orc_residuate_v(mode, m, n, R, M, u, V + (size_t)k * n);
    free(u);
    return orc_error(mode, m, n, r, R, M, U, V);
}

/* Selection statistics for row i (Section "The ByRow strategy"; Algorithm 3):
 *   td(s,t)    = |R_st - max_l(U_sl + V_lt)|             (tropical distance)
 *   td_col[t]  = sum over s of td(s,t)                     (err of ByRow)
 *   colhist[t*r+l] = count of l in the multiset {f(s,t)}_s
 *   rowhist[l]     = count of l in the multiset {f(i,t)}_t
 * Reading: td is defined where R is given, so every sum and multiset runs
 * over given entries only.  td_col is summed in double in row order.       */
void orc_row_stats(int mode, int m, int n, int r, const double *R, const uint8_t *M,
                   const double *U, const double *V, int i, double *td_col,
                   int32_t *colhist, int32_t *rowhist)
{
    double *P1 = (double *)malloc(sizeof(double) * (size_t)m * n);
    int32_t *A = (int32_t *)malloc(sizeof(int32_t) * (size_t)m * n);
    orc_maxplus(mode, m, n, r, U, V, P1, A, NULL);
    for (int t = 0; t < n; ++t) {
        td_col[t] = 0.0;
        for (int l = 0; l < r; ++l) colhist[(size_t)t * r + l] = 0;
    }
    for (int l = 0; l < r; ++l) rowhist[l] = 0;
    for (int s = 0; s < m; ++s)
        for (int t = 0; t < n; ++t) {
            size_t e = (size_t)s * n + t;
            if (!M[e]) continue;
            td_col[t] += fabs(sub_(mode, R[e], P1[e]));
            colhist[(size_t)t * r + A[e]] += 1;
            if (s == i) rowhist[A[e]] += 1;
        }
    free(P1);
    free(A);
}

/* Selections of (j, k) for a fixed row i (Section "The ByRow strategy"):
 *   ORC_SEL_TD_A  columns by err = td_col descending; k = the component that
 *                 occurs most often in {f(i,t)}_t  union  {f(t,j)}_t
 *                 (Algorithm 3, the method's default);
 *   ORC_SEL_TD_B  columns as TD_A; k from the worst entry of row i and of
 *                 column j:  j0 = argmax_t td(i,t), i0 = argmax_s td(s,j),
 *                 k = f(i,j0) if (U(x)V)_{i j0} >= (U(x)V)_{i0 j}, else f(i0,j);
 *   ORC_SEL_TD    columns by their own tropical distance td(i,j) descending;
 *                 k = f(i,j);
 *   ORC_SEL_SEQ   columns in increasing j and, for each, k = 0, 1, ..., r-1.
 * f(s,t) = smallest l attaining max_l (U_sl + V_lt) (Section "The ByRow
 * strategy").  Readings: only j with R_ij given are candidates; td and the
 * multisets run over given entries only; every sort is stable on an
 * increasing list (equal keys keep the smaller index first); every argmax
 * keeps the smaller index on ties; TD_B's argmaxes are taken over the
 * entry-wise td of row i and of column j (as printed, err of ByRow is td_col
 * and does not depend on the row, so its argmax over rows would be
 * degenerate).  Returns the number of (j, k) pairs; js/ks (capacity n, or
 * n * r for SEQ) receive them in order.  Each pair is tried as F-ULF, then
 * F-URF.                                                                     */
int orc_row_order_sel(int mode, int sel, int m, int n, int r, const double *R, const uint8_t *M,
                      const double *U, const double *V, int i, int32_t *js, int32_t *ks)
{
    double *P1 = (double *)malloc(sizeof(double) * (size_t)m * n);
    int32_t *A = (int32_t *)malloc(sizeof(int32_t) * (size_t)m * n);
    double *td = (double *)malloc(sizeof(double) * (size_t)m * n);
    orc_maxplus(mode, m, n, r, U, V, P1, A, NULL);
    for (size_t e = 0; e < (size_t)m * n; ++e) td[e] = M[e] ? fabs(sub_(mode, R[e], P1[e])) : 0.0;
    const double *tdi = td + (size_t)i * n;
    int cnt = 0;
    if (sel == ORC_SEL_SEQ) {
        for (int j = 0; j < n; ++j)
            if (M[(size_t)i * n + j])
                for (int k = 0; k < r; ++k) { js[cnt] = j; ks[cnt] = k; ++cnt; }
        free(P1); free(A); free(td);
        return cnt;
    }
    for (int j = 0; j < n; ++j)
        if (M[(size_t)i * n + j]) js[cnt++] = j;
    if (sel == ORC_SEL_TD) {
        for (int a = 1; a < cnt; ++a) {            /* stable insertion sort, td(i,j) descending */
            int32_t x = js[a];
            int b = a - 1;
            while (b >= 0 && tdi[js[b]] < tdi[x]) { js[b + 1] = js[b]; --b; }
            js[b + 1] = x;
        }
        for (int a = 0; a < cnt; ++a) ks[a] = A[(size_t)i * n + js[a]];
        free(P1); free(A); free(td);
        return cnt;
    }
    /* TD_A and TD_B: td_col over given entries, summed in row order */
    double *td_col = (double *)calloc((size_t)n, sizeof(double));
    for (int s = 0; s < m; ++s)
        for (int t = 0; t < n; ++t)
            if (M[(size_t)s * n + t]) td_col[t] += td[(size_t)s * n + t];
    for (int a = 1; a < cnt; ++a) {                /* stable insertion sort, td_col descending */
        int32_t x = js[a];
        int b = a - 1;
        while (b >= 0 && td_col[js[b]] < td_col[x]) { js[b + 1] = js[b]; --b; }
        js[b + 1] = x;
    }
    if (sel == ORC_SEL_TD_A) {
        int32_t *colhist = (int32_t *)calloc((size_t)n * r, sizeof(int32_t));
        int32_t *rowhist = (int32_t *)calloc((size_t)r, sizeof(int32_t));
        for (int s = 0; s < m; ++s)
            for (int t = 0; t < n; ++t) {
                size_t e = (size_t)s * n + t;
                if (!M[e]) continue;
                colhist[(size_t)t * r + A[e]] += 1;
                if (s == i) rowhist[A[e]] += 1;
            }
        for (int a = 0; a < cnt; ++a) {
            int j = js[a], best = 0;
            int32_t bestc = -1;
            for (int l = 0; l < r; ++l) {
                int32_t c = rowhist[l] + colhist[(size_t)j * r + l];
                if (c > bestc) { bestc = c; best = l; }
            }
            ks[a] = best;
        }
        free(colhist); free(rowhist);
    } else {                                       /* TD_B */
        int j0 = -1;
        for (int t = 0; t < n; ++t)
            if (M[(size_t)i * n + t] && (j0 < 0 || tdi[t] > tdi[j0])) j0 = t;
        for (int a = 0; a < cnt; ++a) {
            int j = js[a], i0 = -1;
            for (int s = 0; s < m; ++s)
                if (M[(size_t)s * n + j] && (i0 < 0 || td[(size_t)s * n + j] > td[(size_t)i0 * n + j])) i0 = s;
            ks[a] = P1[(size_t)i * n + j0] >= P1[(size_t)i0 * n + j] ? A[(size_t)i * n + j0]
                                                                      : A[(size_t)i0 * n + j];
        }
    }
    free(td_col); free(P1); free(A); free(td);
    return cnt;
}

/* Candidate order for row i of Algorithm 3 (TD_A).                          */
int orc_row_order(int mode, int m, int n, int r, const double *R, const uint8_t *M,
                  const double *U, const double *V, int i, int32_t *js, int32_t *ks)
{
    return orc_row_order_sel(mode, ORC_SEL_TD_A, m, n, r, R, M, U, V, i, js, ks);
}

/* One ByRow step on row i (Algorithm 3, body of the row loop) with the
 * selection sel.  Reading of the garbled nesting: for each (j, k) in order,
 * try F-ULF(i,j,k); if the error decreased keep it and end the row, else
 * revert and try F-URF(i,j,k) the same way, else revert and go to the next
 * pair.  "Decreases" is strict: f' < f.  On return *f holds the current
 * error; out = {position in order, j, k, type (0 = F-ULF, 1 = F-URF)} of the
 * kept update; *tried counts the candidates evaluated (both types count).
 * Returns 1 if an update was kept, 0 if the row is left unchanged.         */
int orc_row_step_sel(int mode, int sel, int m, int n, int r, const double *R, const uint8_t *M,
                     double *U, double *V, int i, double *f, int32_t *out, int64_t *tried)
{
    const size_t cap = (size_t)n * (sel == ORC_SEL_SEQ ? r : 1);
    int32_t *js = (int32_t *)malloc(sizeof(int32_t) * cap);
    int32_t *ks = (int32_t *)malloc(sizeof(int32_t) * cap);
    double *ucol = (double *)malloc(sizeof(double) * (size_t)m);
    double *vrow = (double *)malloc(sizeof(double) * (size_t)n);
    int cnt = orc_row_order_sel(mode, sel, m, n, r, R, M, U, V, i, js, ks);
    int kept = 0;
    for (int a = 0; a < cnt && !kept; ++a) {
        int j = js[a], k = ks[a];
        for (int type = 0; type < 2; ++type) {
            get_col(m, r, U, k, ucol);
            memcpy(vrow, V + (size_t)k * n, sizeof(double) * (size_t)n);
            double fn = type == 0 ? orc_fulf(mode, m, n, r, R, M, U, V, i, j, k)
                                  : orc_furf(mode, m, n, r, R, M, U, V, i, j, k);
            if (tried) *tried += 1;
            if (fn < *f) {
                *f = fn;
                if (out) { out[0] = a; out[1] = j; out[2] = k; out[3] = type; }
                kept = 1;
                break;
            }
            set_col(m, r, U, k, ucol);
            memcpy(V + (size_t)k * n, vrow, sizeof(double) * (size_t)n);
        }
    }
    if (!kept && out) { out[0] = -1; out[1] = -1; out[2] = -1; out[3] = -1; }
    free(js); free(ks); free(ucol); free(vrow);
    return kept;
}

int orc_row_step(int mode, int m, int n, int r, const double *R, const uint8_t *M,
                 double *U, double *V, int i, double *f, int32_t *out, int64_t *tried)
{
    return orc_row_step_sel(mode, ORC_SEL_TD_A, m, n, r, R, M, U, V, i, f, out, tried);
}

/* Random Acol initialisation of U (Section "Comparison of strategies"):
 * U_sl = mean of the given entries R_s,c over the picked columns c of
 * component l.  Readings: the sum runs over the picks in order; if none of
 * the picks is given in row s, U_sl is the mean of the given entries of row
 * s (summed in column order).                                               */
void orc_acol_init(int mode, int m, int n, int r, const double *R, const uint8_t *M,
                   const int32_t *picks, int p, double *U)
{
    for (int s = 0; s < m; ++s)
        for (int l = 0; l < r; ++l) {
            double sum = 0.0;
            int cnt = 0;
            for (int q = 0; q < p; ++q) {
                int c = picks[l * p + q];
                if (M[(size_t)s * n + c]) { sum = add_(mode, sum, R[(size_t)s * n + c]); ++cnt; }
            }
            if (cnt == 0) {
                for (int t = 0; t < n; ++t)
                    if (M[(size_t)s * n + t]) { sum = add_(mode, sum, R[(size_t)s * n + t]); ++cnt; }
            }
            U[(size_t)s * r + l] = cnt ? div_(mode, sum, (double)cnt) : 0.0;
        }
}

/* Preparation steps of Algorithm 3 before the loop:
 *   if R is not wide, transpose it (Reading: square counts as wide);
 *   perm <- random permutation, R <- R[perm, :];
 *   initialise U (Random Acol, or the caller's U0 given in the oriented,
 *   permuted frame), then compute V = (-U)^T (x)* R (Reading of "compute V").
 * Outputs the oriented, permuted problem: Ri, Mi (m x n with m <= n), Ui, Vi,
 * perm_out, and *transposed.  perm_in / picks_in may be NULL (then drawn from
 * seed).  Returns the number of empty rows + columns (must be 0).           */
int orc_prepare(int mode, int m0, int n0, int r, const double *R0, const uint8_t *M0,
                const int32_t *perm_in, const int32_t *picks_in, int p, uint64_t seed,
                const double *U0, double *Ri, uint8_t *Mi, double *Ui, double *Vi,
                int32_t *perm_out, int *transposed)
{
    int tr = m0 > n0;
    int m = tr ? n0 : m0, n = tr ? m0 : n0;
    *transposed = tr;
    if (perm_in) memcpy(perm_out, perm_in, sizeof(int32_t) * (size_t)m);
    else orc_randperm(m, seed, perm_out);
    for (int s = 0; s < m; ++s)
        for (int t = 0; t < n; ++t) {
            int so = perm_out[s];
            size_t src = tr ? (size_t)t * n0 + so : (size_t)so * n0 + t;
            Ri[(size_t)s * n + t] = R0[src];
            Mi[(size_t)s * n + t] = M0[src];
        }
    if (U0) {
        memcpy(Ui, U0, sizeof(double) * (size_t)m * r);
    } else {
        int32_t *pk = (int32_t *)malloc(sizeof(int32_t) * (size_t)r * p);
        if (picks_in) memcpy(pk, picks_in, sizeof(int32_t) * (size_t)r * p);
        else orc_acol_picks(n, r, p, seed, pk);
        orc_acol_init(mode, m, n, r, Ri, Mi, pk, p, Ui);
        free(pk);
    }
    double *u = (double *)malloc(sizeof(double) * (size_t)m);
    int empty = 0;
    for (int l = 0; l < r; ++l) {
        get_col(m, r, Ui, l, u);
        empty += orc_residuate_v(mode, m, n, Ri, Mi, u, Vi + (size_t)l * n);
    }
    empty += orc_residuate_u(mode, m, n, Ri, Mi, Vi, u); /* checks rows only */
    free(u);
    return empty;
}

/* Post-processing of Algorithm 3: undo the permutation and the transpose.
 *   not transposed: U_out[perm[s], :] = Ui[s, :], V_out = Vi
 *   transposed:     U_out = Vi^T (m0 x r),  V_out[:, perm[s]] = Ui[s, :]^T  */
void orc_finish(int m0, int n0, int r, int transposed, const double *Ui, const double *Vi,
                const int32_t *perm, double *U_out, double *V_out)
{
    if (!transposed) {
        int m = m0, n = n0;
        for (int s = 0; s < m; ++s)
            for (int l = 0; l < r; ++l) U_out[(size_t)perm[s] * r + l] = Ui[(size_t)s * r + l];
        memcpy(V_out, Vi, sizeof(double) * (size_t)r * n);
    } else {
        int m = n0, n = m0;
        for (int a = 0; a < n; ++a)
            for (int l = 0; l < r; ++l) U_out[(size_t)a * r + l] = Vi[(size_t)l * n + a];
        for (int s = 0; s < m; ++s)
            for (int l = 0; l < r; ++l) V_out[(size_t)l * n0 + perm[s]] = Ui[(size_t)s * r + l];
    }
}

/* FastSTMF, Algorithm 3 (STMF_ByRow_RandPerm_TD_A_W), with the row's
 * selection sel (ORC_SEL_*; TD_A is the published method).
 * Sweeps over all rows; stops after `sweeps` sweeps, or earlier when
 * eps > 0 and the error changed by less than eps over a sweep (Section
 * "Comparison of strategies": convergence when the change in error is below
 * a threshold).  f_hist (nullable) receives sweeps+1 errors (initial, then
 * after each sweep; unused tail left as is).  trace (nullable, capacity
 * trace_cap records of 6 int32) receives one record per row visit:
 * {sweep, row, position, j, k, type} (position = -1 when nothing was kept).
 * counters (nullable) = {sweeps done, candidates tried, updates kept,
 * trace records written}.  Returns the number of empty rows + columns found
 * (0 on success; the run is skipped otherwise).                             */
int orc_factorize_sel(int mode, int sel, int m0, int n0, int r, const double *R0, const uint8_t *M0,
                      int sweeps, double eps, const int32_t *perm_in, const int32_t *picks_in,
                      int p, uint64_t seed, const double *U0, double *U_out, double *V_out,
                      double *f_hist, int32_t *trace, int64_t trace_cap, int64_t *counters)
{
    int tr = m0 > n0;
    int m = tr ? n0 : m0, n = tr ? m0 : n0;
    double *Ri = (double *)malloc(sizeof(double) * (size_t)m * n);
    uint8_t *Mi = (uint8_t *)malloc((size_t)m * n);
    double *Ui = (double *)malloc(sizeof(double) * (size_t)m * r);
    double *Vi = (double *)malloc(sizeof(double) * (size_t)r * n);
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
    int transposed = 0;
    int empty = orc_prepare(mode, m0, n0, r, R0, M0, perm_in, picks_in, p, seed, U0, Ri, Mi,
                            Ui, Vi, perm, &transposed);
    int64_t tried = 0, kept = 0, nrec = 0;
    int done = 0;
    if (empty == 0) {
        double f = orc_error(mode, m, n, r, Ri, Mi, Ui, Vi);
        if (f_hist) f_hist[0] = f;
        for (int sw = 0; sw < sweeps; ++sw) {
            double f_prev = f;
            for (int i = 0; i < m; ++i) {
                int32_t out[4];
                kept += orc_row_step_sel(mode, sel, m, n, r, Ri, Mi, Ui, Vi, i, &f, out, &tried);
                if (trace && nrec < trace_cap) {
                    int32_t *rec = trace + 6 * nrec;
                    rec[0] = sw; rec[1] = i; rec[2] = out[0]; rec[3] = out[1];
                    rec[4] = out[2]; rec[5] = out[3];
                    ++nrec;
                }
            }
            ++done;
            if (f_hist) f_hist[sw + 1] = f;
            if (eps > 0.0 && fabs(f_prev - f) < eps) break;
        }
        orc_finish(m0, n0, r, transposed, Ui, Vi, perm, U_out, V_out);
    }
    if (counters) { counters[0] = done; counters[1] = tried; counters[2] = kept; counters[3] = nrec; }
    free(Ri); free(Mi); free(Ui); free(Vi); free(perm);
    return empty;
}

/* Algorithm 3 with the TD_A selection (the method as published).           */
int orc_factorize(int mode, int m0, int n0, int r, const double *R0, const uint8_t *M0,
                  int sweeps, double eps, const int32_t *perm_in, const int32_t *picks_in,
                  int p, uint64_t seed, const double *U0, double *U_out, double *V_out,
                  double *f_hist, int32_t *trace, int64_t trace_cap, int64_t *counters)
{
    return orc_factorize_sel(mode, ORC_SEL_TD_A, m0, n0, r, R0, M0, sweeps, eps, perm_in, picks_in, p, seed,
                             U0, U_out, V_out, f_hist, trace, trace_cap, counters);
}

/* ------------------------------------------------------------------------
 * STMF_ByElement_PermC_TD_W (Section "The ByElement strategy"; its
 * pseudocode in the Supplement).
 * ---------------------------------------------------------------------- */

/* PermC (Section "Comparison of strategies"): the columns in increasing order
 * of their minimum value.  Reading: the minimum runs over given entries, and
 * equal minima keep the smaller column first (a stable sort of 0..n-1).     */
void orc_colmin_perm(int m, int n, const double *R, const uint8_t *M, int32_t *cperm)
{
    double *mn = (double *)malloc(sizeof(double) * (size_t)n);
    for (int t = 0; t < n; ++t) {
        mn[t] = INFINITY;
        for (int s = 0; s < m; ++s)
            if (M[(size_t)s * n + t] && R[(size_t)s * n + t] < mn[t]) mn[t] = R[(size_t)s * n + t];
        cperm[t] = t;
    }
    for (int a = 1; a < n; ++a) {                  /* stable insertion sort, ascending */
        int32_t x = cperm[a];
        int b = a - 1;
        while (b >= 0 && mn[cperm[b]] > mn[x]) { cperm[b + 1] = cperm[b]; --b; }
        cperm[b + 1] = x;
    }
    free(mn);
}

/* The ByElement scan from element position q0 = i*n + j (row-major): every
 * element with R_ij given and err = td(i,j) > 0 on the current state is tried
 * once, with k = f(i,j): F-ULF; if the error decreased keep it, else revert
 * and try F-URF; if that decreased keep it, else revert.  Elements with
 * err = 0 are skipped.  Returns at the first kept update, with *f the new
 * error and out = {q, i, j, k, type}; returns -1 (state and *f unchanged) when
 * the scan reaches the end of the matrix.  *tried counts the candidates.     */
int orc_element_scan(int mode, int m, int n, int r, const double *R, const uint8_t *M,
                     double *U, double *V, int q0, double *f, int32_t *out, int64_t *tried)
{
    double *ucol = (double *)malloc(sizeof(double) * (size_t)m);
    double *vrow = (double *)malloc(sizeof(double) * (size_t)n);
    int found = -1;
    for (int q = q0; q < m * n && found < 0; ++q) {
        const int i = q / n, j = q % n;
        if (!M[q]) continue;
        double best = -INFINITY;
        int k = 0;
        for (int l = 0; l < r; ++l) {              /* f(i,j): the smaller l on ties */
            double x = add_(mode, U[(size_t)i * r + l], V[(size_t)l * n + j]);
            if (x > best) { best = x; k = l; }
        }
        if (fabs(sub_(mode, R[q], best)) == 0.0) continue;   /* err = 0: skipped */
        for (int type = 0; type < 2; ++type) {
            get_col(m, r, U, k, ucol);
            memcpy(vrow, V + (size_t)k * n, sizeof(double) * (size_t)n);
            double fn = type == 0 ? orc_fulf(mode, m, n, r, R, M, U, V, i, j, k)
                                  : orc_furf(mode, m, n, r, R, M, U, V, i, j, k);
            if (tried) *tried += 1;
            if (fn < *f) {
                *f = fn;
                out[0] = q; out[1] = i; out[2] = j; out[3] = k; out[4] = type;
                found = q;
                break;
            }
            set_col(m, r, U, k, ucol);
            memcpy(V + (size_t)k * n, vrow, sizeof(double) * (size_t)n);
        }
    }
    free(ucol); free(vrow);
    return found;
}

/* The whole ByElement method.  If R is not wide it is transposed (square
 * counts as wide); its columns are then ordered by PermC and its rows keep
 * their order; U is initialised (Random Acol over the permuted columns, or
 * the caller's U0 in that frame) and V = (-U)^T (x)* R.  Each sweep scans all
 * elements once (orc_element_scan from position 0, then from just after
 * each kept update); the loop stops after `sweeps` sweeps, or earlier when
 * eps > 0 and a sweep changed the error by less than eps.  The output undoes
 * the column order and the transpose.  trace (nullable, 6 int32 per record):
 * {sweep, i, q, j, k, type} per kept update and {sweep, -1, -1, -1, -1, -1}
 * at the end of each sweep.  counters as orc_factorize.  Returns the number of
 * empty rows + columns (0 on success).                                      */
int orc_factorize_byelement(int mode, int m0, int n0, int r, const double *R0, const uint8_t *M0,
                            int sweeps, double eps, const int32_t *picks_in, int p, uint64_t seed,
                            const double *U0, double *U_out, double *V_out, double *f_hist,
                            int32_t *trace, int64_t trace_cap, int64_t *counters)
{
    const int tr = m0 > n0;
    const int m = tr ? n0 : m0, n = tr ? m0 : n0;
    double *Ro = (double *)malloc(sizeof(double) * (size_t)m * n);
    uint8_t *Mo = (uint8_t *)malloc((size_t)m * n);
    for (int s = 0; s < m; ++s)
        for (int t = 0; t < n; ++t) {
            size_t src = tr ? (size_t)t * n0 + s : (size_t)s * n0 + t;
            Ro[(size_t)s * n + t] = R0[src];
            Mo[(size_t)s * n + t] = M0[src];
        }
    int32_t *cperm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    orc_colmin_perm(m, n, Ro, Mo, cperm);
    double *Rc = (double *)malloc(sizeof(double) * (size_t)m * n);
    uint8_t *Mc = (uint8_t *)malloc((size_t)m * n);
    for (int s = 0; s < m; ++s)
        for (int t = 0; t < n; ++t) {
            Rc[(size_t)s * n + t] = Ro[(size_t)s * n + cperm[t]];
            Mc[(size_t)s * n + t] = Mo[(size_t)s * n + cperm[t]];
        }
    double *Ri = (double *)malloc(sizeof(double) * (size_t)m * n);
    uint8_t *Mi = (uint8_t *)malloc((size_t)m * n);
    double *Ui = (double *)malloc(sizeof(double) * (size_t)m * r);
    double *Vi = (double *)malloc(sizeof(double) * (size_t)r * n);
    int32_t *ident = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
    int32_t *perm_out = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
    for (int s = 0; s < m; ++s) ident[s] = s;
    int wide_again = 0;
    int empty = orc_prepare(mode, m, n, r, Rc, Mc, ident, picks_in, p, seed, U0, Ri, Mi, Ui, Vi, perm_out,
                            &wide_again);
    int64_t tried = 0, kept = 0, nrec = 0;
    int done = 0;
    if (empty == 0) {
        double f = orc_error(mode, m, n, r, Ri, Mi, Ui, Vi);
        if (f_hist) f_hist[0] = f;
        for (int sw = 0; sw < sweeps; ++sw) {
            double f_prev = f;
            int q = 0;
            for (;;) {
                int32_t out[5];
                int got = orc_element_scan(mode, m, n, r, Ri, Mi, Ui, Vi, q, &f, out, &tried);
                int32_t rec[6] = {sw, -1, -1, -1, -1, -1};
                if (got >= 0) {
                    ++kept;
                    rec[1] = out[1]; rec[2] = out[0]; rec[3] = out[2]; rec[4] = out[3]; rec[5] = out[4];
                }
                if (trace && nrec < trace_cap) memcpy(trace + 6 * nrec, rec, sizeof(rec));
                ++nrec;
                if (got < 0) break;
                q = got + 1;
            }
            ++done;
            if (f_hist) f_hist[sw + 1] = f;
            if (eps > 0.0 && fabs(f_prev - f) < eps) break;
        }
        /* undo the column order, then the transpose */
        if (!tr) {
            memcpy(U_out, Ui, sizeof(double) * (size_t)m * r);
            for (int l = 0; l < r; ++l)
                for (int t = 0; t < n; ++t) V_out[(size_t)l * n + cperm[t]] = Vi[(size_t)l * n + t];
        } else {
            for (int t = 0; t < n; ++t)
                for (int l = 0; l < r; ++l) U_out[(size_t)cperm[t] * r + l] = Vi[(size_t)l * n + t];
            for (int s = 0; s < m; ++s)
                for (int l = 0; l < r; ++l) V_out[(size_t)l * n0 + s] = Ui[(size_t)s * r + l];
        }
    }
    if (trace_cap < nrec) nrec = trace_cap;
    if (counters) { counters[0] = done; counters[1] = tried; counters[2] = kept; counters[3] = nrec; }
    free(Ro); free(Mo); free(cperm); free(Rc); free(Mc); free(Ri); free(Mi); free(Ui); free(Vi);
    free(ident); free(perm_out);
    return empty;
}

/* ------------------------------------------------------------------------
 * STMF_ByMatrix_NoPerm_TD_W (Section "The ByMatrix strategy"; its
 * pseudocode in the Supplement).
 * ---------------------------------------------------------------------- */

/* The coin of "random() < 0.5" (Reading: one fair coin per iteration and
 * element, drawn from SplitMix64 keyed by seed ^ 0x5A5A...5A at counter
 * it * m * n + q; the top bit 0 chooses F-ULF, 1 F-URF).                    */
int orc_matrix_coin(uint64_t seed, int64_t it, int m, int n, int q)
{
    uint64_t c = (uint64_t)it * (uint64_t)m * (uint64_t)n + (uint64_t)q;
    return (int)(orc_splitmix64(seed ^ 0x5A5A5A5A5A5A5A5Aull, c) >> 63);
}

typedef struct { double err; int32_t q; } orc_err_item;

static int cmp_err_desc(const void *a, const void *b)
{
    const orc_err_item *x = (const orc_err_item *)a, *y = (const orc_err_item *)b;
    if (x->err != y->err) return x->err > y->err ? -1 : 1;   /* decreasing err */
    return x->q < y->q ? -1 : (x->q > y->q);                  /* then smaller q */
}

/* The ByMatrix order of one iteration: every given element (i, j) with
 *   err(i,j) = td_row(i) + td_col(j) - td(i,j)
 * (td over given entries; td_row and td_col summed in double in index order;
 * err evaluated as (td_row + td_col) - td in double), sorted by decreasing
 * err, equal err keeping the smaller q = i*n + j first; each with k = f(i,j)
 * and the iteration's coin.  Returns the count; qs, ks, types, errs
 * (nullable) receive them in order.                                         */
int orc_matrix_order(int mode, int m, int n, int r, const double *R, const uint8_t *M, const double *U,
                     const double *V, uint64_t seed, int64_t it, int32_t *qs, int32_t *ks, int32_t *types,
                     double *errs)
{
    double *P1 = (double *)malloc(sizeof(double) * (size_t)m * n);
    int32_t *A = (int32_t *)malloc(sizeof(int32_t) * (size_t)m * n);
    double *td = (double *)malloc(sizeof(double) * (size_t)m * n);
    double *tdr = (double *)calloc((size_t)m, sizeof(double));
    double *tdc = (double *)calloc((size_t)n, sizeof(double));
    orc_maxplus(mode, m, n, r, U, V, P1, A, NULL);
    for (size_t e = 0; e < (size_t)m * n; ++e) td[e] = M[e] ? fabs(sub_(mode, R[e], P1[e])) : 0.0;
    for (int s = 0; s < m; ++s)
        for (int t = 0; t < n; ++t)
            if (M[(size_t)s * n + t]) tdr[s] += td[(size_t)s * n + t];
    for (int t = 0; t < n; ++t)
        for (int s = 0; s < m; ++s)
            if (M[(size_t)s * n + t]) tdc[t] += td[(size_t)s * n + t];
    orc_err_item *it_ = (orc_err_item *)malloc(sizeof(orc_err_item) * (size_t)m * n);
    int cnt = 0;
    for (int q = 0; q < m * n; ++q)
        if (M[q]) {
            it_[cnt].err = (tdr[q / n] + tdc[q % n]) - td[q];
            it_[cnt].q = q;
            ++cnt;
        }
    qsort(it_, (size_t)cnt, sizeof(orc_err_item), cmp_err_desc);
    for (int a = 0; a < cnt; ++a) {
        qs[a] = it_[a].q;
        ks[a] = A[it_[a].q];
        types[a] = orc_matrix_coin(seed, it, m, n, it_[a].q);
        if (errs) errs[a] = it_[a].err;
    }
    free(P1); free(A); free(td); free(tdr); free(tdc); free(it_);
    return cnt;
}

/* One ByMatrix iteration: in the order of orc_matrix_order, apply the
 * element's update (F-ULF or F-URF by its coin); keep the first that lowers
 * the error (strictly) and end the iteration, else revert and go on.
 * out = {position, i, j, k, type}; returns 1 if an update was kept.         */
int orc_matrix_step(int mode, int m, int n, int r, const double *R, const uint8_t *M, double *U, double *V,
                    uint64_t seed, int64_t it, double *f, int32_t *out, int64_t *tried)
{
    int32_t *qs = (int32_t *)malloc(sizeof(int32_t) * (size_t)m * n);
    int32_t *ks = (int32_t *)malloc(sizeof(int32_t) * (size_t)m * n);
    int32_t *ty = (int32_t *)malloc(sizeof(int32_t) * (size_t)m * n);
    double *ucol = (double *)malloc(sizeof(double) * (size_t)m);
    double *vrow = (double *)malloc(sizeof(double) * (size_t)n);
    int cnt = orc_matrix_order(mode, m, n, r, R, M, U, V, seed, it, qs, ks, ty, NULL);
    int kept = 0;
    for (int a = 0; a < cnt && !kept; ++a) {
        const int i = qs[a] / n, j = qs[a] % n, k = ks[a];
        get_col(m, r, U, k, ucol);
        memcpy(vrow, V + (size_t)k * n, sizeof(double) * (size_t)n);
        double fn = ty[a] == 0 ? orc_fulf(mode, m, n, r, R, M, U, V, i, j, k)
                               : orc_furf(mode, m, n, r, R, M, U, V, i, j, k);
        if (tried) *tried += 1;
        if (fn < *f) {
            *f = fn;
            out[0] = a; out[1] = i; out[2] = j; out[3] = k; out[4] = ty[a];
            kept = 1;
        } else {
            set_col(m, r, U, k, ucol);
            memcpy(V + (size_t)k * n, vrow, sizeof(double) * (size_t)n);
        }
    }
    if (!kept) { out[0] = -1; out[1] = -1; out[2] = -1; out[3] = -1; out[4] = -1; }
    free(qs); free(ks); free(ty); free(ucol); free(vrow);
    return kept;
}

/* The whole ByMatrix method: R oriented wide (square counts as wide), no
 * permutation, U initialised (Random Acol, or U0 in the oriented frame) and
 * V = (-U)^T (x)* R; then `iterations` iterations of orc_matrix_step (each
 * keeps at most one update), stopping earlier when eps > 0 and an iteration
 * changed the error by less than eps.  trace (nullable, 6 int32 per record):
 * {iteration, i, position, j, k, type} per iteration (position -1: nothing
 * kept).  counters as orc_factorize.                                        */
int orc_factorize_bymatrix(int mode, int m0, int n0, int r, const double *R0, const uint8_t *M0,
                           int iterations, double eps, const int32_t *picks_in, int p, uint64_t seed,
                           const double *U0, double *U_out, double *V_out, double *f_hist,
                           int32_t *trace, int64_t trace_cap, int64_t *counters)
{
    const int tr = m0 > n0;
    const int m = tr ? n0 : m0, n = tr ? m0 : n0;
    double *Ri = (double *)malloc(sizeof(double) * (size_t)m * n);
    uint8_t *Mi = (uint8_t *)malloc((size_t)m * n);
    double *Ui = (double *)malloc(sizeof(double) * (size_t)m * r);
    double *Vi = (double *)malloc(sizeof(double) * (size_t)r * n);
    int32_t *ident = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
    int32_t *perm_out = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
    for (int s = 0; s < m; ++s) ident[s] = s;
    int transposed = 0;
    int empty = orc_prepare(mode, m0, n0, r, R0, M0, ident, picks_in, p, seed, U0, Ri, Mi, Ui, Vi, perm_out,
                            &transposed);
    int64_t tried = 0, kept = 0, nrec = 0;
    int done = 0;
    if (empty == 0) {
        double f = orc_error(mode, m, n, r, Ri, Mi, Ui, Vi);
        if (f_hist) f_hist[0] = f;
        for (int it = 0; it < iterations; ++it) {
            double f_prev = f;
            int32_t out[5];
            kept += orc_matrix_step(mode, m, n, r, Ri, Mi, Ui, Vi, seed, it, &f, out, &tried);
            if (trace && nrec < trace_cap) {
                int32_t *rec = trace + 6 * nrec;
                rec[0] = it; rec[1] = out[1]; rec[2] = out[0]; rec[3] = out[2]; rec[4] = out[3]; rec[5] = out[4];
                ++nrec;
            }
            ++done;
            if (f_hist) f_hist[it + 1] = f;
            if (eps > 0.0 && fabs(f_prev - f) < eps) break;
        }
        orc_finish(m0, n0, r, transposed, Ui, Vi, ident, U_out, V_out);
    }
    if (counters) { counters[0] = done; counters[1] = tried; counters[2] = kept; counters[3] = nrec; }
    free(Ri); free(Mi); free(Ui); free(Vi); free(ident); free(perm_out);
    return empty;
}
