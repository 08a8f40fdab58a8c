// Kernels of the F-ULF / F-URF updates (Algorithms 1 and 2) and of the ByRow
// row loop of Algorithm 3, apart from the window evaluation itself
// (kernels_eval.cu): packing, initialisation, the residuation statistics,
// the candidate window, the seeds, the decision and the row-loop control.
//
// F-ULF(i,j,k) on the state (U, V):
//   seed   U''_ik = R_ij - V_kj
//   V'_kt  = min over given s of (R_st - U''_sk)
//          = min( R_it - U''_ik ,  min over s != i of (R_st - U_sk) )
//            -- O(n) from the column statistics (min1, argmin, min2) of k
//   U'_sk  = min over given t of (R_st - V'_kt)            (row pass, phase 1)
//   f'     = sum over given (s,t) of |R_st - max(E_st, U'_sk + V'_kt)|
//            with E = max over l != k of (U_sl + V_lt) = (A == k ? P2 : P1)
//            (phase 2, as the change f' - f summed per entry)
// F-URF is the mirror image (row statistics, then a column pass over RT).
//
// The seeds and the residuations are computed with the same FP32 operations
// as the plain definition, so a candidate's U', V' are bit-identical to it.
#include "common.cuh"

#define QNAN __int_as_float(0x7fffffff)
#define FULL 0xffffffffu

// ------------------------------------------------------------------ set-up

// Rp[s][t] = given ? R[s][t] : NaN over the padded mp x ldp area.
__global__ void k_pack(const float *__restrict__ R, int ldr, const uint32_t *__restrict__ mask, int ldm,
                       int m, int n, float *__restrict__ Rp, int ldp, int mp, int *__restrict__ bad)
{
    const int t = blockIdx.x * 32 + threadIdx.x;
    const int s = blockIdx.y * 8 + threadIdx.y;
    if (s >= mp || t >= ldp) return;
    float v = QNAN;
    if (s < m && t < n) {
        const bool given = mask ? ((mask[(size_t)s * ldm + (t >> 5)] >> (t & 31)) & 1u) : true;
        if (given) {
            v = R[(size_t)s * ldr + t];
            if (!(fabsf(v) < STMF_R_LIMIT)) { atomicOr(bad, 1); v = QNAN; }   // not finite, or too large
        }
    }
    Rp[(size_t)s * ldp + t] = v;
}

// Oriented, permuted copy: Rp[s][t] = R0[perm[s]][c(t)], or for a transposed
// (tall) input Rp[s][t] = R0[c(t)][perm[s]], with c(t) = cperm[t] (ByElement's
// PermC) or t (cperm NULL); NaN where not given.
__global__ void k_pack_oriented(const float *__restrict__ R, int ldr, const uint32_t *__restrict__ mask,
                                int ldm, int m, int n, int transposed, const int *__restrict__ perm,
                                const int *__restrict__ cperm, float *__restrict__ Rp, int ldp, int mp,
                                int *__restrict__ bad)
{
    const int t = blockIdx.x * 32 + threadIdx.x;
    const int s = blockIdx.y * 8 + threadIdx.y;
    if (s >= mp || t >= ldp) return;
    float v = QNAN;
    if (s < m && t < n) {
        const int so = perm[s], to = cperm ? cperm[t] : t;
        const int a = transposed ? to : so, b = transposed ? so : to;   // source row, column
        const bool given = mask ? ((mask[(size_t)a * ldm + (b >> 5)] >> (b & 31)) & 1u) : true;
        if (given) {
            v = R[(size_t)a * ldr + b];
            if (!(fabsf(v) < STMF_R_LIMIT)) { atomicOr(bad, 1); v = QNAN; }   // not finite, or too large
        }
    }
    Rp[(size_t)s * ldp + t] = v;
}

// Undo the permutations and the transpose (end of Algorithm 3; the ByElement
// pseudocode), with c(t) = cperm[t] or t:
//   not transposed: U_out[perm[s], :] = U[s, :],  V_out[:, c(t)] = V[:, t]
//   transposed:     U_out[c(t), :] = V[:, t]^T,   V_out[:, perm[s]] = U[s, :]^T
__global__ void k_unorient(const float *__restrict__ U, const float *__restrict__ V, int m, int n, int r,
                           int np, int transposed, const int *__restrict__ perm, const int *__restrict__ cperm,
                           float *__restrict__ U_out, float *__restrict__ V_out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m * r) {
        const int s = e / r, l = e % r;
        if (!transposed) U_out[(size_t)perm[s] * r + l] = U[e];
        else V_out[(size_t)l * m + perm[s]] = U[e];
    }
    if (e < r * n) {
        const int l = e / n, t = e % n;
        const int c = cperm ? cperm[t] : t;
        if (!transposed) V_out[(size_t)l * n + c] = V[(size_t)l * np + t];
        else U_out[(size_t)c * r + l] = V[(size_t)l * np + t];
    }
}

// PermC keys (ByElement): the minimum given entry of every column of the
// packed R (NaN where not given, which fminf drops).  A block covers 32
// columns; its 32 warps stride over the rows.
__global__ void __launch_bounds__(1024) k_col_min(const float *__restrict__ Rp, int ldp, int m, int n,
                                                  float *__restrict__ cmin)
{
    __shared__ float red[32][33];
    const int c = threadIdx.x & 31, q = threadIdx.x >> 5;
    const int t = blockIdx.x * 32 + c;
    float x = INFINITY;
    if (t < n)
        for (int s = q; s < m; s += 32) x = fminf(x, Rp[(size_t)s * ldp + t]);
    red[q][c] = x;
    __syncthreads();
    if (q == 0 && t < n) {
        for (int z = 1; z < 32; ++z) x = fminf(x, red[z][c]);
        cmin[t] = x;
    }
}

// PermC order (ByElement): the columns by increasing minimum given entry,
// equal minima keeping the smaller column first.  Keys are the minima mapped
// to unsigned integers that order like the floats (-0 counts as +0, as in a
// float comparison); rank_t = #{e : key_e < key_t} + #{e < t : key_e = key_t},
// counted over a 2-D grid (columns x key chunks held in shared memory).
constexpr int PERMC_CHUNK = 512;
__device__ __forceinline__ unsigned ordered_key(float x)
{
    const unsigned b = __float_as_uint(x + 0.0f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__global__ void __launch_bounds__(256) k_permc_rank(const float *__restrict__ cmin, int n, int *__restrict__ rank)
{
    __shared__ unsigned sk[PERMC_CHUNK];
    const int t = blockIdx.x * 256 + threadIdx.x;
    const int base = blockIdx.y * PERMC_CHUNK;
    const int len = min(PERMC_CHUNK, n - base);
    for (int e = threadIdx.x; e < len; e += 256) sk[e] = ordered_key(cmin[base + e]);
    __syncthreads();
    if (t >= n) return;
    const unsigned kt = ordered_key(cmin[t]);
    const int tl = t - base;   // chunk-local index of t (may be outside the chunk)
    int cnt = 0;
    for (int e = 0; e < len; ++e) {
        const unsigned x = sk[e];
        cnt += (x < kt) | ((x == kt) & (e < tl));
    }
    if (cnt) atomicAdd(&rank[t], cnt);
}

__global__ void k_permc_scatter(const int *__restrict__ rank, int n, int *__restrict__ cperm)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) cperm[rank[t]] = t;
}

// Number of rows among the first `rows` that hold no given (non-NaN) entry.
__global__ void k_empty_rows(const float *__restrict__ X, int ldx, int rows, int *__restrict__ nempty)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= rows) return;
    int cnt = 0;
    for (int t = lane; t < ldx; t += 32) cnt += X[(size_t)warp * ldx + t] == X[(size_t)warp * ldx + t];
    cnt = __reduce_add_sync(FULL, cnt);
    if (lane == 0 && cnt == 0) atomicAdd(nempty, 1);
}

__global__ void k_transpose(const float *__restrict__ X, int ldx, int rows, int cols,
                            float *__restrict__ XT, int ldxt)
{
    __shared__ float tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += 8) {
        const int rr = r0 + y, cc = c0 + threadIdx.x;
        tile[y][threadIdx.x] = (rr < rows && cc < cols) ? X[(size_t)rr * ldx + cc] : QNAN;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += 8) {
        const int cc = c0 + y, rr = r0 + threadIdx.x;
        if (cc < cols && rr < rows) XT[(size_t)cc * ldxt + rr] = tile[threadIdx.x][y];
    }
}

// Random Acol (Section "Comparison of strategies"): U_sl = mean of the given
// R_s,c over the picks c of component l, summed in pick order; if none is
// given, the mean of the given entries of row s in column order.
__global__ void k_acol(const float *__restrict__ R, int ld, int m, int n, int r,
                       const int *__restrict__ picks, int p, float *__restrict__ U)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * r) return;
    const int s = e / r, l = e % r;
    const float *row = R + (size_t)s * ld;
    float sum = 0.f;
    int cnt = 0;
    for (int q = 0; q < p; ++q) {
        const float v = row[picks[l * p + q]];
        if (v == v) { sum += v; ++cnt; }
    }
    if (cnt == 0)
        for (int t = 0; t < n; ++t) {
            const float v = row[t];
            if (v == v) { sum += v; ++cnt; }
        }
    U[(size_t)s * r + l] = cnt ? sum / (float)cnt : 0.f;
}

__global__ void k_copy_rows(const float *__restrict__ src, int lds, float *__restrict__ dst, int ldd,
                            int rows, int cols)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x, s = blockIdx.y;
    if (t < cols && s < rows) dst[(size_t)s * ldd + t] = src[(size_t)s * lds + t];
}

// ---------------------------------------------------- residuation statistics

__device__ __forceinline__ void top2_push(float d, int idx, float &a1, int &ai, float &a2)
{
    // NaN (entry not given) compares false and is dropped by fminf
    if (d < a1) { a2 = a1; a1 = d; ai = idx; }
    else a2 = fminf(a2, d);
}

__device__ __forceinline__ void top2_warp_merge(float &a1, int &ai, float &a2)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const float b1 = __shfl_xor_sync(FULL, a1, o), b2 = __shfl_xor_sync(FULL, a2, o);
        const int bi = __shfl_xor_sync(FULL, ai, o);
        if (b1 < a1 || (b1 == a1 && bi < ai)) { a2 = fminf(b2, a1); a1 = b1; ai = bi; }
        else a2 = fminf(a2, b1);
    }
}

// Top-2 residuation statistics of the component(s) named by ctl->dirty_k
// (-1: every component, -2: nothing to do):
//   column statistics of k (warps 0..n-1, one row of RT each):
//     d_s = R_st - U_sk over given s; cmin1 = min d, carg = smallest s at the
//     minimum, cmin2 = min over s != carg
//   row statistics of k (warps n..n+m-1, one row of R each):
//     d_t = R_st - V_kt over given t; rmin1, rarg, rmin2 likewise.
// V'_kt of F-ULF is min(R_it - U''_ik, carg == i ? cmin2 : cmin1) and U'_sk of
// F-URF is min(R_sj - V''_kj, rarg == j ? rmin2 : rmin1): O(n) / O(m) seeds.
__global__ void __launch_bounds__(256) k_stats(stmf_problem P)
{
    const int dk = P.ctl->dirty_k;
    if (dk == -2) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= P.n + P.m) return;
    const bool col = warp < P.n;
    const int row = col ? warp : warp - P.n;
    const float4 *x4 = reinterpret_cast<const float4 *>(col ? P.RT + (size_t)row * P.mp : P.R + (size_t)row * P.np);
    const int len4 = (col ? P.mp : P.np) >> 2;
    const int l0 = dk < 0 ? 0 : dk, l1 = dk < 0 ? P.r : dk + 1;
    for (int l = l0; l < l1; ++l) {
        float a1 = INFINITY, a2 = INFINITY;
        int ai = 0x7fffffff;
        // two float4 per lane and step: independent loads in flight
        for (int f0 = lane; f0 < len4; f0 += 64) {
            float4 x[2];
            float y[2][4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int f = f0 + 32 * h;
                x[h] = f < len4 ? x4[f] : make_float4(NAN, NAN, NAN, NAN);
                if (col) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) y[h][q] = f < len4 ? P.U[(size_t)(4 * f + q) * P.r + l] : 0.f;
                } else {
                    const float4 v = f < len4 ? reinterpret_cast<const float4 *>(P.V + (size_t)l * P.np)[f]
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
                    y[h][0] = v.x; y[h][1] = v.y; y[h][2] = v.z; y[h][3] = v.w;
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int f = f0 + 32 * h;
                top2_push(x[h].x - y[h][0], 4 * f + 0, a1, ai, a2);
                top2_push(x[h].y - y[h][1], 4 * f + 1, a1, ai, a2);
                top2_push(x[h].z - y[h][2], 4 * f + 2, a1, ai, a2);
                top2_push(x[h].w - y[h][3], 4 * f + 3, a1, ai, a2);
            }
        }
        top2_warp_merge(a1, ai, a2);
        if (lane == 0) {
            if (col) {
                const size_t e = (size_t)l * P.np + row;
                P.cmin1[e] = a1; P.cmin2[e] = a2; P.carg[e] = ai;
            } else {
                const size_t e = (size_t)l * P.mp + row;
                P.rmin1[e] = a1; P.rmin2[e] = a2; P.rarg[e] = ai;
            }
        }
    }
}

// --------------------------------------------------------------- row loop

// The single-block kernels of the row loop (k_row_begin, k_select) work on a
// shared-memory copy of the control block: one coalesced load at the start
// and one store at the end replace the chain of dependent global
// read-modify-writes of its many fields.  No other kernel of the problem
// runs while they do.
constexpr int CTL_WORDS = (int)(sizeof(stmf_ctl) / sizeof(unsigned));
static_assert(sizeof(stmf_ctl) % sizeof(unsigned) == 0, "control block is not a whole number of words");

__device__ __forceinline__ void ctl_load(stmf_ctl &dst, const stmf_ctl *src)
{
    const unsigned *s = reinterpret_cast<const unsigned *>(src);
    unsigned *d = reinterpret_cast<unsigned *>(&dst);
    for (int w = threadIdx.x; w < CTL_WORDS; w += blockDim.x) d[w] = s[w];
    __syncthreads();
}

__device__ __forceinline__ void ctl_store(stmf_ctl *dst, const stmf_ctl &src)
{
    __syncthreads();
    const unsigned *s = reinterpret_cast<const unsigned *>(&src);
    unsigned *d = reinterpret_cast<unsigned *>(dst);
    for (int w = threadIdx.x; w < CTL_WORDS; w += blockDim.x) d[w] = s[w];
}

// A built window: not yet evaluated (timestamps reset), awaiting its
// decision; the next build covers twice the j-candidates, up to wmax / 2.
__device__ __forceinline__ void window_opened(stmf_win *win, stmf_ctl *ctl)
{
    win->live = 1;
    win->placeholder = 0;
    ctl->real_built += 1;
    ctl->last_ph = 0;
    win->screened = 0;
    win->ev_t0 = ~0ull;
    win->ev_t1 = 0ull;
    win->ev_r1 = 0ull;
    win->ev_d0 = ~0ull;
    ctl->wj = min(ctl->wj * 2, ctl->wmax / 2);
}

// An empty window in the pipeline (short rows): it takes no position, slot
// number or size, so the windows after it are those of the unpipelined loop;
// its evaluation does no work and its decision only moves the row on.
__device__ __forceinline__ void open_placeholder(stmf_win *win, stmf_ctl *ctl)
{
    win->nc = 0; win->na = 0; win->nu = 0; win->nv = 0;
    win->exhausted = 0;
    win->live = 1;
    win->placeholder = 1;
    win->screened = 0;
    win->ev_t0 = ~0ull; win->ev_t1 = 0ull; win->ev_r1 = 0ull; win->ev_d0 = ~0ull;
    ctl->last_ph = 1;
}

// Window of candidates (Algorithm 3; selections of Section "The ByRow
// strategy"): the next wj pairs (j, k) of the row's order with R_ij given.
//   TD_A: j along the column order (td_col descending); k_j = argmax_l
//         (rowhist_i[l] + colhist[j][l]) (the multiset union adds
//         multiplicities; smaller l on ties);
//   TD_B: j as TD_A; k_j = A[i][j0] if P1[i][j0] >= P1[i0][j] else A[i0][j],
//         j0 the row's largest td (found at the row's first window), i0 the
//         column's (from the refresh);
//   TD:   j along the row's own order (td(i, j) descending); k_j = A[i][j];
//   SEQ:  position q = j r + k, j increasing, then k.
// With the ByElement strategy the positions are the elements q = i n + j in
// row-major order, from where the scan stands (not reset per row): an
// element is a candidate when R_ij is given and td(i,j) > 0, i.e. R_ij !=
// P1_ij, with k = f(i,j) = A_ij; the window's elements may span rows.
// With the ByMatrix strategy the positions are those of the iteration's
// sorted order of the given elements (kernels_bymatrix.cu); each element is
// one candidate, F-ULF or F-URF by its coin, with k = A_ij; a window takes at
// most STMF_WMAX / 2 of them (phase 1 holds at most that many of one type).
// Otherwise each pair gives F-ULF (slot 2a) then F-URF (slot 2a+1), the
// order in which Algorithm 3 tries them.  At the first window of a row the
// row histogram (and TD_B's j0) is rebuilt.  Windows are built one ahead of
// the decisions: the position, the slot numbering (nbuilt) and the window
// size (wj, doubled after each build up to wmax / 2) belong to the builds;
// a window never depends on the decision of the one before it, only on
// whether the row goes on.  Runs in a block of 1024 threads: at the start of
// a row (k_row_begin) and in k_select after a decision that did not end the
// row; the window goes into P.win and P.cand (the buffer P points at).
__device__ __forceinline__ void build_window(const stmf_problem &P, stmf_ctl *ctl, bool row_start)
{
    stmf_win *win = P.win;
    __shared__ int sh[STMF_MAX_RANK];
    __shared__ int sj[STMF_WMAX / 2], sk[STMF_WMAX / 2], si[STMF_WMAX / 2], sq[STMF_WMAX / 2], sty[STMF_WMAX / 2];
    __shared__ int scount, spos;
    __shared__ unsigned long long sj0;
    const bool elem = P.strategy == STMF_STRATEGY_BYELEMENT, mat = P.strategy == STMF_STRATEGY_BYMATRIX;
    const int i = (elem || mat) ? 0 : ctl->i, tid = threadIdx.x, r = P.r, sel = P.sel;
    const float *Ri = P.R + (size_t)i * P.np;
    // positions of the row's order (ByElement: of the whole sweep; ByMatrix:
    // of the iteration's sorted order)
    const int lim = elem ? P.m * P.n : mat ? (int)P.ngiven : (sel == STMF_SEL_SEQ ? P.n * r : P.n);
    if (row_start && (elem || mat)) {
        if (tid == 0) { ctl->ncand_row = 0; ctl->nbuilt = 0; }
        __syncthreads();
    } else if (row_start) {
        if (tid < r) sh[tid] = 0;
        if (tid == 0) sj0 = 0ull;
        __syncthreads();
        const uint8_t *Ai = P.A + (size_t)i * P.np;
        const float *P1i = P.P1 + (size_t)i * P.np;
        unsigned long long best = 0ull;
        for (int t = tid; t < P.n; t += 1024)
            if (Ri[t] == Ri[t]) {
                atomicAdd(&sh[Ai[t]], 1);
                if (sel == STMF_SEL_TD_B) {
                    const unsigned long long key = td_argmax_key(fabsf(Ri[t] - P1i[t]), t);
                    best = key > best ? key : best;
                }
            }
        if (sel == STMF_SEL_TD_B) {
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const unsigned long long ob = __shfl_xor_sync(FULL, best, o);
                best = ob > best ? ob : best;
            }
            if ((tid & 31) == 0 && best) atomicMax(&sj0, best);
        }
        __syncthreads();
        if (tid < r) P.rowhist[tid] = sh[tid];
        if (tid == 0) {
            ctl->pos = 0;
            ctl->ncand_row = 0;
            ctl->nbuilt = 0;
            ctl->tdb_j0 = sj0 ? td_argmax_index(sj0) : 0;    // every row has a given entry (checked at set-up)
        }
        __syncthreads();
    } else if (sel == STMF_SEL_TD_A) {
        if (tid < r) sh[tid] = P.rowhist[tid];
        __syncthreads();
    }
    if (tid < 32) {
        const int want = mat ? min(2 * ctl->wj, ctl->wmax / 2) : min(ctl->wj, ctl->wmax / 2);
        int pos = ctl->pos, have = 0;
        const int lane = tid;
        const int *ord = sel == STMF_SEL_TD ? P.roworder : P.order;
        while (have < want && pos < lim) {
            const int q = pos + lane;
            int j = 0, k = 0, ei = i, ty = 0;
            bool ok = false;
            if (q < lim) {
                if (mat) {
                    const unsigned qe = P.sval[q];
                    ok = qe < (unsigned)P.m * (unsigned)P.n;   // the first ngiven of the order are the given elements
                    if (ok) {
                        ei = (int)(qe / (unsigned)P.n); j = (int)(qe - (unsigned)ei * (unsigned)P.n);
                        k = P.A[(size_t)ei * P.np + j];
                        const unsigned long long c = (unsigned long long)ctl->sweep * (unsigned long long)P.m *
                                                     (unsigned long long)P.n + qe;
                        ty = (int)(splitmix64_draw(P.coin_key, c) >> 63);
                    }
                } else if (elem) {
                    ei = q / P.n; j = q - ei * P.n;
                    const size_t e = (size_t)ei * P.np + j;
                    const float x = P.R[e];
                    ok = x == x && x != P.P1[e];         // given, and td(i,j) > 0
                    k = P.A[e];
                } else {
                    if (sel == STMF_SEL_SEQ) { j = q / r; k = q - j * r; }
                    else j = ord[q];
                    ok = Ri[j] == Ri[j];
                }
            }
            const unsigned b = __ballot_sync(FULL, ok);
            const int rank = __popc(b & ((1u << lane) - 1u));
            if (ok && have + rank < want) {
                sj[have + rank] = j; sk[have + rank] = k; si[have + rank] = ei; sq[have + rank] = q;
                sty[have + rank] = ty;
            }
            const int take = min(__popc(b), want - have);
            if (take < __popc(b)) {
                unsigned bb = b;          // stop at the first given entry not taken
                for (int z = 0; z < take; ++z) bb &= bb - 1u;
                pos += __ffs(bb) - 1;
            } else {
                pos += 32;
            }
            have += take;
        }
        if (lane == 0) { scount = have; spos = min(pos, lim); }
    }
    __syncthreads();
    const int cnt = scount;
    if (elem || mat) {
        // k = f(i,j) was read with the element
    } else if (sel == STMF_SEL_TD_A) {
        // warp a takes column a of the window; lane l loads component l's
        // count, and the warp keeps the largest (the smaller l on ties)
        const int a = tid >> 5, l = tid & 31;
        if (a < cnt) {
            const int j = sj[a];
            int c = l < r ? sh[l] + P.colhist[(size_t)j * r + l] : -1;
            int bl = l;
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const int oc = __shfl_xor_sync(FULL, c, o), ol = __shfl_xor_sync(FULL, bl, o);
                if (oc > c || (oc == c && ol < bl)) { c = oc; bl = ol; }
            }
            if (l == 0) sk[a] = bl;
        }
    } else if (sel != STMF_SEL_SEQ && tid < cnt) {
        const int j = sj[tid];
        if (sel == STMF_SEL_TD) {
            sk[tid] = P.A[(size_t)i * P.np + j];
        } else {
            const int j0 = ctl->tdb_j0, i0 = P.colarg[j];
            const size_t e0 = (size_t)i * P.np + j0, e1 = (size_t)i0 * P.np + j;
            sk[tid] = P.P1[e0] >= P.P1[e1] ? P.A[e0] : P.A[e1];
        }
    }
    __syncthreads();
    if (mat) {
        // one slot per element, in the order: j, k, type (its coin), index
        // within the iteration, screen flag, row i, position in the order
        if (tid < cnt) {
            int *c0 = P.cand + 8 * tid;
            c0[0] = sj[tid]; c0[1] = sk[tid]; c0[2] = sty[tid]; c0[3] = ctl->nbuilt + tid; c0[4] = 0;
            c0[5] = si[tid]; c0[6] = sq[tid];
        }
        if (tid == 0) {
            int idx[STMF_WMAX / 2];
            for (int a = 0; a < cnt; ++a) {          // grouped by k (stable)
                int b = a - 1;
                while (b >= 0 && sk[idx[b]] > sk[a]) { idx[b + 1] = idx[b]; --b; }
                idx[b + 1] = a;
            }
            int nu = 0, nv = 0;
            for (int a = 0; a < cnt; ++a) {
                const int c = idx[a];
                win->alist[a] = c;
                if (sty[c] == 0) win->ulist[nu++] = c;
                else win->vlist[nv++] = c;
            }
            win->nc = cnt;
            win->na = cnt;
            win->nu = nu;
            win->nv = nv;
            win->exhausted = spos >= lim;
            ctl->pos = spos;
            ctl->nbuilt += cnt;
            window_opened(win, ctl);
        }
        return;
    }
    if (tid < cnt) {
        // slot: j, k, type, index within the row (or ByElement segment),
        // screen flag, row i, position recorded in the trace
        const int base = ctl->nbuilt / 2;
        const int ci = elem ? si[tid] : i, cq = elem ? sq[tid] : base + tid;
        int *c0 = P.cand + 8 * (2 * tid);
        c0[0] = sj[tid]; c0[1] = sk[tid]; c0[2] = 0; c0[3] = base + tid; c0[4] = 0; c0[5] = ci; c0[6] = cq;
        int *c1 = P.cand + 8 * (2 * tid + 1);
        c1[0] = sj[tid]; c1[1] = sk[tid]; c1[2] = 1; c1[3] = base + tid; c1[4] = 0; c1[5] = ci; c1[6] = cq;
    }
    if (tid == 0) {
        // evaluation lists grouped by k (stable), so the evaluation recomputes
        // E = max over l != k only when k changes; the slots keep the paper's order
        int idx[STMF_WMAX / 2];
        for (int a = 0; a < cnt; ++a) {
            int b = a - 1;
            while (b >= 0 && sk[idx[b]] > sk[a]) { idx[b + 1] = idx[b]; --b; }
            idx[b + 1] = a;
        }
        for (int a = 0; a < cnt; ++a) {
            win->ulist[a] = 2 * idx[a];
            win->vlist[a] = 2 * idx[a] + 1;
            win->alist[2 * a] = 2 * idx[a];
            win->alist[2 * a + 1] = 2 * idx[a] + 1;
        }
        win->nc = 2 * cnt;
        win->na = 2 * cnt;
        win->nu = cnt;
        win->nv = cnt;
        win->exhausted = spos >= lim;
        ctl->pos = spos;
        ctl->nbuilt += 2 * cnt;
        window_opened(win, ctl);
    }
}

// Seeds: F-ULF slots get V'_k. from the column statistics, F-URF slots U'_.k
// from the row statistics, for the slot's own row i (ByElement and ByMatrix
// windows span rows); the other factor of each slot (the residuation of
// phase 1, combined with atomic minima) starts at +inf.  grid.y = slot,
// grid.x covers max(np, mp).
__global__ void k_seed(stmf_problem P)
{
    const int c = blockIdx.y;
    if (c >= P.win->nc) return;
    const int *cd = P.cand + 8 * c;
    const int j = cd[0], k = cd[1], type = cd[2], i = cd[5];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (type == 0) {
        if (x < P.mp) P.Uc[(size_t)c * P.mp + x] = x < P.m ? INFINITY : 0.f;
        if (x >= P.np) return;
        const float useed = P.R[(size_t)i * P.np + j] - P.V[(size_t)k * P.np + j];   // U''_ik
        float v = 0.f;
        if (x < P.n) {
            const size_t e = (size_t)k * P.np + x;
            const float rest = P.carg[e] == i ? P.cmin2[e] : P.cmin1[e];
            v = fminf(P.R[(size_t)i * P.np + x] - useed, rest);
        }
        P.Vc[(size_t)c * P.np + x] = v;
    } else {
        if (x < P.np) P.Vc[(size_t)c * P.np + x] = x < P.n ? INFINITY : 0.f;
        if (x >= P.mp) return;
        const float vseed = P.R[(size_t)i * P.np + j] - P.U[(size_t)i * P.r + k];    // V''_kj
        float u = 0.f;
        if (x < P.m) {
            const size_t e = (size_t)k * P.mp + x;
            const float rest = P.rarg[e] == j ? P.rmin2[e] : P.rmin1[e];
            u = fminf(P.RT[(size_t)j * P.mp + x] - vseed, rest);
        }
        P.Uc[(size_t)c * P.mp + x] = u;
    }
}

__device__ __forceinline__ void put_trace(stmf_ctl *ctl, int pos, int j, int k, int type, double f)
{
    if (!ctl->trace || ctl->ntrace >= ctl->trace_cap) return;
    int32_t *rec = ctl->trace + STMF_TRACE_INTS * ctl->ntrace;
    rec[0] = ctl->sweep; rec[1] = ctl->i; rec[2] = pos; rec[3] = j; rec[4] = k; rec[5] = type;
    const long long bits = __double_as_longlong(f);
    rec[6] = (int32_t)(bits & 0xffffffffll);
    rec[7] = (int32_t)(bits >> 32);
    ctl->ntrace += 1;
}

// Decision of the window in P.win (one pipeline step behind the evaluation):
// sums the phase-2 block partials of every candidate (fixed order) into its
// change Delta = f' - f, keeps the first candidate in the paper's order with
// Delta < 0 (select_mode 1: the smallest), commits it, writes the trace
// record and advances the row; a window that is not live (the first step of
// a row) has nothing to decide.  If the row goes on, builds the window after
// the one being evaluated into the same buffer.  `other` is the other
// buffer's window (evaluated meanwhile; dropped when this decision ends the
// row).  In a graph it also sets the conditions of the row loop: h_win and
// h_step (another pipeline step in this row), h_dirty (refresh before the
// next row), h_row (another row in this sweep).
__global__ void __launch_bounds__(1024) k_select(stmf_problem P, const stmf_win *other, int nblk, int in_graph,
                                                int single, cudaGraphConditionalHandle h_row,
                                                cudaGraphConditionalHandle h_dirty,
                                                cudaGraphConditionalHandle h_win,
                                                cudaGraphConditionalHandle h_step)
{
    __shared__ double sf[STMF_WMAX];
    __shared__ int skept, slive, snc;
    __shared__ stmf_ctl sctl;
    stmf_win *win = P.win;
    if (threadIdx.x == 0) { slive = win->live; snc = win->nc; }
    ctl_load(sctl, P.ctl);
    stmf_ctl *ctl = &sctl;
    const int tid = threadIdx.x;
    const bool live = slive;
    const int nc = live ? snc : 0;
    // 16 threads per candidate, four independent float-float sums each (the
    // loads of a thread are all in flight together); fixed order
    {
        const int c = tid >> 4, sub = tid & 15;
        stmf_ff x = {0.f, 0.f};
        const bool on = c < nc && !P.cand[8 * c + 4];    // dropped: proved non-improving by the FP16 screen
        if (on) {
            const float2 *part = P.part + (size_t)c * nblk;
            stmf_ff x0 = {0.f, 0.f}, x1 = x0, x2 = x0, x3 = x0;
            int b = sub;
            for (; b + 48 < nblk; b += 64) {
                const float2 p0 = part[b], p1 = part[b + 16], p2 = part[b + 32], p3 = part[b + 48];
                x0 = ff_add(x0, {p0.x, p0.y}); x1 = ff_add(x1, {p1.x, p1.y});
                x2 = ff_add(x2, {p2.x, p2.y}); x3 = ff_add(x3, {p3.x, p3.y});
            }
            for (; b < nblk; b += 16) x0 = ff_add(x0, {part[b].x, part[b].y});
            x = ff_add(ff_add(x0, x1), ff_add(x2, x3));
        }
#pragma unroll
        for (int o = 8; o; o >>= 1) x = ff_add(x, {__shfl_xor_sync(FULL, x.hi, o), __shfl_xor_sync(FULL, x.lo, o)});
        if (c < nc && sub == 0) {
            const double d = (double)x.hi + (double)x.lo;
            sf[c] = on ? d : INFINITY;
            P.fc[c] = on ? ctl->f + d : INFINITY;
        }
    }
    __syncthreads();
    if (tid < 32) {
        // the first improving candidate (select_mode 0) or the smallest
        // change, the earlier one on ties (select_mode 1), over nc <= 64
        const int lane = tid;
        int kept = -1;
        if (ctl->select_mode == 0) {
            const unsigned b0 = __ballot_sync(FULL, lane < nc && sf[lane] < 0.0);
            const unsigned b1 = __ballot_sync(FULL, lane + 32 < nc && sf[lane + 32] < 0.0);
            kept = b0 ? __ffs(b0) - 1 : (b1 ? 32 + __ffs(b1) - 1 : -1);
        } else {
            double bv = INFINITY;
            int bi = -1;
            for (int c = lane; c < nc; c += 32)
                if (sf[c] < 0.0 && (bi < 0 || sf[c] < bv)) { bv = sf[c]; bi = c; }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const double ov = __shfl_xor_sync(FULL, bv, o);
                const int oi = __shfl_xor_sync(FULL, bi, o);
                if (oi >= 0 && (bi < 0 || ov < bv || (ov == bv && oi < bi))) { bv = ov; bi = oi; }
            }
            kept = bi;
        }
        if (lane == 0) skept = kept;
    }
    __syncthreads();
    if (tid == 0 && !single && live && ++ctl->win_row > ctl->win_cap) {
        // more windows in this row than its candidates allow: stop every loop
        ctl->err = STMF_ERR_TIMEOUT;
        skept = -1;
    }
    __syncthreads();
    if (tid == 0 && ctl->err == STMF_ERR_TIMEOUT && !single) {
        ctl->row_done = 1;
        ctl->more = 0;
        if (in_graph) {
            cudaGraphSetConditional(h_win, 0u);
            cudaGraphSetConditional(h_step, 0u);
            cudaGraphSetConditional(h_dirty, 0u);
            cudaGraphSetConditional(h_row, 0u);
        }
    } else if (tid == 0 && !live) {
        // first step of a row: window 0 is being evaluated, window 1 is built below
        if (in_graph && !single && !ctl->row_done) {
            cudaGraphSetConditional(h_win, 1u);
            cudaGraphSetConditional(h_step, 1u);
        }
    } else if (tid == 0) {
        const int kept = skept;
        win->live = 0;
        ctl->issued += nc;
        ctl->windows += 1;
        ctl->real_dec += win->placeholder ? 0 : 1;
        ctl->screened += win->screened;
        if (nc > 0 && win->ev_t1 > win->ev_t0) {     // an empty window does no evaluation work
            ctl->eval_ns += (long long)(win->ev_t1 - win->ev_t0);
            ctl->eval_launches += 1;
            ctl->eval_cands += nc;
            if (win->ev_r1 > win->ev_t0) ctl->res_ns += (long long)(win->ev_r1 - win->ev_t0);
            if (win->ev_t1 > win->ev_d0) ctl->delta_ns += (long long)(win->ev_t1 - win->ev_d0);
        }
        ctl->tried += (ctl->select_mode == 0 && kept >= 0) ? kept + 1 : nc;
        ctl->ncand_row += nc;
        ctl->kept = kept >= 0;
        if (kept >= 0) {
            const int *cd = P.cand + 8 * kept;
            ctl->kept_c = kept;
            ctl->kept_j = cd[0]; ctl->kept_k = cd[1]; ctl->kept_type = cd[2]; ctl->kept_pos = cd[3];
            ctl->f_new = ctl->f + sf[kept];
        }
        if (!single) {
            const bool elem = P.strategy == STMF_STRATEGY_BYELEMENT, mat = P.strategy == STMF_STRATEGY_BYMATRIX;
            if (kept >= 0) {
                const int *cd = P.cand + 8 * kept;
                ctl->f = ctl->f_new;          // exact value recomputed by the refresh
                ctl->dirty_k = cd[1];
                ctl->accepted += 1;
                if (elem || mat) ctl->i = cd[5];
                if (elem) ctl->pos = cd[6] + 1;   // ByElement: the scan goes on from the next element
                put_trace(ctl, cd[6], cd[0], cd[1], cd[2], ctl->f_new);
                ctl->row_done = 1;
            } else if (win->exhausted) {
                if (mat) ctl->i = -1;
                if (!elem) put_trace(ctl, -1, -1, -1, -1, ctl->f);
                ctl->row_done = 1;
            } else {
                ctl->row_done = 0;
            }
            if (ctl->row_done) {
                if (other && other->live) ctl->discarded += other->nc;   // evaluated ahead, not needed
                ctl->real_prev = ctl->real_dec;
                if (mat) {
                    ctl->more = 0;            // ByMatrix: one iteration per sweep
                } else if (elem) {
                    ctl->more = kept >= 0 && ctl->pos < P.m * P.n;
                    if (!ctl->more) {
                        ctl->i = -1;          // end of the sweep's scan
                        put_trace(ctl, -1, -1, -1, -1, ctl->f);
                    }
                } else {
                    ctl->i += 1;
                    ctl->more = ctl->i < ctl->m;
                }
                // the next row's first window covers as many columns as this
                // row consumed (rounded up to a power of two): a window's
                // size never changes the decision, only the work per launch
                const int used = kept >= 0 ? P.cand[8 * kept + 3] + 1 : ctl->ncand_row / 2;
                int w = 2;
                while (w < used && w < ctl->wmax / 2) w *= 2;
                ctl->wj0 = ctl->wj0_fixed > 0 ? ctl->wj0_fixed : w;
            }
            if (in_graph) {
                cudaGraphSetConditional(h_win, ctl->row_done ? 0u : 1u);
                cudaGraphSetConditional(h_step, ctl->row_done ? 0u : 1u);
                if (ctl->row_done) {
                    cudaGraphSetConditional(h_dirty, kept >= 0 ? 1u : 0u);
                    cudaGraphSetConditional(h_row, ctl->more ? 1u : 0u);
                }
            }
        }
    }
    __syncthreads();
    const int kept = ctl->err == STMF_ERR_TIMEOUT ? -1 : skept;
    if (kept >= 0) {
        const int k = P.cand[8 * kept + 1];
        for (int s = tid; s < P.m; s += 1024) P.U[(size_t)s * P.r + k] = P.Uc[(size_t)kept * P.mp + s];
        for (int t = tid; t < P.n; t += 1024) P.V[(size_t)k * P.np + t] = P.Vc[(size_t)kept * P.np + t];
    }
    if (!single) {
        __syncthreads();
        // every thread takes the same branch (build_window has barriers):
        // the choice is read from the shared control block before anyone writes it
        const bool ph = !ctl->row_done && ctl->short_row && !ctl->last_ph && ctl->real_built <= 2;
        const bool real = !ctl->row_done && !ph;
        __syncthreads();
        if (ph) {
            if (tid == 0) open_placeholder(win, ctl);
        } else if (real) {
            build_window(P, ctl, false);
        } else if (tid == 0) {
            win->nc = 0;          // nothing to seed or evaluate in this buffer
            win->live = 0;
        }
    }
    ctl_store(P.ctl, sctl);
}

// Start of a row: row state reset and the row's first window, built into
// the buffer P points at; the other buffer (`other`) is emptied, so the
// first pipeline step has nothing to decide.  In a graph, opens the window
// loop.
__global__ void __launch_bounds__(1024) k_row_begin(stmf_problem P, stmf_win *other, int in_graph,
                                                    cudaGraphConditionalHandle h_win,
                                                    cudaGraphConditionalHandle h_step,
                                                    cudaGraphConditionalHandle h_row)
{
    __shared__ stmf_ctl sctl;
    ctl_load(sctl, P.ctl);
    stmf_ctl *ctl = &sctl;
    __shared__ int sstop;
    if (threadIdx.x == 0) {
        if (P.strategy != STMF_STRATEGY_BYELEMENT) ctl->pos = 0;   // ByElement: the scan position carries on
        ctl->ncand_row = 0;
        ctl->nbuilt = 0;
        ctl->wj = ctl->wj0;
        ctl->kept = 0;
        ctl->row_done = 0;
        ctl->win_row = 0;
        ctl->short_row = ctl->real_prev <= 2;
        ctl->real_built = 0;
        ctl->real_dec = 0;
        ctl->last_ph = 0;
        other->nc = 0;
        other->live = 0;
        // more row visits in this sweep than the sweep has rows (segments):
        // stop every loop
        if (++ctl->rows_sweep > ctl->row_cap) ctl->err = STMF_ERR_TIMEOUT;
        sstop = ctl->err == STMF_ERR_TIMEOUT;
        if (sstop) {
            ctl->row_done = 1;
            ctl->more = 0;
            P.win->nc = 0;
            P.win->live = 0;
        }
        if (in_graph) {
            cudaGraphSetConditional(h_win, sstop ? 0u : 1u);
            cudaGraphSetConditional(h_step, sstop ? 0u : 1u);
            if (sstop) cudaGraphSetConditional(h_row, 0u);
        }
    }
    __syncthreads();
    if (!sstop) build_window(P, ctl, true);
    ctl_store(P.ctl, sctl);
}

// Start of a sweep: row 0; in a graph, opens the row loop and asks for a
// refresh if a previous update left the planes stale.
__global__ void k_sweep_begin(stmf_problem P, int in_graph, cudaGraphConditionalHandle h_row,
                              cudaGraphConditionalHandle h_dirty)
{
    stmf_ctl *ctl = P.ctl;
    ctl->i = 0;
    ctl->pos = 0;
    ctl->rows_sweep = 0;
    ctl->more = ctl->m > 0 && ctl->err != STMF_ERR_TIMEOUT;
    if (in_graph) {
        cudaGraphSetConditional(h_row, ctl->more ? 1u : 0u);
        cudaGraphSetConditional(h_dirty, ctl->dirty_k != -2 ? 1u : 0u);
    }
}

// Device-driven job (batched form): opens the sweep loop.
__global__ void k_job_begin(stmf_problem P, cudaGraphConditionalHandle h_sweep)
{
    stmf_ctl *ctl = P.ctl;
    ctl->f_prev = ctl->f;
    cudaGraphSetConditional(h_sweep, ctl->sweep < ctl->sweep_target ? 1u : 0u);
}

// End of a sweep of a device-driven job: next sweep unless the target is
// reached or (eps > 0) the sweep changed the error by less than eps
// (convergence rule of Section "Comparison of strategies").
__global__ void k_sweep_end(stmf_problem P, cudaGraphConditionalHandle h_sweep)
{
    stmf_ctl *ctl = P.ctl;
    ctl->sweep += 1;
    const double d = ctl->f_prev - ctl->f;
    const bool converged = ctl->eps > 0.0 && d < ctl->eps && -d < ctl->eps;
    ctl->f_prev = ctl->f;
    cudaGraphSetConditional(h_sweep, (ctl->sweep < ctl->sweep_target && !converged && !ctl->err) ? 1u : 0u);
}

// One explicit candidate (stmf_update_U / stmf_update_V): slot 0 of the
// buffer P points at.
__global__ void k_single(stmf_problem P, int i, int j, int k, int type)
{
    stmf_ctl *ctl = P.ctl;
    stmf_win *win = P.win;
    int *c0 = P.cand;
    c0[0] = j; c0[1] = k; c0[2] = type; c0[3] = 0; c0[4] = 0; c0[5] = i; c0[6] = 0;
    ctl->i = i;
    win->nc = 1;
    win->nu = type == 0 ? 1 : 0;
    win->nv = type == 1 ? 1 : 0;
    win->ulist[0] = 0;
    win->vlist[0] = 0;
    win->alist[0] = 0;
    win->na = 1;
    win->exhausted = 1;
    win->live = 1;
    win->placeholder = 0;
    win->screened = 0;
    win->ev_t0 = ~0ull;
    win->ev_t1 = 0ull;
    win->ev_r1 = 0ull;
    win->ev_d0 = ~0ull;
    ctl->ncand_row = 0;
    ctl->select_mode = 0;
}

// Unconditional commit of slot 0 (commit_if_decreases = 0).
__global__ void k_commit0(stmf_problem P)
{
    stmf_ctl *ctl = P.ctl;
    const int k = P.cand[1];
    for (int s = threadIdx.x; s < P.m; s += blockDim.x) P.U[(size_t)s * P.r + k] = P.Uc[s];
    for (int t = threadIdx.x; t < P.n; t += blockDim.x) P.V[(size_t)k * P.np + t] = P.Vc[t];
    if (threadIdx.x == 0) {
        ctl->kept = 1; ctl->kept_c = 0; ctl->kept_k = k; ctl->f_new = P.fc[0];
    }
}

// ---------------------------------------------------------------- launchers

cudaError_t launch_pack(cudaStream_t st, const float *R, int ldr, const uint32_t *mask, int ldm, int m, int n,
                        float *Rp, int ldp, int mp, int *bad)
{
    dim3 grid(ldp / 32, mp / 8), block(32, 8);
    k_pack<<<grid, block, 0, st>>>(R, ldr, mask, ldm, m, n, Rp, ldp, mp, bad);
    return cudaGetLastError();
}

cudaError_t launch_pack_oriented(cudaStream_t st, const float *R, int ldr, const uint32_t *mask, int ldm,
                                 int m, int n, int transposed, const int *perm, const int *cperm, float *Rp,
                                 int ldp, int mp, int *bad)
{
    dim3 grid(ldp / 32, mp / 8), block(32, 8);
    k_pack_oriented<<<grid, block, 0, st>>>(R, ldr, mask, ldm, m, n, transposed, perm, cperm, Rp, ldp, mp, bad);
    return cudaGetLastError();
}

cudaError_t launch_col_min(cudaStream_t st, const float *Rp, int ldp, int m, int n, float *cmin)
{
    k_col_min<<<(n + 31) / 32, 1024, 0, st>>>(Rp, ldp, m, n, cmin);
    return cudaGetLastError();
}

cudaError_t launch_unorient(cudaStream_t st, const stmf_problem *P, int transposed, const int *perm,
                            const int *cperm, float *U_out, float *V_out)
{
    const int tot = max(P->m * P->r, P->r * P->n);
    k_unorient<<<(tot + 255) / 256, 256, 0, st>>>(P->U, P->V, P->m, P->n, P->r, P->np, transposed, perm, cperm,
                                                  U_out, V_out);
    return cudaGetLastError();
}

// cperm = the PermC order of the n column minima cmin (device); rank is n
// ints of scratch.
cudaError_t launch_permc_order(cudaStream_t st, const float *cmin, int n, int *rank, int *cperm)
{
    cudaError_t e = cudaMemsetAsync(rank, 0, sizeof(int) * (size_t)n, st);
    if (e != cudaSuccess) return e;
    dim3 grid((n + 255) / 256, (n + PERMC_CHUNK - 1) / PERMC_CHUNK);
    k_permc_rank<<<grid, 256, 0, st>>>(cmin, n, rank);
    k_permc_scatter<<<(n + 255) / 256, 256, 0, st>>>(rank, n, cperm);
    return cudaGetLastError();
}

cudaError_t launch_empty_rows(cudaStream_t st, const float *X, int ldx, int rows, int *nempty)
{
    k_empty_rows<<<(rows * 32 + 255) / 256, 256, 0, st>>>(X, ldx, rows, nempty);
    return cudaGetLastError();
}

cudaError_t launch_transpose(cudaStream_t st, const float *X, int ldx, int rows, int cols, float *XT, int ldxt)
{
    dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
    k_transpose<<<grid, block, 0, st>>>(X, ldx, rows, cols, XT, ldxt);
    return cudaGetLastError();
}

cudaError_t launch_acol(cudaStream_t st, const float *R, int ld, int m, int n, int r, const int *picks, int p,
                        float *U)
{
    k_acol<<<(m * r + 255) / 256, 256, 0, st>>>(R, ld, m, n, r, picks, p, U);
    return cudaGetLastError();
}

cudaError_t launch_copy_rows(cudaStream_t st, const float *src, int lds, float *dst, int ldd, int rows, int cols)
{
    dim3 grid((cols + 255) / 256, rows);
    k_copy_rows<<<grid, 256, 0, st>>>(src, lds, dst, ldd, rows, cols);
    return cudaGetLastError();
}

cudaError_t launch_stats(cudaStream_t st, stmf_problem *P)
{
    const long long threads = (long long)(P->n + P->m) * 32;
    k_stats<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(*P);
    return cudaGetLastError();
}


cudaError_t launch_seed(cudaStream_t st, stmf_problem *P, int nslots)
{
    dim3 grid((max(P->np, P->mp) + 255) / 256, nslots);
    k_seed<<<grid, 256, 0, st>>>(*P);
    return cudaGetLastError();
}

// mode 0: both phases; 1: phase 1 (residuations); 2: phase 2 (error changes).
cudaError_t launch_eval(cudaStream_t st, stmf_problem *P, int mode)
{
    cudaError_t e = cudaSuccess;
    if (mode != 2) e = launch_res(st, P);
    if (e == cudaSuccess && mode != 1) e = launch_delta(st, P);
    return e;
}

// Evaluation of the window in buffer b (its slots were seeded one step
// earlier).  With FP16 screening it splits into phase 1 (every candidate's
// U'/V'), the screen, and phase 2 over the candidates it kept.
cudaError_t launch_window_eval(cudaStream_t st, stmf_problem *P, int b)
{
    stmf_problem v = window_view(P, b);
    if (P->precision == 1) {
        cudaError_t e = launch_eval(st, &v, 1);
        if (e == cudaSuccess) e = launch_screen(st, &v);
        if (e == cudaSuccess) e = launch_eval(st, &v, 2);
        return e;
    }
    return launch_eval(st, &v, 0);
}

// Decision of the window in buffer b, the build of the next window into it
// and that window's seeds.
cudaError_t launch_window_next(cudaStream_t st, stmf_problem *P, int b, int in_graph)
{
    stmf_problem v = window_view(P, b);
    k_select<<<1, 1024, 0, st>>>(v, P->win + (1 - b), delta_parts(P), in_graph, 0, P->h_row, P->h_dirty, P->h_win,
                                 P->h_step);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_seed(st, &v, P->ctl_host->wmax);
    return e;
}

// The decision of a single explicit candidate (buffer 0).
cudaError_t launch_select_single(cudaStream_t st, stmf_problem *P)
{
    k_select<<<1, 1024, 0, st>>>(*P, nullptr, delta_parts(P), 0, 1, P->h_row, P->h_dirty, P->h_win, P->h_step);
    return cudaGetLastError();
}

cudaError_t launch_single(cudaStream_t st, stmf_problem *P, int i, int j, int k, int type)
{
    k_single<<<1, 1, 0, st>>>(*P, i, j, k, type);
    return cudaGetLastError();
}

cudaError_t launch_commit0(cudaStream_t st, stmf_problem *P)
{
    k_commit0<<<1, 256, 0, st>>>(*P);
    return cudaGetLastError();
}

cudaError_t launch_row_begin(cudaStream_t st, stmf_problem *P, int in_graph)
{
    if (P->sel == STMF_SEL_TD) {
        const cudaError_t e = launch_row_order(st, P);     // the row's own column order
        if (e != cudaSuccess) return e;
    }
    if (P->strategy == STMF_STRATEGY_BYMATRIX) {
        const cudaError_t e = launch_matrix_order(st, P);  // the iteration's order of all given elements
        if (e != cudaSuccess) return e;
    }
    k_row_begin<<<1, 1024, 0, st>>>(*P, P->win + 1, in_graph, P->h_win, P->h_step, P->h_row);
    const cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : launch_seed(st, P, P->ctl_host->wmax);   // window 0 (buffer 0)
}

cudaError_t launch_job_begin(cudaStream_t st, stmf_problem *P)
{
    k_job_begin<<<1, 1, 0, st>>>(*P, P->h_sweep);
    return cudaGetLastError();
}

cudaError_t launch_sweep_end(cudaStream_t st, stmf_problem *P)
{
    k_sweep_end<<<1, 1, 0, st>>>(*P, P->h_sweep);
    return cudaGetLastError();
}

cudaError_t launch_sweep_begin(cudaStream_t st, stmf_problem *P, int in_graph)
{
    k_sweep_begin<<<1, 1, 0, st>>>(*P, in_graph, P->h_row, P->h_dirty);
    return cudaGetLastError();
}
