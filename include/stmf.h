/*
 * stmf.h -- C ABI of the GB300 (sm_103a) FastSTMF hot path.
 *
 * FastSTMF (Omanovic, Oblak, Curk, arXiv 2205.06619) approximates a partially
 * given matrix R (m x n) by a tropical (max,+) product U (x) V with U m x r,
 * V r x n (Section "Related work", the tropical matrix factorization
 * problem).  This library computes, on one GPU:
 *   - the masked max-plus product with per-entry max, argmax and runner-up;
 *   - the F-ULF / F-URF single-step updates (Algorithms 1 and 2);
 *   - the full ByRow / TD_A / RandPerm / wide method (Algorithm 3).
 *
 * Conventions shared by every entry point
 *   Memory.  Every array argument is DEVICE memory owned by the caller
 *     (e.g. a torch CUDA tensor), unless its comment says "host".  The library
 *     owns only its opaque objects and their device workspaces, and frees them
 *     in the matching destroy call.
 *   Layout.  Row-major FP32 with a leading dimension (elements between row
 *     starts): R and P planes m x n with ld >= n; U m x r with ldu >= r;
 *     V r x n with ldv >= n.
 *   Mask.  Bit-packed uint32, row-major, ldm_words >= ceil(n/32) words per
 *     row; bit (t & 31) of word [s*ldm_words + t/32] set <=> R_st is given
 *     (observed).  NULL mask = every entry given.  Entries not given are never
 *     read from R.
 *   Stream.  Every call enqueues its work on the context's stream; calls that
 *     return host values (errors, reports) synchronize that stream.
 *   Errors.  No exception crosses the ABI.  Each call returns an
 *     stmf_status; STMF_ERR_INVALID is returned, with nothing launched, for a
 *     bad argument (size < 1, r outside [1, STMF_MAX_RANK], a too-small
 *     leading dimension, a NULL required pointer, an index out of range, a
 *     row or column with no given entry, a given entry that is not finite
 *     or has magnitude 2^60 or more: the evaluation keeps entries that are
 *     not given at a finite sentinel far above that range).  The text
 *     of the last error of a context is available from stmf_last_error().
 *     Device-side loops are bounded: the sweep, row and window loops of a
 *     factorization run as conditional nodes of a CUDA graph, driven by the
 *     device; a row never needs more windows than its candidate order has
 *     positions, nor a sweep more row visits than m n + 1.  Should a loop
 *     pass its bound (a logic error), every loop stops, nothing more is
 *     committed, and the call returns STMF_ERR_TIMEOUT; the context and the
 *     device stay usable.  No kernel spin-waits.
 */
#ifndef STMF_H
#define STMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STMF_MAX_RANK 32

typedef enum {
    STMF_OK = 0,
    STMF_ERR_INVALID = 1,  /* bad argument; nothing was launched             */
    STMF_ERR_CUDA = 2,     /* a CUDA runtime call failed                      */
    STMF_ERR_OOM = 3,      /* device workspace allocation failed              */
    STMF_ERR_TIMEOUT = 4,  /* a bound of the device-driven loops ran out      */
    STMF_ERR_INTERNAL = 5  /* an internal consistency check failed            */
} stmf_status;

typedef struct stmf_ctx stmf_ctx;         /* device, stream, error text       */
typedef struct stmf_problem stmf_problem; /* R, mask, U, V, planes, stats    */
typedef struct stmf_mlp stmf_mlp;         /* learned-initialisation network  */

/* Selections of (j, k) within a row (Section "The ByRow strategy").  Every
 * selection tries its (j, k) pairs in order, F-ULF then F-URF for each, and
 * keeps the first candidate that lowers the error; only given entries R_ij
 * are candidates; sorts keep the smaller index first on equal keys, and
 * every argmax the smaller index on ties.
 *   TD_A: columns by td_col descending; k = the component occurring most
 *         often in f(i, .) and f(., j) together (Algorithm 3, the default).
 *   TD_B: columns as TD_A; j0 = argmax_t td(i,t), i0 = argmax_s td(s,j);
 *         k = f(i,j0) if (U(x)V)_{i j0} >= (U(x)V)_{i0 j}, else f(i0,j).
 *         (Reading: the argmaxes run over the entry-wise td of row i and of
 *         column j; td_col itself does not depend on the row.)
 *   TD:   columns by their own td(i,j) descending; k = f(i,j).
 *   SEQ:  columns in increasing j, each with k = 0, 1, ..., r-1.
 * td(s,t) = |R_st - (U(x)V)_st| over given entries; f(s,t) = the smallest
 * l attaining (U(x)V)_st. */
enum { STMF_SEL_TD_A = 0, STMF_SEL_TD_B = 1, STMF_SEL_TD = 2, STMF_SEL_SEQ = 3 };

/* Update strategies (Section "The ByElement strategy", Section "The ByRow
 * strategy").
 *   BYROW:     Algorithm 3 (FastSTMF): rows in a random order, one kept
 *              update per row at most, (j, k) by `selection`.
 *   BYELEMENT: STMF_ByElement_PermC_TD_W (the Supplement's pseudocode): R
 *              oriented wide, its columns in increasing order of their
 *              minimum given entry (equal minima: smaller column first), rows
 *              in their own order.  A sweep visits every element (i, j) in
 *              row-major order; an element with R_ij given and
 *              td(i,j) = |R_ij - (U(x)V)_ij| > 0 is tried once with
 *              k = f(i,j): F-ULF, else F-URF, keeping the first that lowers
 *              the error; the scan goes on from the next element.  Needs
 *              perm = NULL and selection = TD_A; U0 / V0 are in the frame of
 *              the oriented, column-permuted matrix.  Trace: one record per
 *              kept update {sweep, i, q = i*n + j, j, k, type, f} (oriented,
 *              permuted frame) and one {sweep, -1, -1, -1, -1, -1, f} at the
 *              end of each sweep.
 *   BYMATRIX:  STMF_ByMatrix_NoPerm_TD_W (the Supplement's pseudocode): R
 *              oriented wide, no permutation.  Each iteration ranks every
 *              given element by err = td_row(i) + td_col(j) - td(i,j)
 *              (td_row, td_col summed in FP64 in index order; decreasing err,
 *              equal err: smaller q = i*n + j first) and tries them in that
 *              order with k = f(i,j) and F-ULF or F-URF by a fair coin (the
 *              top bit of SplitMix64 keyed by seed ^ 0x5A5A5A5A5A5A5A5A at
 *              counter it*m*n + q: 0 = F-ULF), ending at the first update that
 *              lowers the error.  `sweeps` counts iterations.  Needs perm =
 *              NULL and selection = TD_A.  Trace: one record per iteration
 *              {it, i, position in the order, j, k, type, f}, or
 *              {it, -1, -1, -1, -1, -1, f} when nothing was kept. */
enum { STMF_STRATEGY_BYROW = 0, STMF_STRATEGY_BYELEMENT = 1, STMF_STRATEGY_BYMATRIX = 2 };

/* Options of the factorization (Algorithm 3 and its readings). */
typedef struct {
    int sweeps;          /* passes over all rows (the loop "while not converged") */
    double eps;          /* > 0: also stop when a sweep changes the error by < eps
                            (convergence rule of Section "Comparison of strategies") */
    int window;          /* candidates evaluated per device pass (speculative window);
                            0 = library default.  Never changes which update is kept. */
    int select;          /* 0 = keep the first improving candidate in the paper's order
                            (default, Algorithm 3); 1 = keep the best of the window    */
    int precision;       /* 0 = FP32 (default); 1 = FP16 screening + FP32 re-check:
                            each window's candidates are first evaluated in packed
                            half2 arithmetic; a candidate is dropped only when a
                            rigorous error bound proves its FP32 change >= 0, and the
                            others are re-evaluated in FP32 in the paper's order, so
                            the kept updates are those of precision 0.  Extra device
                            memory: three mp x np half planes.                        */
    int acol_p;          /* Random Acol: columns averaged per component; 0 = 5 (clamped to n) */
    uint64_t seed;       /* draws the row permutation and the Acol picks (SplitMix64)  */
    const int32_t *perm;  /* HOST, nullable: explicit row permutation of the oriented R
                            (length = oriented m); overrides the seed                  */
    const int32_t *picks; /* HOST, nullable: explicit Acol picks, r x acol_p column
                            indices of the oriented R; overrides the seed              */
    const float *U0;     /* DEVICE, nullable: initial U of the oriented, permuted problem
                            (m x r, ld r); replaces Random Acol                          */
    int32_t *trace;      /* HOST, nullable: one record of STMF_TRACE_INTS per row visit */
    int64_t trace_cap;   /* capacity of trace in records                               */
    const float *V0;     /* DEVICE, nullable, needs U0: V of the oriented problem (r x n,
                            ld n) used as given instead of the residuation of U0.
                            With the U0, V0 and perm of a saved state, a new run
                            continues exactly as the interrupted one would have
                            (checkpoint / resume between sweeps).                  */
    const stmf_mlp *mlp; /* nullable: learned initialisation (an addition to the paper).
                            U0 of the oriented, permuted problem = MLP(row sketch) +
                            row median, computed on the device; the network's rank
                            must be r, it must belong to the same context, and the
                            oriented n must be <= 12288.  U0, if given, wins.      */
    int selection;       /* STMF_SEL_*: how a row picks its (j, k) pairs; 0 = TD_A.
                            TD keeps a per-row column order (three extra launches
                            per row); TD_B a per-column argmax (one extra launch
                            per refresh).                                          */
    int strategy;        /* STMF_STRATEGY_*: 0 = ByRow (Algorithm 3), 1 = ByElement,
                            2 = ByMatrix                                           */
    int res_chunk;       /* launch shape of the window evaluation's phase 1: columns
                            per task, a multiple of 8 in [32, 128]; 0 = the
                            library's choice (the batched form's autotuner, else a
                            wave heuristic).  Never changes a result.             */
    int delta_blocks_per_sm; /* phase 2's blocks per SM, 1..5 (1..4 with 8-row
                            tiles); 0 = the library's choice.                    */
    int delta_tile_rows; /* phase 2's thread tile: 4 or 8 rows of one float4 column;
                            0 = the library's choice.  The last two regroup the
                            FP32 error sums (within their float-float accuracy)
                            and change no decision but at an exact tie.          */
} stmf_options;

/* A trace record: sweep, row (oriented, permuted index), position of the kept
 * candidate among the row's candidates (-1: nothing kept), j, k,
 * type (0 = F-ULF, 1 = F-URF), and the error after the row as two int32
 * halves of a double (little-endian). */
#define STMF_TRACE_INTS 8

typedef struct {
    double f_init;            /* b-norm error after initialisation                  */
    double f_final;           /* b-norm error at the end                            */
    int sweeps_done;
    int transposed;           /* 1 if the input was tall and was transposed          */
    int64_t candidates_tried; /* sequential-method candidates (up to the kept one)  */
    int64_t candidates_issued;/* candidates evaluated on the device (>= tried)      */
    int64_t accepted;         /* updates kept                                        */
    int64_t refreshes;        /* product/statistics refreshes                        */
    int64_t windows;          /* device windows evaluated                            */
    int64_t trace_records;    /* trace records written                               */
    int64_t eval_ns;          /* summed device durations of the window evaluations
                                 (phase-1 start to phase-2 end, %globaltimer)       */
    int64_t eval_launches;    /* window evaluations timed                            */
    int64_t eval_candidates;  /* candidates those evaluations covered                */
    double seconds;           /* wall time of the sweep loop                         */
    int64_t candidates_screened; /* candidates the FP16 screen proved non-improving
                                    (precision 1; counted in candidates_issued)   */
    int64_t eval_res_ns;      /* summed durations of the phase-1 (residuation) launches */
    int64_t eval_delta_ns;    /* summed durations of the phase-2 (error change) launches */
    int64_t candidates_discarded; /* candidates evaluated one window ahead of the decisions
                                     and dropped because the row ended first (not in
                                     candidates_issued)                              */
    int64_t eval_res_chunk;   /* phase 1's column chunk (launch shape in use)          */
    int64_t eval_delta_blocks;/* phase 2's blocks per launch (launch shape in use)     */
    int64_t eval_delta_rows;  /* phase 2's thread-tile rows (launch shape in use)      */
} stmf_report;

/* Context: binds a device and a stream (cudaStream_t passed as void*; NULL =
 * the legacy default stream).  out receives the new context. */
stmf_status stmf_create(stmf_ctx **out, int device, void *cuda_stream);
void stmf_destroy(stmf_ctx *ctx);
/* Text of the last error of ctx (static storage owned by ctx; "" if none). */
const char *stmf_last_error(const stmf_ctx *ctx);
/* Changes the stream of ctx. */
stmf_status stmf_set_stream(stmf_ctx *ctx, void *cuda_stream);

/* Masked max-plus product with top-2 tracking (Section "Related work",
 * tropical matrix multiplication; f(i,j) of Section "The ByRow strategy"):
 *   P1_ij = max_l (U_il + V_lj)
 *   A_ij  = smallest l attaining P1_ij          (uint8; needs r <= 255)
 *   P2_ij = max over l != A_ij of (U_il + V_lj) (-inf when r == 1)
 * Sums and max are FP32 (IEEE, round to nearest).  Entries (i,j) not given by
 * the mask are written as P1 = P2 = NaN, A = 255.  A and P2 may be NULL.
 * P1/P2 use ldp, A uses lda (bytes).  Device pointers; no workspace. */
stmf_status stmf_maxplus(stmf_ctx *ctx, int m, int n, int r,
                         const float *U, int ldu, const float *V, int ldv,
                         const uint32_t *mask, int ldm_words,
                         float *P1, int ldp, uint8_t *A, int lda, float *P2);

/* Selection statistics of the ByRow / TD_A strategy (Section "The ByRow
 * strategy"; Algorithm 3) over the given entries, from the product above:
 *   td_col[j]          = sum over given i of |R_ij - (U (x) V)_ij|   (FP64)
 *   colhist[j*r + l]   = #{given i : f(i,j) = l}                      (int32)
 *   *f_host            = sum over j of td_col[j]  (the b-norm error)   (HOST),
 *                        summed on the device in the fixed order of the
 *                        factorization's own error
 * td_col, colhist device (either may be NULL); f_host may be NULL.  Uses a
 * device workspace owned by ctx (grown on demand). */
stmf_status stmf_selection_stats(stmf_ctx *ctx, int m, int n, int r,
                                 const float *R, int ldr, const uint32_t *mask, int ldm_words,
                                 const float *U, int ldu, const float *V, int ldv,
                                 double *td_col, int32_t *colhist, double *f_host);

/* RMSE-A and RMSE-P (Section "Evaluation metrics": the root-mean-square
 * error of the approximation on the training data, RMSE-A, and on the test
 * data of the prediction task, RMSE-P; Section "Evaluation": 20% of the
 * entries are masked uniformly at random and form the test set):
 *   RMSE_S = sqrt( (1/|S|) sum over (i,j) in S of (R_ij - (U (x) V)_ij)^2 )
 * with S_A = the given entries (mask bit 1; every entry when mask is NULL)
 * and S_P = the entries not given whose true value R holds (R_ij not NaN).
 * (U (x) V)_ij and R_ij - (U (x) V)_ij are FP32, as in the factorization;
 * squares and sums FP64 in a fixed order.  R (m x n, ld ldr), mask, U (m x r,
 * ld ldu), V (r x n, ld ldv) device; out_host (host, 4 doubles) receives
 * {RMSE-A, RMSE-P, |S_A|, |S_P|}, NaN for an empty set.  Uses the context's
 * workspace (grown on demand) and synchronizes its stream. */
stmf_status stmf_rmse(stmf_ctx *ctx, int m, int n, int r, const float *R, int ldr,
                      const uint32_t *mask, int ldm_words, const float *U, int ldu,
                      const float *V, int ldv, double *out_host);

/* stmf_selection_stats without any allocation.  The paper has no counterpart:
 * this entry point exists for callers that may not allocate device memory
 * when they call (a process whose device-memory budget is fixed at start-up,
 * or a loop that cannot pay for cudaMalloc's synchronisation).  Arguments,
 * layouts and results are those of stmf_selection_stats, bit for bit (the
 * same kernels and the same fixed summation orders).  Its scratch is one
 * file-scope device array of STMF_NOALLOC_SCRATCH_BYTES that every GPU loading
 * the library holds until the process exits; a problem needs
 *   8 * (ceil(m/128) * n + n + 1) + 4 * ceil(m/128) * n * r  bytes,
 * and larger problems are rejected with STMF_ERR_INVALID (nothing launched).
 * The first call made for a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  The call allocates nothing: no cudaMalloc, no
 * cudaFree, no allocating library routine.  All calls share the one array, so
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race; serialise them.  Nothing in the array needs clearing between calls. */
#define STMF_NOALLOC_SCRATCH_BYTES (16 * 1024 * 1024)
stmf_status stmf_selection_stats_noalloc(stmf_ctx *ctx, int m, int n, int r,
                                         const float *R, int ldr, const uint32_t *mask, int ldm_words,
                                         const float *U, int ldu, const float *V, int ldv,
                                         double *td_col, int32_t *colhist, double *f_host);

/* A problem: a copy of R (m x n, not transposed, not permuted) and its mask,
 * the factors U, V and the device state F-ULF / F-URF need.  U0 (device,
 * m x r, ld r) may be NULL: then U comes from Random Acol with opts->seed
 * (opts->picks if given).  V is always computed as (-U)^T (x)* R.  opts may
 * be NULL (defaults).  Fails with STMF_ERR_INVALID if a row or a column of R
 * has no given entry. */
stmf_status stmf_problem_create(stmf_ctx *ctx, int m, int n, int r,
                                const float *R, int ldr, const uint32_t *mask, int ldm_words,
                                const float *U0, const stmf_options *opts, stmf_problem **out);
void stmf_problem_destroy(stmf_problem *prob);

/* F-ULF(i, j, k) (Algorithm 1): U_ik <- R_ij - V_kj; V_k. <- (-U_.k)^T (x)* R;
 * U_.k <- R (x)* (-V_k.)^T; f' = ||R - U (x) V||_b over given entries.
 * commit_if_decreases = 1: keep the update only if f' < f (the paper's
 * revert, Algorithm 3); 0: keep it unconditionally.  Requires R_ij given.
 * f_new (host) receives f'; accepted (host) receives 1 if kept.
 * Both nullable. */
stmf_status stmf_update_U(stmf_problem *prob, int i, int j, int k, int commit_if_decreases,
                          double *f_new, int *accepted);
/* F-URF(i, j, k) (Algorithm 2): V_kj <- R_ij - U_ik; U_.k <- R (x)* (-V_k.)^T;
 * V_k. <- (-U_.k)^T (x)* R; then as stmf_update_U. */
stmf_status stmf_update_V(stmf_problem *prob, int i, int j, int k, int commit_if_decreases,
                          double *f_new, int *accepted);
/* Copies the current factors out (device U m x r ld r, V r x n ld n; either
 * may be NULL) and the current error (host, nullable). */
stmf_status stmf_problem_get(stmf_problem *prob, float *U, float *V, double *f);

/* FastSTMF, Algorithm 3 (STMF_ByRow_RandPerm_TD_A_W): transpose a tall R,
 * permute rows at random, Random Acol init, V by residuation, then sweeps of
 * the ByRow loop: per row, candidates j in decreasing td_col (given R_ij
 * only, ties to the smaller j), k by TD_A, F-ULF then F-URF, first strict
 * decrease kept.  U_out (m x r, ld r) and V_out (r x n, ld n) are device
 * arrays in the caller's orientation.  report (host) nullable. */
stmf_status stmf_factorize(stmf_ctx *ctx, int m, int n, int r,
                           const float *R, int ldr, const uint32_t *mask, int ldm_words,
                           const stmf_options *opts, float *U_out, float *V_out,
                           stmf_report *report);

/* The same method in three steps, so that sweeps can be run (and timed) in
 * pieces on one live problem:
 *   stmf_factorize_begin: orientation, permutation, Random Acol (or opts->U0),
 *     V by residuation, product planes and statistics; *out receives the
 *     problem (free it with stmf_problem_destroy).  opts is copied, except
 *     that opts->trace, if set, must stay valid until stmf_factorize_end.
 *   stmf_factorize_run: `sweeps` more sweeps (stops early when eps > 0 and a
 *     sweep changed the error by less than eps); report (host, nullable)
 *     receives the cumulative counters of the problem.
 *   stmf_factorize_end: writes U_out, V_out (device, caller's orientation,
 *     both nullable) and copies up to trace_cap trace records to trace (host,
 *     nullable).  The problem stays valid. */
stmf_status stmf_factorize_begin(stmf_ctx *ctx, int m, int n, int r,
                                 const float *R, int ldr, const uint32_t *mask, int ldm_words,
                                 const stmf_options *opts, stmf_problem **out);
stmf_status stmf_factorize_run(stmf_problem *prob, int sweeps, double eps, stmf_report *report);
stmf_status stmf_factorize_end(stmf_problem *prob, float *U_out, float *V_out,
                               int32_t *trace, int64_t trace_cap);

/* One problem of a batch (all pointers device memory, caller orientation). */
typedef struct {
    int m, n, r;                 /* shape and rank                                   */
    const float *R;              /* m x n, ld ldr                                    */
    int ldr;
    const uint32_t *mask;        /* bit-packed, nullable                             */
    int ldm_words;
    float *U_out;                /* m x r, ld r                                      */
    float *V_out;                /* r x n, ld n                                      */
    uint64_t seed;               /* draws its permutation and Acol picks             */
    int sweeps;                  /* sweeps of this problem                           */
    int32_t *trace;              /* HOST, nullable: this problem's trace records, as  */
    int64_t trace_cap;           /* stmf_options.trace of a single call; capacity    */
} stmf_batch_problem;

/* Many independent FastSTMF problems (Algorithm 3 each) of uneven size and
 * rank in ONE device launch: the whole job -- every problem's sweeps, rows,
 * windows, refreshes and convergence tests -- is one CUDA graph whose
 * branches (one per problem, each a device-driven loop of conditional nodes)
 * run concurrently.  Decisions, factors and errors are exactly those of
 * stmf_factorize on each problem with the same options.  opts (nullable):
 * eps, select and window apply to every problem; window == 0 lets the
 * library's autotuner pick each problem's window from one timed sweep per size
 * class on scratch copies (cached in ctx).  reports (host, nprob entries) and
 * tuned_windows (host, nprob ints) are nullable.  A problem whose trace is set
 * receives up to trace_cap records of its row visits (the records of
 * stmf_factorize; report[i].trace_records counts those written).  Set-up (allocation,
 * initialisation) runs before the launch; report[i].seconds is the wall time
 * of the single launch. */
stmf_status stmf_factorize_batched(stmf_ctx *ctx, int nprob, const stmf_batch_problem *probs,
                                   const stmf_options *opts, stmf_report *reports, int *tuned_windows);

/* ---- Learned initialisation of U (an addition to the paper, which uses
 * Random Acol, Section "Comparison of strategies").  A row of R is summarised
 * by a 32-quantile sketch of its given entries centred on the row median; an
 * MLP 32 -> 128 -> 128 -> r (ReLU, BF16 weights, FP32 accumulation) maps the
 * sketch to the row of U minus its median.  Random Acol stays the fallback. */
/* sketch[s*32 + q] = v[floor((q+0.5)*c/32)] - median_s and median[s] =
 * v[floor(c/2)], where v are the c given entries of row s sorted ascending
 * (nearest-rank quantiles).  R, mask, sketch (m x 32), median (m) device;
 * n <= 12288.  mask NULL: the given entries are those of R that are not NaN. */
stmf_status stmf_row_sketch(stmf_ctx *ctx, int m, int n, const float *R, int ldr, const uint32_t *mask,
                            int ldm_words, float *sketch, float *median);
/* Number of parameters of the MLP for rank r (-1 if r is out of range).
 * Layout: W1 [32 x 128] | W2 [128 x 128] | W3 [128 x r] | b1 [128] | b2 [128] | b3 [r]
 * (row-major, input index first). */
int stmf_mlp_param_count(int r);
/* Creates an MLP from host FP32 parameters (copied); Adam state zeroed. */
stmf_status stmf_mlp_create(stmf_ctx *ctx, int r, const float *params_host, stmf_mlp **out);
void stmf_mlp_destroy(stmf_mlp *mlp);
/* Copies the FP32 master parameters to host memory. */
stmf_status stmf_mlp_get_params(stmf_mlp *mlp, float *params_host);
/* Y (B x r, device) = MLP(X (B x 32, device)), BF16 weights, FP32 accumulation. */
stmf_status stmf_mlp_forward(stmf_mlp *mlp, int B, const float *X, float *Y);
/* Mean squared error of MLP(X) against T (B x r, device) and its gradient
 * with respect to every parameter (loss, grad_host nullable; grad in the
 * parameter layout).  Every gradient element is a fixed-order FP32 sum. */
stmf_status stmf_mlp_gradient(stmf_mlp *mlp, int B, const float *X, const float *T, double *loss,
                              float *grad_host);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on the FP32 master parameters
 * with learning rate lr; loss (host, nullable) receives the batch loss. */
stmf_status stmf_mlp_train_step(stmf_mlp *mlp, int B, const float *X, const float *T, float lr, double *loss);

/* U0 (m x r, device) = MLP(sketch of row s of R) + median of row s: the
 * learned start (the sketch as stmf_row_sketch; mask NULL: the given entries
 * are those of R that are not NaN); n <= 12288.  Uses the MLP's context and
 * stream; returns when U0 is written. */
stmf_status stmf_mlp_predict(stmf_mlp *mlp, int m, int n, const float *R, int ldr, const uint32_t *mask,
                             int ldm_words, float *U0);
/* Training targets from a factorization (U m x r, V r x n; device, row
 * strides ldu, ldv): the gauge (U_.l + c, V_l. - c leaves U (x) V unchanged,
 * and so does any order of the components) is fixed by c_l = max over t < n
 * of V_lt, and the components are ordered by decreasing sum over rows of
 * U_sl + c_l (FP64, rows in index order; equal sums: smaller l first).
 * sorted = 0: T[s*r + p] = (U_s,l_p + c_l_p) - median[s], l_p the component at
 * position p; sorted = 1: row s's values U_sl + c_l in decreasing order, minus
 * median[s].  FP32; T (m x r) and median (m) device.  Scratch is allocated and
 * freed inside; the call returns when T is written. */
stmf_status stmf_mlp_targets(stmf_ctx *ctx, int m, int n, int r, const float *U, int ldu, const float *V, int ldv,
                             const float *median, int sorted, float *T);
/* out[s*ldo + l] = the value of row s of Y whose rank in its row (decreasing)
 * equals the rank of U_ref[s*ldu + l] in its row (decreasing; equal values:
 * the smaller index first): predictions made for "sorted" targets handed to
 * the components in the order of a reference start.  Device pointers, r <=
 * STMF_MAX_RANK; out may not alias Y.  Asynchronous on ctx's stream. */
stmf_status stmf_assign_by_rank(stmf_ctx *ctx, int m, int r, const float *Y, int ldy, const float *U_ref, int ldu,
                                float *out, int ldo);

/* Fills *opts with the defaults (sweeps 1, eps 0, library window, first
 * improving, FP32, acol_p 5, seed 0, no explicit draws, no trace, no MLP). */
void stmf_default_options(stmf_options *opts);
/* sizeof of the ABI's structs as this library was compiled (host pointers,
 * each nullable), so that a binding can check its own layouts. */
void stmf_struct_sizes(size_t *options, size_t *report, size_t *batch_problem);

/* FP32 add+max issue-rate microbenchmark: runs `iters` dependent-chain
 * iterations of (FADD, FMNMX) pairs on every SM and returns, in *gops
 * (host), the measured giga-operations per second (FADD and FMNMX count one
 * each).  mode 0: 1:1 FADD/FMNMX; 1: FADD only; 2: FMNMX only;
 * 3: packed half2 HADD2/HMNMX2 (two operations per lane); 4: packed
 * FP32x2 adds only; 5: one packed FP32x2 add then two scalar FMNMX (1:1 mix
 * with the additions packed).  Modes 6 and 7 run the instruction mixes of
 * the window evaluation's two passes and count their algorithmic operations
 * per given entry and candidate (the units the benchmark reports): 6, the
 * error-change pass (per two entries a packed add u + v, two FMNMX for
 * max(E, x), a packed sub P1 - max and a packed accumulation: 4 operations
 * per entry); 7, the residuation pass (per two entries two FADD for R - w
 * and one three-input minimum: 2 operations per entry).  Uses the context's
 * stream and synchronizes it. */
stmf_status stmf_peak_addmax(stmf_ctx *ctx, int mode, int iters, double *gops);

#ifdef __cplusplus
}
#endif
#endif /* STMF_H */
