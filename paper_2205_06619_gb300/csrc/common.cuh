// Internal declarations of the FastSTMF CUDA library (sm_103a).
//
// Device layout of a problem (every row a whole number of 256-float chunks,
// every row count a multiple of 256):
//   R    mp x np  fp32, given entries as given, every other entry (including
//                 padding) a quiet NaN.  The NaN is the mask of the hot loops:
//                 x - NaN = NaN, fminf/fmaxf drop a NaN operand, so residuation
//                 minima skip entries that are not given and |R - P| folded
//                 through fmaxf(|d|, 0) contributes 0 for them.
//   RT   np x mp  transpose of R (column passes of F-URF read rows of RT).
//   U    mp x r   row-major (rows >= m are 0).
//   V    r x np   row-major (columns >= n are 0).
//   P1, P2 mp x np fp32, A mp x np uint8: top-2 planes of U (x) V at given
//                 entries; P1 = P2 = STMF_SENTINEL elsewhere.
//   Rh, P1h, P2h mp x np fp16 (precision 1 only): R, P1, P2 rounded to
//                 nearest half at given entries, a quiet NaN elsewhere.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "stmf.h"

#define STMF_PAD 256
#define STMF_WMAX 64          // candidates per device window (upper bound)
#define STMF_R_LIMIT 1.152921504606846976e18f   // 2^60: given entries of R must be smaller in magnitude
// P1 and P2 planes hold this value where R is not given (and in padding):
// every error change the evaluation forms there is exactly 0 (see k_delta).
#define STMF_SENTINEL 8.5070592e37f                 // 2^126
#define STMF_DELTA_MAX_BLOCKS_PER_SM 8   // capacity of the phase-2 partials, per SM

static inline int stmf_roundup(int x, int a) { return (x + a - 1) / a * a; }

// Float-float (hi, lo) accumulation, about 48 significant bits, with FP32
// operations only (FP64 is slow on this part).  Knuth's TwoSum on the high
// parts, the low parts added to its error, then renormalised.
struct stmf_ff {
    float hi, lo;
};

__device__ __forceinline__ stmf_ff ff_add(stmf_ff a, stmf_ff b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e += a.lo + b.lo;
    const float h = s + e;
    return {h, e - (h - s)};
}

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) as a counter-based
// generator: the output of a SplitMix64 whose state was `key` after c + 1
// steps.  ByMatrix's coin ("random() < 0.5") for iteration it and element q is
// the top bit of draw(coin_key, it m n + q): 0 = F-ULF, 1 = F-URF.
__device__ __forceinline__ unsigned long long splitmix64_draw(unsigned long long key, unsigned long long c)
{
    unsigned long long z = key + (c + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Argmax key of the TD_B / TD selections: the largest td first, then the
// smaller index.  td >= 0, so its float bits order like its value.
__device__ __forceinline__ unsigned long long td_argmax_key(float td, int idx)
{
    return ((unsigned long long)__float_as_uint(td) << 32) | (unsigned)(0xffffffffu - (unsigned)idx);
}
__device__ __forceinline__ int td_argmax_index(unsigned long long key)
{
    return (int)(0xffffffffu - (unsigned)(key & 0xffffffffull));
}

struct stmf_ctx {
    int device;
    cudaStream_t stream;
    int num_sms;
    char err[512];
    void *ws;          // workspace for stmf_selection_stats
    size_t ws_bytes;
    void *tune;        // autotuner cache (std::map of size class -> window and launch shapes), owned
};

// One window of candidates and its evaluation.  Two of them alternate so
// that the evaluation of window t (the phase-1 and phase-2 kernels) runs
// while k_select decides window t-1 and builds window t+1 into the other
// buffer: each kernel touches only its own buffer's window, candidate slots,
// U'/V' and partials.
struct stmf_win {
    int nc;            // candidates in the window
    int na;            // slots to evaluate in phase 2 (after the FP16 screen)
    int nu, nv;        // F-ULF / F-URF slots of phase 1
    int exhausted;     // 1 when the window reached the end of the row's candidates
    int live;          // 1 from the build until the decision
    int screened;      // candidates the FP16 screen proved non-improving
    int placeholder;   // 1: an empty window that only keeps the pipeline in step (short rows)
    int ulist[STMF_WMAX / 2], vlist[STMF_WMAX / 2];   // phase-1 slots per type, grouped by k
    int alist[STMF_WMAX];                             // phase-2 slots, grouped by k
    unsigned long long ev_t0, ev_t1;   // earliest start / latest end of the window's evaluation
    unsigned long long ev_r1, ev_d0;   // end of its phase-1 launch / start of its phase-2 launch
};

// Control block in device memory.  The kernels of the row loop read and
// update it, so one sweep runs as a single CUDA graph launch with no host
// round trip: select decides, commits and advances the row; the graph's
// conditional nodes read the flags the kernels set.
struct stmf_ctl {
    int i;             // current row
    int m;             // rows per sweep
    int sweep;         // sweep index (for the trace)
    int pos;           // next position in the column order (of the next window to build)
    int wj;            // j-candidates of the next window to build (each gives F-ULF, F-URF)
    int wj0;           // j-candidates of a row's first window (what the previous row consumed)
    int wj0_fixed;     // > 0: every row's first window takes this many instead (autotuner trials)
    // short rows: a row whose predecessor decided at most two real windows
    // follows each of its first two real windows with an empty placeholder,
    // so that no window is evaluated before the decision that may end the row
    int short_row;     // this row runs so
    int real_prev;     // real windows the previous row decided
    int real_built;    // real windows built in this row
    int real_dec;      // real windows decided in this row
    int last_ph;       // 1 if the last window built is a placeholder
    int wmax;          // candidates per window (upper bound, even)
    int ncand_row;     // candidates of the row decided so far
    int nbuilt;        // candidates of the row put in windows so far (runs one window ahead)
    int kept;          // 1 if the last select kept a candidate
    int row_done;      // 1 once the row is finished (kept or exhausted)
    int kept_pos, kept_j, kept_k, kept_type, kept_c;
    int dirty_k;       // -2: planes current; -1: refresh all components; k: refresh k
    int select_mode;   // 0 first improving (paper), 1 best of window
    int err;           // device-detected error code (0 = none)
    long long tried;   // sequential-method candidates tried (cumulative)
    long long issued;  // candidates evaluated on the device (cumulative)
    long long accepted;
    long long refreshes;
    long long windows;
    long long discarded;// candidates of windows evaluated ahead and dropped at the end of a row
    long long res_ns, delta_ns;        // summed durations of the phase-1 / phase-2 launches
    long long eval_ns;                 // summed durations of the window evaluations (%globaltimer)
    long long eval_launches;
    long long eval_cands;              // candidates those evaluations covered
    int sweep_target;  // sweeps of a device-driven job (batched form)
    double eps;        // convergence threshold of a device-driven job (0: off)
    double f_prev;     // error at the start of the current sweep
    double f;          // current error (sum over j of td_col[j])
    double f_new;      // error after the kept candidate (f + Delta)
    int32_t *trace;    // device trace buffer (STMF_TRACE_INTS per record) or NULL
    long long trace_cap, ntrace;
    // FP16 screening (precision 1)
    unsigned scr_mr;   // running max of |R| over given entries (float bits)
    unsigned scr_mp;   // running max of the finite |P1|, |P2| over given entries (float bits)
    long long screened;// candidates the screen proved non-improving (cumulative)
    int tdb_j0;        // TD_B: column of the largest td(i, t) of the current row
    int more;          // the row loop goes on (ByRow: rows left; ByElement: elements left in the sweep)
    // Bounds of the device-driven loops (conditional graph nodes): a correct
    // run never reaches them; past one the loops end with err =
    // STMF_ERR_TIMEOUT and nothing more is committed.
    long long win_row, win_cap;     // windows of the current row (ByElement: segment) / their bound
    long long rows_sweep, row_cap;  // row visits (segments) of the current sweep / their bound
};

struct stmf_problem {
    stmf_ctx *ctx;
    int m, n, r;
    int mp, np;        // padded sizes (multiples of STMF_PAD)
    float *R, *RT, *U, *V, *P1, *P2;
    uint8_t *A;
    float *cmin1, *cmin2; int *carg;   // r x np: min over given s of R_st - U_sk (top-2)
    float *rmin1, *rmin2; int *rarg;   // r x mp: min over given t of R_st - V_kt (top-2)
    double *tdpart;    // nparts x np partial column sums of td (128-row parts)
    int *chpart;       // nparts x np x r partial column histograms
    double *tdcol;     // np
    int *colhist;      // np x r
    int *rowhist;      // r
    int *rank;         // np
    int *order;        // np: columns by decreasing td_col, ties to smaller j
    // selection of (j, k) within a row (STMF_SEL_*); the buffers of the
    // selections other than TD_A are NULL unless that selection is used
    int sel;
    int strategy;      // STMF_STRATEGY_*
    int *cperm;        // ByElement: n, oriented column t <- source column cperm[t] (PermC); NULL otherwise
    double *rowkey;    // np: TD keys td(i, t) of the current row (0 where not given)
    int *rowrank;      // np
    int *roworder;     // np: TD order of the current row (decreasing td(i, t), ties to smaller t)
    int *colarg;       // np: TD_B i0 of column t: the row of the largest td(s, t), the smaller s on ties
    // ByMatrix order (NULL / 0 otherwise)
    long long ngiven;  // given entries: the length of the order
    size_t nsort;      // padded sort length (a power of two)
    double *tdr_seq, *tdc_seq;   // m, n: td_row, td_col summed in FP64 in index order
    unsigned long long *skey;    // nsort sort keys
    unsigned *sval;              // nsort: element q = i n + j, in the iteration's order after the sort
    unsigned long long *scnt;    // slot counter of the keys
    unsigned long long coin_key; // key of the per-element coin (seed ^ 0x5A5A...5A)
    // window buffers: the arrays below hold two buffers back to back and
    // point at buffer 0; window_view(P, b) points them at buffer b
    stmf_win *win;     // the window
    int *cand;         // STMF_WMAX x 8: j, k, type, position (4 spare)
    float *Uc;         // STMF_WMAX x mp candidate U'_.k
    float *Vc;         // STMF_WMAX x np candidate V'_k.
    float2 *part;      // STMF_WMAX x (phase-2 blocks) partial changes, float-float (hi, lo)
    double *fc;        // STMF_WMAX candidate errors
    // launch shapes of the window evaluation (0: the defaults; set by the
    // autotuner before any capture): phase 1's column chunk (a multiple of 8
    // in [32, 128]), phase 2's blocks per SM (1..5; 1..4 with 8-row tiles)
    // and phase 2's thread-tile rows (4 or 8)
    int res_chunk_sel, delta_bps_sel, delta_rows_sel;
    // FP16 screening (precision 1; all NULL otherwise)
    int precision;
    __half *Rh, *P1h, *P2h;
    int scr_blocks;    // row blocks of the screen
    float2 *scr_sum;   // STMF_WMAX x scr_blocks screened changes (float-float)
    float2 *scr_cnt;   // STMF_WMAX x scr_blocks counts of possibly changed given entries (float-float)
    float *scr_umax;   // STMF_WMAX x scr_blocks max |U'_sk| over the block's rows
    float *scr_vmax;   // STMF_WMAX max |V'_kt| over t < n
    stmf_ctl *ctl;     // device control block
    stmf_ctl *ctl_host;// pinned host mirror
    int32_t *trace_dev;// device trace buffer
    // factorization bookkeeping
    int transposed;    // input was tall and is stored transposed
    int m0, n0;        // caller's shape
    int *perm;         // device permutation (oriented rows -> caller rows/cols)
    double f_init;     // error after initialisation
    int sweeps_done;
    double seconds;    // wall time spent in sweeps
    // sweep graph
    cudaGraphExec_t sweep_exec;
    cudaGraph_t sweep_graph;
    unsigned long long h_row, h_dirty, h_win;   // cudaGraphConditionalHandle values
    unsigned long long h_step;                  // second pipeline step of a window-loop iteration
    unsigned long long h_sweep;                 // sweep loop of a device-driven job
};

// Sizes of one window buffer, in elements of each array.
inline size_t win_cand_elems() { return 8 * STMF_WMAX; }
inline size_t win_uc_elems(const stmf_problem *P) { return (size_t)STMF_WMAX * P->mp; }
inline size_t win_vc_elems(const stmf_problem *P) { return (size_t)STMF_WMAX * P->np; }
inline size_t win_part_elems(int num_sms) { return (size_t)STMF_DELTA_MAX_BLOCKS_PER_SM * num_sms * STMF_WMAX; }

// The problem with its window arrays pointed at buffer b (0 or 1).
inline stmf_problem window_view(const stmf_problem *P, int b)
{
    stmf_problem v = *P;
    v.win += b;
    v.cand += b * win_cand_elems();
    v.Uc += b * win_uc_elems(P);
    v.Vc += b * win_vc_elems(P);
    v.part += b * win_part_elems(P->ctx->num_sms);
    v.fc += b * STMF_WMAX;
    return v;
}

// ---------------------------------------------------------------- launchers
// kernels_product.cu
cudaError_t launch_maxplus(cudaStream_t st, int m, int n, int r, const float *U, int ldu,
                           const float *V, int ldv, const uint32_t *mask, int ldm,
                           float *P1, int ldp, uint8_t *A, int lda, float *P2,
                           const float *R, int ldr, double *tdpart, int *colhist);
cudaError_t launch_planes(cudaStream_t st, stmf_problem *P, int *chpart);
int planes_nparts(int m);
cudaError_t launch_td_finalize2(cudaStream_t st, const double *tdpart, const int *chpart, int nparts,
                                int ldpart, int n, int r, double *tdcol, int *colhist);
cudaError_t launch_refresh_planes(cudaStream_t st, stmf_problem *P);
cudaError_t launch_error_sum(cudaStream_t st, const double *tdcol, int n, double *out);   // fixed-order sum
int rmse_blocks(int m, int num_sms);
cudaError_t launch_rmse(cudaStream_t st, int num_sms, int m, int n, int r, const float *R, int ldr,
                        const uint32_t *mask, int ldm, const float *U, int ldu, const float *V, int ldv,
                        double *part, double *out);
cudaError_t launch_row_order(cudaStream_t st, stmf_problem *P);
// kernels_bymatrix.cu
size_t matrix_sort_len(long long ngiven);
cudaError_t launch_matrix_order(cudaStream_t st, stmf_problem *P);
cudaError_t launch_count_given(cudaStream_t st, const stmf_problem *P, unsigned long long *d_cnt);

// kernels_update.cu
cudaError_t launch_pack(cudaStream_t st, const float *R, int ldr, const uint32_t *mask, int ldm,
                        int m, int n, float *Rp, int ldp, int mp, int *bad);
cudaError_t launch_pack_oriented(cudaStream_t st, const float *R, int ldr, const uint32_t *mask, int ldm,
                                 int m, int n, int transposed, const int *perm, const int *cperm, float *Rp,
                                 int ldp, int mp, int *bad);
cudaError_t launch_col_min(cudaStream_t st, const float *Rp, int ldp, int m, int n, float *cmin);
cudaError_t launch_permc_order(cudaStream_t st, const float *cmin, int n, int *rank, int *cperm);
cudaError_t launch_unorient(cudaStream_t st, const stmf_problem *P, int transposed, const int *perm, const int *cperm,
                            float *U_out, float *V_out);
cudaError_t launch_empty_rows(cudaStream_t st, const float *X, int ldx, int rows, int *nempty);
cudaError_t launch_transpose(cudaStream_t st, const float *X, int ldx, int rows, int cols,
                             float *XT, int ldxt);
cudaError_t launch_acol(cudaStream_t st, const float *R, int ld, int m, int n, int r,
                        const int *picks, int p, float *U);
cudaError_t launch_copy_rows(cudaStream_t st, const float *src, int lds, float *dst, int ldd,
                             int rows, int cols);
cudaError_t launch_stats(cudaStream_t st, stmf_problem *P);
cudaError_t launch_seed(cudaStream_t st, stmf_problem *P, int nslots);
cudaError_t launch_eval(cudaStream_t st, stmf_problem *P, int mode = 0);
cudaError_t launch_window_eval(cudaStream_t st, stmf_problem *P, int b);
cudaError_t launch_window_next(cudaStream_t st, stmf_problem *P, int b, int in_graph);

// kernels_eval.cu
cudaError_t launch_res(cudaStream_t st, stmf_problem *P);
cudaError_t launch_delta(cudaStream_t st, stmf_problem *P);
int delta_grid(const stmf_problem *P);
int delta_parts(const stmf_problem *P);   // phase-2 partials per candidate
bool delta_fills_gpu(const stmf_problem *P);   // phase 2 alone has a tile for every resident block
int delta_depth(const stmf_problem *P);
int delta_rows(const stmf_problem *P);
cudaError_t delta_prepare();                     // before any capture
int res_chunk(const stmf_problem *P);            // phase 1's column chunk for this problem
cudaError_t launch_select_single(cudaStream_t st, stmf_problem *P);
cudaError_t launch_single(cudaStream_t st, stmf_problem *P, int i, int j, int k, int type);
cudaError_t launch_commit0(cudaStream_t st, stmf_problem *P);
cudaError_t launch_row_begin(cudaStream_t st, stmf_problem *P, int in_graph);
cudaError_t launch_sweep_begin(cudaStream_t st, stmf_problem *P, int in_graph);
cudaError_t launch_job_begin(cudaStream_t st, stmf_problem *P);
cudaError_t launch_sweep_end(cudaStream_t st, stmf_problem *P);

// kernels_screen.cu
constexpr int SCR_ROWS = 8;
constexpr int SCR_THREADS = 128;
cudaError_t screen_prepare(stmf_problem *P);
cudaError_t launch_screen(cudaStream_t st, stmf_problem *P);

// mlp.cu
stmf_status mlp_predict_rows(stmf_ctx *ctx, stmf_mlp *M, int m, int n, const float *R, int ldr,
                             const uint32_t *mask, int ldm_words, float *U0);
int mlp_rank(const stmf_mlp *M);

// peak.cu
cudaError_t launch_peak(cudaStream_t st, int mode, int iters, int blocks, float *sink);
double peak_ops(int mode, int iters, int blocks);
