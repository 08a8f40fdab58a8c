// Internal declarations of the FastSTMF CUDA library (sm_103a).
//
// Device layout of a problem (all padded so that every row is a whole number
// of 256-float chunks and every row count a multiple of 256):
//   R    mp x np  fp32, given entries as given, every other entry (including
//                 padding) a quiet NaN.  The NaN is the mask of the hot loops:
//                 x - NaN = NaN, fminf/fmaxf drop a NaN operand, so residuation
//                 minima skip entries that are not given and |R - P| folded
//                 through fmaxf(|d|, 0) contributes 0 for them.
//   RT   np x mp  transpose of R (column passes of F-URF read rows of RT).
//   U    mp x r   row-major (rows >= m are 0).
//   V    r x np   row-major (columns >= n are 0).
//   P1, P2 mp x np fp32, A mp x np uint8: top-2 planes of U (x) V.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "stmf.h"

#define STMF_PAD 256
#define STMF_WMAX 64          // candidates per device window (upper bound)

static inline int stmf_roundup(int x, int a) { return (x + a - 1) / a * a; }

struct stmf_ctx {
    int device;
    cudaStream_t stream;
    int num_sms;
    char err[512];
    void *ws;          // workspace for stmf_selection_stats
    size_t ws_bytes;
};

// Control block kept in device memory; kernels of one window read and write
// it, so a window can be replayed from a CUDA graph without host arguments.
struct stmf_ctl {
    int i;             // current row
    int pos;           // next position in the column order
    int row_start;     // 1 before the first window of a row
    int wj;            // j-candidates per window (each gives F-ULF and F-URF)
    int nc;            // candidates in the current window
    int ncand_row;     // candidates of the row consumed so far (sequential index)
    int kept;          // result of the last select: 1 if a candidate was kept
    int row_done;      // 1 once the row is finished (kept or exhausted)
    int kept_pos;      // position (candidate index / 2) of the kept candidate
    int kept_j, kept_k, kept_type;
    int kept_c;        // window slot of the kept candidate
    int err;           // device-detected error code (0 = none)
    int nu, nv;        // F-ULF / F-URF candidates of the window
    int exhausted;     // 1 when the window reached the end of the row's candidates
    int ulist[STMF_WMAX / 2], vlist[STMF_WMAX / 2];   // window slots per type
    long long tried;   // sequential-method candidates tried (cumulative)
    long long issued;  // candidates evaluated on the device (cumulative)
    double f_ulf;      // current error in the F-ULF kernel's summation tree
    double f_urf;      // current error in the F-URF kernel's summation tree
    double f_new;      // error after the kept candidate
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
    int *order;        // np: columns by decreasing td_col, ties to smaller j
    int *cand;         // STMF_WMAX x 8: j, k, type, position (4 spare)
    float *Uc;         // STMF_WMAX x mp candidate U'_.k
    float *Vc;         // STMF_WMAX x np candidate V'_k.
    double *part_ulf;  // (mp/4) x STMF_WMAX partial errors of F-ULF blocks
    double *part_urf;  // (np/32) x STMF_WMAX partial errors of F-URF blocks
    double *fc;        // STMF_WMAX candidate errors
    stmf_ctl *ctl;     // device control block
    stmf_ctl *ctl_host;// pinned host mirror
    int window;        // candidates per window (even, <= STMF_WMAX)
    long long refreshes;
    int dirty_k;       // component to refresh (-1: all), -2: clean
};

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
cudaError_t launch_order(cudaStream_t st, const double *tdcol, int n, int *order);

// kernels_update.cu
cudaError_t launch_pack(cudaStream_t st, const float *R, int ldr, const uint32_t *mask, int ldm,
                        int m, int n, float *Rp, int ldp, int mp, int *bad);
cudaError_t launch_pack_oriented(cudaStream_t st, const float *R, int ldr, const uint32_t *mask, int ldm,
                                 int m, int n, int transposed, const int *perm, float *Rp, int ldp,
                                 int mp, int *bad);
cudaError_t launch_unorient(cudaStream_t st, const stmf_problem *P, int transposed, const int *perm,
                            float *U_out, float *V_out);
cudaError_t launch_empty_rows(cudaStream_t st, const float *X, int ldx, int rows, int *nempty);
cudaError_t launch_transpose(cudaStream_t st, const float *X, int ldx, int rows, int cols,
                             float *XT, int ldxt);
cudaError_t launch_rowstat(cudaStream_t st, const float *X, int ldx, int rows, int cols,
                           const float *y, int ystride, float *min1, float *min2, int *arg);
cudaError_t launch_acol(cudaStream_t st, const float *R, int ld, int m, int n, int r,
                        const int *picks, int p, float *U);
cudaError_t launch_copy_rows(cudaStream_t st, const float *src, int lds, float *dst, int ldd,
                             int rows, int cols);
cudaError_t launch_begin_row(cudaStream_t st, stmf_problem *P, int i, int wj0);
cudaError_t launch_window(cudaStream_t st, stmf_problem *P);
cudaError_t launch_seed(cudaStream_t st, stmf_problem *P, int nslots);
cudaError_t launch_eval(cudaStream_t st, stmf_problem *P, int null_mode);
cudaError_t launch_select(cudaStream_t st, stmf_problem *P, int mode);
cudaError_t launch_single(cudaStream_t st, stmf_problem *P, int i, int j, int k, int type);
cudaError_t launch_commit0(cudaStream_t st, stmf_problem *P);

// peak.cu
cudaError_t launch_peak(cudaStream_t st, int mode, int iters, int blocks, float *sink);
