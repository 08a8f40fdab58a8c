// stmf_selection_stats_noalloc: the selection statistics of stmf_selection_stats
// without any allocation, for callers that may not allocate device memory at
// call time (a serving process whose device-memory budget is fixed when it
// starts, or a latency-critical loop that cannot afford the synchronisation
// and the allocator work that cudaMalloc implies).
//
// The scratch (partial column sums and histograms per 128-row part, the
// column sums when the caller passes no td_col, and the error) lives in one
// file-scope device array of STMF_NOALLOC_SCRATCH_BYTES.  Every GPU that
// loads the library holds this array until the process exits.  In host code
// the array's name is only a host-side stand-in, so its device address is
// looked up with cudaGetSymbolAddress, once per device, with that device
// current, on the first call made for that device.
#include <cstdio>
#include <mutex>

#include "common.cuh"

#define STMF_NOALLOC_MAX_DEVICES 64

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[STMF_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[STMF_NOALLOC_MAX_DEVICES];

stmf_status nfail(stmf_ctx *ctx, stmf_status st, const char *msg)
{
    if (ctx) snprintf(ctx->err, sizeof(ctx->err), "%s", msg);
    return st;
}

}  // namespace

extern "C" stmf_status stmf_selection_stats_noalloc(stmf_ctx *ctx, int m, int n, int r, const float *R, int ldr,
                                                    const uint32_t *mask, int ldm_words, const float *U, int ldu,
                                                    const float *V, int ldv, double *td_col, int32_t *colhist,
                                                    double *f_host)
{
    if (!ctx) return STMF_ERR_INVALID;
    if (m < 1 || n < 1) return nfail(ctx, STMF_ERR_INVALID, "sizes must be >= 1");
    if (r < 1 || r > STMF_MAX_RANK) return nfail(ctx, STMF_ERR_INVALID, "rank outside [1, STMF_MAX_RANK]");
    if (!R || !U || !V) return nfail(ctx, STMF_ERR_INVALID, "R, U and V are required");
    if (ldr < n || ldu < r || ldv < n) return nfail(ctx, STMF_ERR_INVALID, "leading dimension too small");
    if (mask && ldm_words < (n + 31) / 32) return nfail(ctx, STMF_ERR_INVALID, "ldm_words < ceil(n/32)");
    if (ctx->device < 0 || ctx->device >= STMF_NOALLOC_MAX_DEVICES)
        return nfail(ctx, STMF_ERR_INVALID, "device index beyond the no-alloc table");

    // scratch layout: tdpart (nparts x n doubles) | tdtmp (n doubles) | f (1 double)
    //                 | chpart (nparts x n x r int32)
    const size_t nparts = (size_t)planes_nparts(m);
    const size_t need = sizeof(double) * (nparts * n + n + 1) + sizeof(int32_t) * nparts * n * r;
    if (need > (size_t)STMF_NOALLOC_SCRATCH_BYTES) {
        snprintf(ctx->err, sizeof(ctx->err),
                 "stmf_selection_stats_noalloc: a %dx%d rank-%d problem needs %zu bytes of scratch, above the "
                 "fixed %d-byte limit (use stmf_selection_stats)",
                 m, n, r, need, (int)STMF_NOALLOC_SCRATCH_BYTES);
        return STMF_ERR_INVALID;
    }

    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return nfail(ctx, STMF_ERR_CUDA, cudaGetErrorString(e));
    unsigned char *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[ctx->device]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                snprintf(ctx->err, sizeof(ctx->err), "cudaGetSymbolAddress of the no-alloc scratch failed: %s",
                         cudaGetErrorString(e));
                return STMF_ERR_CUDA;
            }
            g_noalloc_ptr[ctx->device] = p;
        }
        scratch = (unsigned char *)g_noalloc_ptr[ctx->device];
    }
    // Every field is fully written before it is read, so nothing needs
    // clearing: the kernels write every (part, column) partial, the column
    // sums and the error.
    double *tdpart = (double *)scratch;
    double *tdtmp = tdpart + nparts * n;
    double *fdev = tdtmp + n;
    int32_t *chpart = (int32_t *)(fdev + 1);

    cudaStream_t st = ctx->stream;
    e = launch_maxplus(st, m, n, r, U, ldu, V, ldv, mask, ldm_words, nullptr, 0, nullptr, 0, nullptr, R, ldr, tdpart,
                       chpart);
    double *tdout = td_col ? td_col : tdtmp;
    if (e == cudaSuccess) e = launch_td_finalize2(st, tdpart, chpart, (int)nparts, n, n, r, tdout, colhist);
    if (e == cudaSuccess && f_host) {
        e = launch_error_sum(st, tdout, n, fdev);
        if (e == cudaSuccess) e = cudaMemcpyAsync(f_host, fdev, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return nfail(ctx, STMF_ERR_CUDA, cudaGetErrorString(e));
    return STMF_OK;
}
