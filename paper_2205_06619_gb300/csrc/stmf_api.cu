// Host side of the C ABI declared in include/stmf.h: argument validation,
// device workspaces, set-up of a problem, the F-ULF / F-URF single updates
// and the row loop of Algorithm 3 (FastSTMF).
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <chrono>
#include <cmath>
#include <map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace {

// SplitMix64 (Steele, Lea, Flood 2014) as a counter-based generator:
// draw(key, c) = output of a SplitMix64 seeded with key after c+1 steps.
uint64_t draw(uint64_t key, uint64_t c)
{
    uint64_t z = key + (c + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Random permutation of 0..m-1: Fisher-Yates from the top,
// b = draw(seed, m-1-a) mod (a+1) for a = m-1 .. 1.
void random_permutation(int m, uint64_t seed, std::vector<int> &perm)
{
    perm.resize(m);
    for (int s = 0; s < m; ++s) perm[s] = s;
    for (int a = m - 1; a >= 1; --a) {
        const int b = (int)(draw(seed, (uint64_t)(m - 1 - a)) % (uint64_t)(a + 1));
        std::swap(perm[a], perm[b]);
    }
}

// Random Acol picks: per component l, p distinct columns of 0..n-1 by a
// partial Fisher-Yates with draws (seed ^ 0xA5A5...A5, l*p + q).
void acol_picks(int n, int r, int p, uint64_t seed, std::vector<int> &picks)
{
    picks.resize((size_t)r * p);
    std::vector<int> arr(n);
    const uint64_t key = seed ^ 0xA5A5A5A5A5A5A5A5ull;
    for (int l = 0; l < r; ++l) {
        for (int t = 0; t < n; ++t) arr[t] = t;
        for (int q = 0; q < p; ++q) {
            const int b = q + (int)(draw(key, (uint64_t)l * p + q) % (uint64_t)(n - q));
            std::swap(arr[q], arr[b]);
            picks[(size_t)l * p + q] = arr[q];
        }
    }
}

stmf_status fail(stmf_ctx *ctx, stmf_status st, const char *fmt, ...)
{
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? STMF_ERR_OOM : STMF_ERR_CUDA,      \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);    \
    } while (0)

#define CK2(c, call)                                                                              \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(c, STMF_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));               \
    } while (0)

// NVTX ranges (header-only NVTX 3) around the host driver's phases, so a
// timeline tool shows preparation, sweeps, the batched launch and tuning.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Host-side fault injection for tests: with STMF_TEST_FAIL_ALLOC=N in the
// environment, the N-th device allocation of every problem reports
// cudaErrorMemoryAllocation (nothing is allocated), so the error paths can be
// exercised without exhausting or faulting a GPU.
int g_alloc_index = 0;

template <class T>
cudaError_t dalloc(T **p, size_t count)
{
    const char *inj = getenv("STMF_TEST_FAIL_ALLOC");
    if (inj && ++g_alloc_index == atoi(inj)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc((void **)p, sizeof(T) * (count ? count : 1));
}

void problem_free(stmf_problem *P)
{
    if (!P) return;
    if (P->sweep_exec) cudaGraphExecDestroy(P->sweep_exec);
    if (P->sweep_graph) cudaGraphDestroy(P->sweep_graph);
    void *ptrs[] = {P->R, P->RT, P->U, P->V, P->P1, P->P2, P->A, P->cmin1, P->cmin2, P->carg,
                    P->rmin1, P->rmin2, P->rarg, P->tdpart, P->chpart, P->tdcol, P->colhist,
                    P->rowhist, P->rank, P->order, P->win, P->cand, P->Uc, P->Vc, P->part, P->fc,
                    P->ctl, P->trace_dev, P->perm, P->Rh, P->P1h, P->P2h, P->scr_sum, P->scr_cnt,
                    P->scr_umax, P->scr_vmax, P->rowkey, P->rowrank, P->roworder, P->colarg, P->cperm,
                    P->tdr_seq, P->tdc_seq, P->skey, P->sval, P->scnt};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (P->ctl_host) cudaFreeHost(P->ctl_host);
    delete P;
}

template <class T>
cudaError_t set_ctl(stmf_problem *P, T stmf_ctl::*field, T value)
{
    // pageable source: the copy has consumed `value` when the call returns
    return cudaMemcpyAsync(&(P->ctl->*field), &value, sizeof(T), cudaMemcpyHostToDevice, P->ctx->stream);
}

stmf_status problem_alloc(stmf_ctx *ctx, int m, int n, int r, int window, stmf_problem **out)
{
    g_alloc_index = 0;
    stmf_problem *P = new stmf_problem();
    memset(P, 0, sizeof(*P));
    P->ctx = ctx;
    P->m = m; P->n = n; P->r = r;
    P->mp = stmf_roundup(m, STMF_PAD);
    P->np = stmf_roundup(n, STMF_PAD);
    const size_t mp = P->mp, np = P->np;
    const int nparts = planes_nparts(m);
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    A(dalloc(&P->R, mp * np)); A(dalloc(&P->RT, np * mp));
    A(dalloc(&P->U, mp * r)); A(dalloc(&P->V, (size_t)r * np));
    A(dalloc(&P->P1, mp * np)); A(dalloc(&P->P2, mp * np)); A(dalloc(&P->A, mp * np));
    A(dalloc(&P->cmin1, (size_t)r * np)); A(dalloc(&P->cmin2, (size_t)r * np)); A(dalloc(&P->carg, (size_t)r * np));
    A(dalloc(&P->rmin1, (size_t)r * mp)); A(dalloc(&P->rmin2, (size_t)r * mp)); A(dalloc(&P->rarg, (size_t)r * mp));
    A(dalloc(&P->tdpart, (size_t)nparts * np)); A(dalloc(&P->chpart, (size_t)nparts * np * r));
    A(dalloc(&P->tdcol, np)); A(dalloc(&P->colhist, np * r)); A(dalloc(&P->rowhist, STMF_MAX_RANK));
    A(dalloc(&P->rank, np)); A(dalloc(&P->order, np));
    // two window buffers (window_view)
    A(dalloc(&P->win, 2)); A(dalloc(&P->cand, 2 * win_cand_elems()));
    A(dalloc(&P->Uc, 2 * win_uc_elems(P))); A(dalloc(&P->Vc, 2 * win_vc_elems(P)));
    A(dalloc(&P->part, 2 * win_part_elems(ctx->num_sms)));   // float2
    A(dalloc(&P->fc, 2 * STMF_WMAX)); A(dalloc(&P->ctl, 1));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&P->ctl_host, sizeof(stmf_ctl));
    if (e == cudaSuccess) e = delta_prepare();
    if (e != cudaSuccess) {
        problem_free(P);
        cudaGetLastError();
        return fail(ctx, STMF_ERR_OOM, "device allocation for a %dx%d rank-%d problem failed: %s", m, n, r,
                    cudaGetErrorString(e));
    }
    cudaStream_t st = ctx->stream;
    stmf_ctl c;
    memset(&c, 0, sizeof(c));
    c.m = m;
    c.wj0 = 2;
    c.wmax = window;
    c.dirty_k = -1;
    c.win_cap = c.row_cap = 1ll << 60;   // refined by the factorization's set-up
    e = cudaMemsetAsync(P->U, 0, sizeof(float) * mp * r, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->V, 0, sizeof(float) * r * np, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->P1, 0, sizeof(float) * mp * np, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->P2, 0, sizeof(float) * mp * np, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->A, 0, mp * np, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->ctl, &c, sizeof(c), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->win, 0, 2 * sizeof(stmf_win), st);   // empty, not live
    if (e != cudaSuccess) { problem_free(P); return fail(ctx, STMF_ERR_CUDA, "memset: %s", cudaGetErrorString(e)); }
    *out = P;
    return STMF_OK;
}

// Statistics of the component named by ctl->dirty_k, then planes, td_col,
// colhist, column order and f (which marks the planes current).
stmf_status refresh(stmf_problem *P)
{
    stmf_ctx *ctx = P->ctx;
    CK(launch_stats(ctx->stream, P));
    CK(launch_refresh_planes(ctx->stream, P));
    return STMF_OK;
}

// After R is packed: checks, RT, U, V = (-U)^T (x)* R, statistics, planes, f.
stmf_status problem_init(stmf_problem *P, const float *U0, int acol_p, uint64_t seed, const int32_t *picks_in,
                         const float *V0 = nullptr)
{
    stmf_ctx *ctx = P->ctx;
    cudaStream_t st = ctx->stream;
    CK(launch_transpose(st, P->R, P->np, P->mp, P->np, P->RT, P->mp));
    int *d_cnt = nullptr;
    CK(cudaMalloc(&d_cnt, 2 * sizeof(int)));
    CK(cudaMemsetAsync(d_cnt, 0, 2 * sizeof(int), st));
    CK(launch_empty_rows(st, P->R, P->np, P->m, d_cnt));
    CK(launch_empty_rows(st, P->RT, P->mp, P->n, d_cnt + 1));
    int cnt[2];
    CK(cudaMemcpyAsync(cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    cudaFree(d_cnt);
    if (cnt[0] || cnt[1])
        return fail(ctx, STMF_ERR_INVALID, "%d rows and %d columns have no given entry", cnt[0], cnt[1]);
    if (U0) {
        CK(cudaMemcpyAsync(P->U, U0, sizeof(float) * P->m * P->r, cudaMemcpyDeviceToDevice, st));
    } else {
        const int p = acol_p > 0 ? (acol_p < P->n ? acol_p : P->n) : (P->n < 5 ? P->n : 5);
        std::vector<int> picks;
        if (picks_in) {
            picks.assign(picks_in, picks_in + (size_t)P->r * p);
            for (int x : picks)
                if (x < 0 || x >= P->n) return fail(ctx, STMF_ERR_INVALID, "Acol pick %d out of range", x);
        } else {
            acol_picks(P->n, P->r, p, seed, picks);
        }
        int *d_picks = nullptr;
        CK(cudaMalloc(&d_picks, sizeof(int) * picks.size()));
        CK(cudaMemcpyAsync(d_picks, picks.data(), sizeof(int) * picks.size(), cudaMemcpyHostToDevice, st));
        CK(launch_acol(st, P->R, P->np, P->m, P->n, P->r, d_picks, p, P->U));
        CK(cudaStreamSynchronize(st));
        cudaFree(d_picks);
    }
    CK(set_ctl(P, &stmf_ctl::dirty_k, -1));
    if (V0) {
        // a saved state (checkpoint): V as given, no residuation
        CK(launch_copy_rows(st, V0, P->n, P->V, P->np, P->r, P->n));
    } else {
        // V = (-U)^T (x)* R: the column minima of component l are the min1 of
        // its column statistics.
        CK(launch_stats(st, P));
        CK(launch_copy_rows(st, P->cmin1, P->np, P->V, P->np, P->r, P->n));
    }
    stmf_status s = refresh(P);        // statistics of the new (U, V), planes, f
    if (s != STMF_OK) return s;
    return STMF_OK;
}

stmf_status read_ctl(stmf_problem *P)
{
    stmf_ctx *ctx = P->ctx;
    CK(cudaMemcpyAsync(P->ctl_host, P->ctl, sizeof(stmf_ctl), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return STMF_OK;
}

stmf_status check_common(stmf_ctx *ctx, int m, int n, int r)
{
    if (!ctx) return STMF_ERR_INVALID;
    if (m < 1 || n < 1) return fail(ctx, STMF_ERR_INVALID, "sizes must be >= 1 (m=%d, n=%d)", m, n);
    if (r < 1 || r > STMF_MAX_RANK) return fail(ctx, STMF_ERR_INVALID, "rank %d outside [1, %d]", r, STMF_MAX_RANK);
    if ((long long)m * n > (1ll << 31) - 1) return fail(ctx, STMF_ERR_INVALID, "m*n too large");
    CK(cudaSetDevice(ctx->device));
    return STMF_OK;
}

stmf_status update(stmf_problem *P, int i, int j, int k, int type, int commit_if_decreases, double *f_new,
                   int *accepted)
{
    if (!P) return STMF_ERR_INVALID;
    stmf_ctx *ctx = P->ctx;
    if (i < 0 || i >= P->m || j < 0 || j >= P->n || k < 0 || k >= P->r)
        return fail(ctx, STMF_ERR_INVALID, "index out of range (i=%d, j=%d, k=%d)", i, j, k);
    float rij;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    CK(cudaMemcpyAsync(&rij, P->R + (size_t)i * P->np + j, sizeof(float), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (rij != rij) return fail(ctx, STMF_ERR_INVALID, "R[%d][%d] is not given", i, j);
    CK(launch_single(st, P, i, j, k, type));
    CK(launch_seed(st, P, 1));
    CK(launch_eval(st, P));
    CK(launch_select_single(st, P));
    if (!commit_if_decreases) CK(launch_commit0(st, P));
    stmf_status s = read_ctl(P);
    if (s != STMF_OK) return s;
    const int kept = P->ctl_host->kept;
    double fval;
    CK(cudaMemcpyAsync(&fval, P->fc, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (f_new) *f_new = fval;
    if (accepted) *accepted = kept;
    if (kept) {
        CK(set_ctl(P, &stmf_ctl::dirty_k, k));
        s = refresh(P);
        if (s != STMF_OK) return s;
    }
    return STMF_OK;
}

// Captures `launch` into graph g after the nodes deps (nullable), and returns
// the node(s) the capture ended with (exactly one for one kernel).
template <class Launch>
stmf_status capture_into(stmf_ctx *ctx, cudaStream_t cap, cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps,
                         Launch launch, cudaGraphNode_t *last)
{
    CK(cudaStreamBeginCaptureToGraph(cap, g, deps, nullptr, ndeps, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = launch(cap);
    if (e != cudaSuccess) {
        cudaGraph_t tmp;
        cudaStreamEndCapture(cap, &tmp);
        return fail(ctx, STMF_ERR_CUDA, "capture: %s", cudaGetErrorString(e));
    }
    if (last) {
        cudaStreamCaptureStatus stat;
        const cudaGraphNode_t *dep = nullptr;
        size_t nd = 0;
        CK(cudaStreamGetCaptureInfo(cap, &stat, nullptr, nullptr, &dep, nullptr, &nd));
        if (nd != 1) return fail(ctx, STMF_ERR_INTERNAL, "capture ended with %zu nodes", nd);
        *last = dep[0];
    }
    cudaGraph_t tmp;
    CK(cudaStreamEndCapture(cap, &tmp));
    return STMF_OK;
}

stmf_status add_conditional(stmf_ctx *ctx, cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps,
                            cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type, cudaGraphNode_t *node,
                            cudaGraph_t *body)
{
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = 1;
    CK(cudaGraphAddNode(node, g, deps, nullptr, ndeps, &p));
    *body = p.conditional.phGraph_out[0];
    return STMF_OK;
}

#define CS(call)                            \
    do {                                    \
        stmf_status s_ = (call);            \
        if (s_ != STMF_OK) return s_;       \
    } while (0)

// One pipeline step into graph g after the nodes deps: the evaluation of the
// window in buffer b on `cap`, beside the decision of the window in buffer
// 1 - b, the build of the next window into it and its seeds on `side`.  The
// step's two end nodes go to ends (nullable).
stmf_status capture_step(stmf_ctx *ctx, cudaStream_t cap, cudaStream_t side, cudaEvent_t fork, cudaEvent_t join,
                         cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps, stmf_problem *P, int b,
                         std::vector<cudaGraphNode_t> *ends)
{
    CK(cudaStreamBeginCaptureToGraph(cap, g, deps, nullptr, ndeps, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaEventRecord(fork, cap);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, fork, 0);
    if (e == cudaSuccess) e = launch_window_eval(cap, P, b);
    if (e == cudaSuccess) e = launch_window_next(side, P, 1 - b, 1);
    if (e == cudaSuccess) e = cudaEventRecord(join, side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, join, 0);
    if (e == cudaSuccess && ends) {
        cudaStreamCaptureStatus stat;
        const cudaGraphNode_t *dep = nullptr;
        size_t nd = 0;
        e = cudaStreamGetCaptureInfo(cap, &stat, nullptr, nullptr, &dep, nullptr, &nd);
        if (e == cudaSuccess) ends->assign(dep, dep + nd);
    }
    cudaGraph_t tmp;
    const cudaError_t e2 = cudaStreamEndCapture(cap, &tmp);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return fail(ctx, STMF_ERR_CUDA, "capture of a pipeline step: %s",
                    cudaGetErrorString(e != cudaSuccess ? e : e2));
    return STMF_OK;
}

// Adds one problem's row loop to graph g (its conditional handles are created
// on `top`, the graph that will be instantiated):
//   sweep_begin;
//   while (h_row) {
//     if (h_dirty) { stats(k), planes, td_col/colhist, rank, order + f }
//     row_begin (window 0 into buffer 0, its seeds);
//     while (h_win) {
//       eval(buffer 0) | select(buffer 1), next window into buffer 1, seeds;
//       if (h_step) { eval(buffer 1) | select(buffer 0), next window into buffer 0, seeds }
//     }
//   }
// ("|": two branches that run at the same time.)  Step t evaluates window t
// while window t-1 is decided; when that decision ends the row, window t's
// evaluation is dropped.
// With job = true the row loop is wrapped in a device-driven sweep loop:
//   job_begin; while (h_sweep) { <row loop>; sweep_end }
// and the job starts after the nodes deps (nullable); *end (nullable)
// receives its last node, the sweep loop.
stmf_status add_problem_nodes(stmf_problem *P, cudaGraph_t top, cudaGraph_t g, bool job, cudaStream_t cap,
                              const cudaGraphNode_t *deps = nullptr, size_t ndeps = 0, cudaGraphNode_t *end = nullptr)
{
    stmf_ctx *ctx = P->ctx;
    cudaGraphConditionalHandle hr, hd, hw, hp, hs = 0;
    CK(cudaGraphConditionalHandleCreate(&hr, top, 0, 0));
    CK(cudaGraphConditionalHandleCreate(&hd, top, 0, 0));
    CK(cudaGraphConditionalHandleCreate(&hw, top, 0, 0));
    CK(cudaGraphConditionalHandleCreate(&hp, top, 0, 0));
    if (job) CK(cudaGraphConditionalHandleCreate(&hs, top, 0, 0));
    P->h_row = hr; P->h_dirty = hd; P->h_win = hw; P->h_step = hp; P->h_sweep = hs;
    cudaStream_t side;
    cudaEvent_t fork, join;
    CK(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    struct SS { cudaStream_t s; ~SS() { cudaStreamDestroy(s); } } ss{side};
    CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    struct EF { cudaEvent_t e; ~EF() { cudaEventDestroy(e); } } ef{fork};
    CK(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
    struct EJ { cudaEvent_t e; ~EJ() { cudaEventDestroy(e); } } ej{join};

    cudaGraph_t target = g;
    if (job) {
        cudaGraphNode_t jb = nullptr, wsw = nullptr;
        CS(capture_into(ctx, cap, g, deps, ndeps, [&](cudaStream_t c) { return launch_job_begin(c, P); }, &jb));
        CS(add_conditional(ctx, g, &jb, 1, hs, cudaGraphCondTypeWhile, &wsw, &target));
        if (end) *end = wsw;
    }
    cudaGraphNode_t sb = nullptr, wrow = nullptr;
    CS(capture_into(ctx, cap, target, nullptr, 0, [&](cudaStream_t c) { return launch_sweep_begin(c, P, 1); }, &sb));
    cudaGraph_t body_row = nullptr;
    CS(add_conditional(ctx, target, &sb, 1, hr, cudaGraphCondTypeWhile, &wrow, &body_row));
    if (job)
        CS(capture_into(ctx, cap, target, &wrow, 1, [&](cudaStream_t c) { return launch_sweep_end(c, P); }, nullptr));

    cudaGraphNode_t nif = nullptr, rb = nullptr, wwin = nullptr;
    cudaGraph_t body_ref = nullptr, body_win = nullptr;
    CS(add_conditional(ctx, body_row, nullptr, 0, hd, cudaGraphCondTypeIf, &nif, &body_ref));
    CS(capture_into(ctx, cap, body_ref, nullptr, 0, [&](cudaStream_t c) {
        cudaError_t e = launch_stats(c, P);
        return e != cudaSuccess ? e : launch_refresh_planes(c, P);
    }, nullptr));
    CS(capture_into(ctx, cap, body_row, &nif, 1, [&](cudaStream_t c) { return launch_row_begin(c, P, 1); }, &rb));
    CS(add_conditional(ctx, body_row, &rb, 1, hw, cudaGraphCondTypeWhile, &wwin, &body_win));
    std::vector<cudaGraphNode_t> ends;
    CS(capture_step(ctx, cap, side, fork, join, body_win, nullptr, 0, P, 0, &ends));
    cudaGraphNode_t nstep = nullptr;
    cudaGraph_t body_step = nullptr;
    CS(add_conditional(ctx, body_win, ends.data(), ends.size(), hp, cudaGraphCondTypeIf, &nstep, &body_step));
    CS(capture_step(ctx, cap, side, fork, join, body_step, nullptr, 0, P, 1, nullptr));
    return STMF_OK;
}

// The sweep of one problem as one graph (the host loops over sweeps).
stmf_status build_sweep_graph(stmf_problem *P)
{
    stmf_ctx *ctx = P->ctx;
    cudaStream_t cap;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    struct SG { cudaStream_t s; ~SG() { cudaStreamDestroy(s); } } sg{cap};
    cudaGraph_t g;
    CK(cudaGraphCreate(&g, 0));
    P->sweep_graph = g;
    CS(add_problem_nodes(P, g, g, false, cap));
    CK(cudaGraphInstantiate(&P->sweep_exec, g, 0));
    return STMF_OK;
}

bool use_graph()
{
    const char *e = getenv("STMF_NO_GRAPH");
    return !(e && e[0] == '1');
}

// One row (ByElement: segment; ByMatrix: iteration) driven from the host:
// the graph's pipeline steps in order on one stream, one synchronisation per
// step.
stmf_status row_host(stmf_problem *P)
{
    stmf_ctx *ctx = P->ctx;
    cudaStream_t st = ctx->stream;
    CK(launch_row_begin(st, P, 0));
    for (int b = 0;; b ^= 1) {
        CK(launch_window_eval(st, P, b));
        CK(launch_window_next(st, P, 1 - b, 0));
        CS(read_ctl(P));
        if (P->ctl_host->row_done) return STMF_OK;
    }
}

// One sweep driven from the host; used when graphs are disabled.
stmf_status sweep_host(stmf_problem *P)
{
    stmf_ctx *ctx = P->ctx;
    cudaStream_t st = ctx->stream;
    CK(launch_sweep_begin(st, P, 0));
    stmf_status s = read_ctl(P);
    if (s != STMF_OK) return s;
    while (P->ctl_host->more) {           // ByRow: one pass per row; ByElement: per kept update
        if (P->ctl_host->dirty_k != -2) {
            s = refresh(P);
            if (s != STMF_OK) return s;
        }
        s = row_host(P);
        if (s != STMF_OK) return s;
    }
    return STMF_OK;
}

// PermC of the ByElement strategy: the columns of the packed, oriented R in
// increasing order of their minimum given entry, equal minima keeping the
// smaller column first (a rank count on the device); R is then packed again
// through that order, which P->cperm keeps for the output.
cudaError_t setup_permc(stmf_problem *P, cudaStream_t st, const float *R, int ldr, const uint32_t *mask,
                        int ldm_words, int *d_bad)
{
    const int m = P->m, n = P->n;
    float *d_cmin = nullptr;
    int *d_rank = nullptr;
    cudaError_t e = cudaMalloc(&d_cmin, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_rank, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMalloc(&P->cperm, sizeof(int) * n);
    if (e == cudaSuccess) e = launch_col_min(st, P->R, P->np, m, n, d_cmin);
    if (e == cudaSuccess) e = launch_permc_order(st, d_cmin, n, d_rank, P->cperm);
    if (e == cudaSuccess)
        e = launch_pack_oriented(st, R, ldr, mask, ldm_words, m, n, P->transposed, P->perm, P->cperm, P->R, P->np,
                                 P->mp, d_bad);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the scratch stays alive until the kernels end
    if (d_cmin) cudaFree(d_cmin);
    if (d_rank) cudaFree(d_rank);
    return e;
}

// The number of given entries of the packed R into P->ngiven (the length of
// every ByMatrix iteration's order).
cudaError_t count_given(stmf_problem *P, cudaStream_t st)
{
    unsigned long long *d_cnt = nullptr, cnt = 0;
    cudaError_t e = cudaMalloc(&d_cnt, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = launch_count_given(st, P, d_cnt);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (d_cnt) cudaFree(d_cnt);
    P->ngiven = (long long)cnt;
    return e;
}

// Algorithm 3 preparation: orientation, permutation, packing, init.
cudaError_t set_loop_bounds(stmf_problem *P);

stmf_status fastmf_begin(stmf_ctx *ctx, int m0, int n0, int r, const float *R, int ldr, const uint32_t *mask,
                         int ldm_words, const stmf_options *opts, stmf_problem **out)
{
    *out = nullptr;
    stmf_status s = check_common(ctx, m0, n0, r);
    if (s != STMF_OK) return s;
    if (!R) return fail(ctx, STMF_ERR_INVALID, "R is required");
    if (ldr < n0) return fail(ctx, STMF_ERR_INVALID, "ldr < n");
    if (mask && ldm_words < (n0 + 31) / 32) return fail(ctx, STMF_ERR_INVALID, "ldm_words < ceil(n/32)");
    stmf_options o;
    if (opts) o = *opts; else stmf_default_options(&o);
    if (o.window < 0 || o.window > STMF_WMAX) return fail(ctx, STMF_ERR_INVALID, "window outside [0, %d]", STMF_WMAX);
    if (o.precision < 0 || o.precision > 1) return fail(ctx, STMF_ERR_INVALID, "precision mode %d unknown", o.precision);
    if (o.select < 0 || o.select > 1) return fail(ctx, STMF_ERR_INVALID, "select mode %d unknown", o.select);
    if (o.V0 && !o.U0) return fail(ctx, STMF_ERR_INVALID, "V0 needs U0");
    if (o.selection < STMF_SEL_TD_A || o.selection > STMF_SEL_SEQ)
        return fail(ctx, STMF_ERR_INVALID, "selection %d unknown", o.selection);
    if (o.strategy < STMF_STRATEGY_BYROW || o.strategy > STMF_STRATEGY_BYMATRIX)
        return fail(ctx, STMF_ERR_INVALID, "strategy %d unknown", o.strategy);
    if (o.res_chunk && (o.res_chunk < 32 || o.res_chunk > 128 || o.res_chunk % 8))
        return fail(ctx, STMF_ERR_INVALID, "res_chunk %d: 0 or a multiple of 8 in [32, 128]", o.res_chunk);
    if (o.delta_tile_rows != 0 && o.delta_tile_rows != 4 && o.delta_tile_rows != 8)
        return fail(ctx, STMF_ERR_INVALID, "delta_tile_rows %d: 0, 4 or 8", o.delta_tile_rows);
    if (o.delta_blocks_per_sm < 0 || o.delta_blocks_per_sm > (o.delta_tile_rows == 8 ? 4 : 5))
        return fail(ctx, STMF_ERR_INVALID, "delta_blocks_per_sm %d outside [0, %d]", o.delta_blocks_per_sm,
                    o.delta_tile_rows == 8 ? 4 : 5);
    const bool elem = o.strategy == STMF_STRATEGY_BYELEMENT, mat = o.strategy == STMF_STRATEGY_BYMATRIX;
    if ((elem || mat) && (o.perm || o.selection != STMF_SEL_TD_A))
        return fail(ctx, STMF_ERR_INVALID, "the %s strategy takes no row permutation and no selection",
                    elem ? "ByElement" : "ByMatrix");
    const int tr = m0 > n0;                 // Algorithm 3: a tall R is transposed
    const int m = tr ? n0 : m0, n = tr ? m0 : n0;
    std::vector<int> perm;
    if (o.perm) {
        perm.assign(o.perm, o.perm + m);
        std::vector<char> seen(m, 0);
        for (int x : perm) {
            if (x < 0 || x >= m || seen[x]) return fail(ctx, STMF_ERR_INVALID, "perm is not a permutation of 0..%d", m - 1);
            seen[x] = 1;
        }
    } else if (elem || mat) {
        perm.resize(m);                     // ByElement and ByMatrix keep the rows in their order
        for (int s = 0; s < m; ++s) perm[s] = s;
    } else {
        random_permutation(m, o.seed, perm);
    }
    const int window = o.window ? (o.window + 1) / 2 * 2 : STMF_WMAX;
    stmf_problem *P = nullptr;
    s = problem_alloc(ctx, m, n, r, window, &P);
    if (s != STMF_OK) return s;
    P->transposed = tr; P->m0 = m0; P->n0 = n0;
    P->sel = o.selection;
    P->strategy = o.strategy;
    P->res_chunk_sel = o.res_chunk;
    P->delta_bps_sel = o.delta_blocks_per_sm;
    P->delta_rows_sel = o.delta_tile_rows;
    {
        cudaError_t ea = cudaSuccess;
        if (P->sel == STMF_SEL_TD) {
            ea = dalloc(&P->rowkey, P->np);
            if (ea == cudaSuccess) ea = dalloc(&P->rowrank, P->np);
            if (ea == cudaSuccess) ea = dalloc(&P->roworder, P->np);
        } else if (P->sel == STMF_SEL_TD_B) {
            ea = dalloc(&P->colarg, P->np);
        }
        if (mat && ea == cudaSuccess) {
            P->coin_key = o.seed ^ 0x5A5A5A5A5A5A5A5Aull;
            ea = dalloc(&P->tdr_seq, (size_t)m);
            if (ea == cudaSuccess) ea = dalloc(&P->tdc_seq, (size_t)n);
            if (ea == cudaSuccess) ea = dalloc(&P->scnt, 1);
        }
        if (ea != cudaSuccess) {
            problem_free(P);
            cudaGetLastError();
            return fail(ctx, STMF_ERR_OOM, "selection buffers: %s", cudaGetErrorString(ea));
        }
    }
    cudaStream_t st = ctx->stream;
    if (o.precision == 1) {
        // half planes and screen partials; the planes are written by every
        // refresh from here on (the first one is in problem_init)
        const size_t cells = (size_t)P->mp * P->np;
        const size_t nblk = (size_t)(P->m + SCR_ROWS - 1) / SCR_ROWS;
        cudaError_t ea = dalloc(&P->Rh, cells);
        if (ea == cudaSuccess) ea = dalloc(&P->P1h, cells);
        if (ea == cudaSuccess) ea = dalloc(&P->P2h, cells);
        if (ea == cudaSuccess) ea = dalloc(&P->scr_sum, STMF_WMAX * nblk);
        if (ea == cudaSuccess) ea = dalloc(&P->scr_cnt, STMF_WMAX * nblk);
        if (ea == cudaSuccess) ea = dalloc(&P->scr_umax, STMF_WMAX);
        if (ea == cudaSuccess) ea = dalloc(&P->scr_vmax, STMF_WMAX);
        if (ea == cudaSuccess) ea = screen_prepare(P);
        if (ea != cudaSuccess) {
            problem_free(P);
            cudaGetLastError();
            return fail(ctx, STMF_ERR_OOM, "FP16 screening buffers: %s", cudaGetErrorString(ea));
        }
        P->precision = 1;
    }
    int *d_bad = nullptr;
    cudaError_t e = cudaMalloc(&P->perm, sizeof(int) * m);
    if (e == cudaSuccess) e = cudaMalloc(&d_bad, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->perm, perm.data(), sizeof(int) * m, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_pack_oriented(st, R, ldr, mask, ldm_words, m, n, tr, P->perm, nullptr, P->R,
                                                   P->np, P->mp, d_bad);
    if (e == cudaSuccess && elem) e = setup_permc(P, st, R, ldr, mask, ldm_words, d_bad);
    if (e == cudaSuccess && mat) {
        e = count_given(P, st);
        P->nsort = matrix_sort_len(P->ngiven);
        if (e == cudaSuccess) {
            cudaError_t ea = dalloc(&P->skey, P->nsort);
            if (ea == cudaSuccess) ea = dalloc(&P->sval, P->nsort);
            if (ea != cudaSuccess) {
                if (d_bad) cudaFree(d_bad);
                problem_free(P);
                cudaGetLastError();
                return fail(ctx, STMF_ERR_OOM, "ByMatrix order buffers: %s", cudaGetErrorString(ea));
            }
        }
    }
    int bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (d_bad) cudaFree(d_bad);
    if (e != cudaSuccess) { problem_free(P); return fail(ctx, STMF_ERR_CUDA, "pack: %s", cudaGetErrorString(e)); }
    if (bad) { problem_free(P); return fail(ctx, STMF_ERR_INVALID, "a given entry of R is not finite or has magnitude >= 2^60"); }
    float *U0_learned = nullptr;
    if (o.mlp && !o.U0) {
        stmf_mlp *net = const_cast<stmf_mlp *>(o.mlp);
        if (mlp_rank(net) != r) { problem_free(P); return fail(ctx, STMF_ERR_INVALID, "the MLP's rank is not r"); }
        if (cudaMalloc(&U0_learned, sizeof(float) * (size_t)m * r) != cudaSuccess) {
            problem_free(P);
            cudaGetLastError();
            return fail(ctx, STMF_ERR_OOM, "learned initialisation buffer");
        }
        s = mlp_predict_rows(ctx, net, m, n, P->R, P->np, nullptr, 0, U0_learned);
        if (s != STMF_OK) { cudaFree(U0_learned); problem_free(P); return s; }
    }
    s = problem_init(P, o.U0 ? o.U0 : U0_learned, o.acol_p, o.seed, o.picks, o.U0 ? o.V0 : nullptr);
    if (U0_learned) cudaFree(U0_learned);
    if (s != STMF_OK) { problem_free(P); return s; }
    e = cudaSuccess;
    if (o.trace && o.trace_cap > 0) {
        e = cudaMalloc(&P->trace_dev, sizeof(int32_t) * STMF_TRACE_INTS * (size_t)o.trace_cap);
        if (e == cudaSuccess) e = set_ctl(P, &stmf_ctl::trace, P->trace_dev);
        if (e == cudaSuccess) e = set_ctl(P, &stmf_ctl::trace_cap, (long long)o.trace_cap);
    }
    if (e == cudaSuccess) e = set_ctl(P, &stmf_ctl::select_mode, o.select);
    if (e == cudaSuccess) e = set_loop_bounds(P);
    if (e != cudaSuccess) { problem_free(P); return fail(ctx, STMF_ERR_CUDA, "trace buffer: %s", cudaGetErrorString(e)); }
    s = read_ctl(P);
    if (s != STMF_OK) { problem_free(P); return s; }
    P->f_init = P->ctl_host->f;
    *out = P;
    return STMF_OK;
}

// Bounds of the device-driven loops.  A row (ByElement: a segment of the
// scan) consumes at least one position of its order per window, so it never
// needs more windows than the order has positions; a sweep never visits more
// rows (segments) than m n + 1.  Reaching a bound means a logic error: the
// loops stop with STMF_ERR_TIMEOUT instead of running on.  For tests,
// STMF_TEST_WINDOW_CAP=N in the environment sets the window bound to N.
cudaError_t set_loop_bounds(stmf_problem *P)
{
    long long lim = P->n;
    if (P->sel == STMF_SEL_SEQ) lim = (long long)P->n * P->r;
    if (P->strategy == STMF_STRATEGY_BYELEMENT || P->strategy == STMF_STRATEGY_BYMATRIX) lim = (long long)P->m * P->n;
    long long win_cap = lim + 4;          // and up to two placeholders (short rows)
    const char *t = getenv("STMF_TEST_WINDOW_CAP");
    if (t && atoll(t) > 0) win_cap = atoll(t);
    cudaError_t e = set_ctl(P, &stmf_ctl::win_cap, win_cap);
    if (e == cudaSuccess) e = set_ctl(P, &stmf_ctl::row_cap, (long long)P->m * P->n + 2);
    return e;
}

stmf_status device_error(stmf_problem *P, int q)
{
    const int err = P->ctl_host->err;
    if (err == STMF_ERR_TIMEOUT)
        return fail(P->ctx, STMF_ERR_TIMEOUT, "problem %d: a bound of the device-driven loops ran out (%lld windows "
                    "in one row, %lld row visits in one sweep)", q, P->ctl_host->win_row, P->ctl_host->rows_sweep);
    return fail(P->ctx, STMF_ERR_INTERNAL, "problem %d: device error %d", q, err);
}

stmf_status fastmf_run(stmf_problem *P, int sweeps, double eps)
{
    stmf_ctx *ctx = P->ctx;
    cudaStream_t st = ctx->stream;
    const bool graph = use_graph();
    if (graph && !P->sweep_exec) {
        stmf_status s = build_sweep_graph(P);
        if (s != STMF_OK) return s;
    }
    auto t0 = std::chrono::steady_clock::now();
    for (int sw = 0; sw < sweeps; ++sw) {
        NvtxRange range("stmf sweep");
        const double f_prev = P->ctl_host->f;
        CK(set_ctl(P, &stmf_ctl::sweep, P->sweeps_done));
        if (graph) {
            CK(cudaGraphLaunch(P->sweep_exec, st));
        } else {
            stmf_status s = sweep_host(P);
            if (s != STMF_OK) return s;
        }
        stmf_status s = read_ctl(P);
        if (s != STMF_OK) return s;
        if (P->ctl_host->err) return device_error(P, 0);
        P->sweeps_done += 1;
        const double f = P->ctl_host->f;
        if (eps > 0.0 && f_prev - f < eps && f - f_prev < eps) break;
    }
    if (P->ctl_host->dirty_k != -2) {
        stmf_status s = refresh(P);
        if (s != STMF_OK) return s;
        s = read_ctl(P);
        if (s != STMF_OK) return s;
    }
    auto t1 = std::chrono::steady_clock::now();
    P->seconds += std::chrono::duration<double>(t1 - t0).count();
    return STMF_OK;
}

void fill_report(const stmf_problem *P, stmf_report *rep)
{
    if (!rep) return;
    memset(rep, 0, sizeof(*rep));
    const stmf_ctl &c = *P->ctl_host;
    rep->f_init = P->f_init;
    rep->f_final = c.f;
    rep->sweeps_done = P->sweeps_done;
    rep->transposed = P->transposed;
    rep->candidates_tried = c.tried;
    rep->candidates_issued = c.issued;
    rep->accepted = c.accepted;
    rep->refreshes = c.refreshes;
    rep->windows = c.windows;
    rep->trace_records = c.ntrace;
    rep->eval_ns = c.eval_ns;
    rep->eval_launches = c.eval_launches;
    rep->eval_candidates = c.eval_cands;
    rep->seconds = P->seconds;
    rep->candidates_screened = c.screened;
    rep->eval_res_ns = c.res_ns;
    rep->eval_delta_ns = c.delta_ns;
    rep->candidates_discarded = c.discarded;
    rep->eval_res_chunk = res_chunk(P);
    rep->eval_delta_blocks = delta_grid(P);
    rep->eval_delta_rows = delta_rows(P);
}

stmf_status fastmf_end(stmf_problem *P, float *U_out, float *V_out, int32_t *trace_out, int64_t trace_cap)
{
    stmf_ctx *ctx = P->ctx;
    cudaStream_t st = ctx->stream;
    if (U_out && V_out) CK(launch_unorient(st, P, P->transposed, P->perm, P->cperm, U_out, V_out));
    stmf_status s = read_ctl(P);
    if (s != STMF_OK) return s;
    if (trace_out && P->trace_dev) {
        const long long nrec = P->ctl_host->ntrace < trace_cap ? P->ctl_host->ntrace : trace_cap;
        if (nrec > 0)
            CK(cudaMemcpyAsync(trace_out, P->trace_dev, sizeof(int32_t) * STMF_TRACE_INTS * nrec,
                               cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return STMF_OK;
}

// ------------------------------------------------------------ autotuner
// Autotuner of a problem size class: the launch shapes of the window
// evaluation (phase 1's column chunk, phase 2's thread-tile rows and blocks
// per SM).  Each trial runs the first rows of sweep 0 on a scratch copy of the
// problem, host-driven, with every window full (64 candidates from each
// row's start, as in the later sweeps, where rows scan thousands of
// candidates); the shapes change no decision, so every trial evaluates the
// same windows, and each phase's shape is scored by the mean %globaltimer
// span of its own kernel.  The window itself is not tuned: it is the largest
// (64 candidates), since a row's first window already adapts to what the
// previous row consumed, and trials in sweep 0, whose rows keep an update
// within a few windows, favoured smaller caps that multiply the windows of
// the later sweeps (four problems of up to 1294 x 6914 entries, 10 sweeps
// each, ran at 0.80x of one problem at a time with them).
struct tune_result {
    int window, res_chunk, delta_bps, delta_rows;
};

stmf_status fastmf_begin(stmf_ctx *ctx, int m0, int n0, int r, const float *R, int ldr, const uint32_t *mask,
                         int ldm_words, const stmf_options *opts, stmf_problem **out);
stmf_status sweep_rows_host(stmf_problem *P, int rows);

uint64_t size_class(int m, int n, int r)
{
    const int mo = m < n ? m : n, no = m < n ? n : m;
    const double e = (double)stmf_roundup(mo, STMF_PAD) * stmf_roundup(no, STMF_PAD);
    const int lg = (int)std::floor(std::log2(e));
    return ((uint64_t)lg << 8) | (uint64_t)r;
}

// One trial: window w, shapes (chunk, bps, rows) (0: defaults).  Returns
// the mean durations of the two phases' launches; *chunk_used, *rows_used
// (nullable) the chunk and tile rows the trial ran with.
stmf_status tune_trial(stmf_ctx *ctx, const stmf_batch_problem &bp, const stmf_options &base, int w, int chunk,
                       int bps, int rows, double *res_s, double *delta_s, int *chunk_used, int *rows_used = nullptr)
{
    stmf_options o = base;
    o.window = w; o.trace = nullptr; o.trace_cap = 0; o.perm = nullptr; o.picks = nullptr; o.U0 = nullptr;
    o.V0 = nullptr;
    o.seed = bp.seed;
    stmf_problem *P = nullptr;
    CS(fastmf_begin(ctx, bp.m, bp.n, bp.r, bp.R, bp.ldr, bp.mask, bp.ldm_words, &o, &P));
    const int full = P->ctl_host->wmax / 2;                   // j-candidates of a full window
    stmf_status sf = STMF_OK;
    if (set_ctl(P, &stmf_ctl::wj0_fixed, full) != cudaSuccess || set_ctl(P, &stmf_ctl::wj0, full) != cudaSuccess)
        sf = fail(ctx, STMF_ERR_CUDA, "autotuner set-up failed");
    if (sf != STMF_OK) { problem_free(P); return sf; }
    P->res_chunk_sel = chunk;
    P->delta_bps_sel = bps;
    P->delta_rows_sel = rows;
    if (chunk_used) *chunk_used = res_chunk(P);
    if (rows_used) *rows_used = delta_rows(P);
    stmf_status s = sweep_rows_host(P, 24);
    if (s == STMF_OK) s = read_ctl(P);
    if (s != STMF_OK) { problem_free(P); return s; }
    const stmf_ctl &c = *P->ctl_host;
    const double nl = c.eval_launches > 0 ? (double)c.eval_launches : 1.0;
    *res_s = c.res_ns * 1e-9 / nl;
    *delta_s = c.delta_ns * 1e-9 / nl;
    problem_free(P);
    return STMF_OK;
}

stmf_status tune_shapes(stmf_ctx *ctx, const stmf_batch_problem &bp, const stmf_options &base, tune_result *best)
{
    auto *cache = static_cast<std::map<uint64_t, tune_result> *>(ctx->tune);
    if (!cache) ctx->tune = cache = new std::map<uint64_t, tune_result>();
    const uint64_t key = size_class(bp.m, bp.n, bp.r);
    auto it = cache->find(key);
    if (it != cache->end()) { *best = it->second; return STMF_OK; }
    tune_result t = {STMF_WMAX, 0, 0, 0};
    double best_res, best_delta;
    int chunk0 = 0, rows0 = 4;
    CS(tune_trial(ctx, bp, base, t.window, 0, 0, 0, &best_res, &best_delta, &chunk0, &rows0));
    // the defaults (measured above: the wave heuristic's chunk, the size's
    // default tile rows) against neighbouring chunks and the other tile
    // heights and blocks per SM
    t.res_chunk = chunk0;
    t.delta_rows = rows0;
    t.delta_bps = rows0 == 8 ? 3 : 5;
    // phase 2: the other tile height at its default blocks per SM, and the
    // default height at one block per SM fewer
    const int other = rows0 == 8 ? 4 : 8;
    const int alt[2][3] = {{chunk0 - 8, other, other == 8 ? 3 : 5}, {chunk0 + 8, rows0, t.delta_bps - 1}};
    for (int a = 0; a < 2; ++a) {
        const int ch = alt[a][0] >= 32 && alt[a][0] <= 128 ? alt[a][0] : chunk0;
        double rs, ds;
        CS(tune_trial(ctx, bp, base, t.window, ch, alt[a][2], alt[a][1], &rs, &ds, nullptr));
        if (rs < best_res) { best_res = rs; t.res_chunk = ch; }
        if (ds < best_delta) { best_delta = ds; t.delta_bps = alt[a][2]; t.delta_rows = alt[a][1]; }
    }
    (*cache)[key] = t;
    *best = t;
    return STMF_OK;
}

// Rows 0..rows-1 of sweep 0, host-driven (used by the autotuner).
stmf_status sweep_rows_host(stmf_problem *P, int rows)
{
    stmf_ctx *ctx = P->ctx;
    cudaStream_t st = ctx->stream;
    CK(launch_sweep_begin(st, P, 0));
    stmf_status s = read_ctl(P);
    if (s != STMF_OK) return s;
    const int nr = rows < P->m ? rows : P->m;
    for (int i = 0; i < nr && P->ctl_host->more; ++i) {
        if (P->ctl_host->dirty_k != -2) CS(refresh(P));
        CS(row_host(P));
    }
    return STMF_OK;
}

// ------------------------------------------------------------ batched form
stmf_status batched(stmf_ctx *ctx, int nprob, const stmf_batch_problem *probs, const stmf_options *opts,
                    stmf_report *reports, int *tuned)
{
    stmf_options o;
    if (opts) o = *opts; else stmf_default_options(&o);
    if (o.precision < 0 || o.precision > 1) return fail(ctx, STMF_ERR_INVALID, "precision mode %d unknown", o.precision);
    if (o.window < 0 || o.window > STMF_WMAX) return fail(ctx, STMF_ERR_INVALID, "window outside [0, %d]", STMF_WMAX);
    for (int q = 0; q < nprob; ++q) {
        const stmf_batch_problem &b = probs[q];
        CS(check_common(ctx, b.m, b.n, b.r));
        if (!b.R || !b.U_out || !b.V_out) return fail(ctx, STMF_ERR_INVALID, "problem %d: R, U_out, V_out required", q);
        if (b.ldr < b.n) return fail(ctx, STMF_ERR_INVALID, "problem %d: ldr < n", q);
        if (b.mask && b.ldm_words < (b.n + 31) / 32) return fail(ctx, STMF_ERR_INVALID, "problem %d: ldm_words", q);
        if (b.sweeps < 0) return fail(ctx, STMF_ERR_INVALID, "problem %d: sweeps < 0", q);
        if (b.trace_cap < 0 || (b.trace_cap > 0 && !b.trace))
            return fail(ctx, STMF_ERR_INVALID, "problem %d: trace_cap without a trace buffer", q);
    }
    std::vector<tune_result> tr(nprob, tune_result{o.window ? (o.window + 1) / 2 * 2 : 0, 0, 0, 0});
    if (!o.window)
        for (int q = 0; q < nprob; ++q) CS(tune_shapes(ctx, probs[q], o, &tr[q]));
    if (tuned)
        for (int q = 0; q < nprob; ++q) tuned[q] = tr[q].window;

    std::vector<stmf_problem *> Ps(nprob, nullptr);
    struct Free { std::vector<stmf_problem *> &v; ~Free() { for (auto *p : v) problem_free(p); } } fr{Ps};
    for (int q = 0; q < nprob; ++q) {
        const stmf_batch_problem &b = probs[q];
        stmf_options po = o;
        po.window = tr[q].window; po.seed = b.seed; po.perm = nullptr; po.picks = nullptr; po.U0 = nullptr;
        po.V0 = nullptr;
        po.trace = b.trace_cap > 0 ? b.trace : nullptr;
        po.trace_cap = b.trace_cap > 0 ? b.trace_cap : 0;
        CS(fastmf_begin(ctx, b.m, b.n, b.r, b.R, b.ldr, b.mask, b.ldm_words, &po, &Ps[q]));
        if (!o.res_chunk) Ps[q]->res_chunk_sel = tr[q].res_chunk;          // the caller's shapes win
        if (!o.delta_tile_rows && !o.delta_blocks_per_sm) {
            Ps[q]->delta_rows_sel = tr[q].delta_rows;
            Ps[q]->delta_bps_sel = tr[q].delta_bps;
        }
        CK(set_ctl(Ps[q], &stmf_ctl::sweep_target, b.sweeps));
        CK(set_ctl(Ps[q], &stmf_ctl::eps, o.eps));
        CK(set_ctl(Ps[q], &stmf_ctl::sweep, 0));
    }
    // one graph: one independent device-driven job per problem
    cudaStream_t cap;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    struct SG { cudaStream_t s; ~SG() { cudaStreamDestroy(s); } } sg{cap};
    cudaGraph_t g;
    CK(cudaGraphCreate(&g, 0));
    struct GG { cudaGraph_t g; cudaGraphExec_t x = nullptr; ~GG() { if (x) cudaGraphExecDestroy(x); cudaGraphDestroy(g); } } gg{g};
    // A problem whose phase 2 fills every SM on its own gains nothing from
    // running beside another such problem and loses L2: each one's per-window
    // working set (R, R^T, P1, P2, A) fits the L2 only alone.  Those run one
    // after another, in input order; the smaller ones run side by side.
    cudaGraphNode_t prev = nullptr;
    for (int q = 0; q < nprob; ++q) {
        const bool big = delta_fills_gpu(Ps[q]);
        cudaGraphNode_t end = nullptr;
        CS(add_problem_nodes(Ps[q], g, g, true, cap, big && prev ? &prev : nullptr, big && prev ? 1 : 0, &end));
        if (big) prev = end;
    }
    CK(cudaGraphInstantiate(&gg.x, g, 0));
    cudaStream_t st = ctx->stream;
    CK(cudaStreamSynchronize(st));
    auto t0 = std::chrono::steady_clock::now();
    CK(cudaGraphLaunch(gg.x, st));
    CK(cudaStreamSynchronize(st));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int q = 0; q < nprob; ++q) {
        stmf_problem *P = Ps[q];
        CS(read_ctl(P));
        if (P->ctl_host->err) return device_error(P, q);
        if (P->ctl_host->dirty_k != -2) { CS(refresh(P)); CS(read_ctl(P)); }
        P->sweeps_done = P->ctl_host->sweep;
        P->seconds = secs;
        CS(fastmf_end(P, probs[q].U_out, probs[q].V_out, probs[q].trace_cap > 0 ? probs[q].trace : nullptr,
                      probs[q].trace_cap));
        if (reports) fill_report(P, &reports[q]);
    }
    CK(cudaStreamSynchronize(st));
    return STMF_OK;
}

}  // namespace

extern "C" {

void stmf_struct_sizes(size_t *options, size_t *report, size_t *batch_problem)
{
    if (options) *options = sizeof(stmf_options);
    if (report) *report = sizeof(stmf_report);
    if (batch_problem) *batch_problem = sizeof(stmf_batch_problem);
}

void stmf_default_options(stmf_options *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->sweeps = 1;
    o->window = 0;
    o->acol_p = 5;
}

stmf_status stmf_create(stmf_ctx **out, int device, void *cuda_stream)
{
    if (!out) return STMF_ERR_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return STMF_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return STMF_ERR_CUDA;
    stmf_ctx *c = new stmf_ctx();
    memset(c, 0, sizeof(*c));
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    *out = c;
    return STMF_OK;
}

void stmf_destroy(stmf_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->ws) cudaFree(ctx->ws);
    delete static_cast<std::map<uint64_t, tune_result> *>(ctx->tune);
    delete ctx;
}

const char *stmf_last_error(const stmf_ctx *ctx) { return ctx ? ctx->err : "no context"; }

stmf_status stmf_set_stream(stmf_ctx *ctx, void *cuda_stream)
{
    if (!ctx) return STMF_ERR_INVALID;
    ctx->stream = (cudaStream_t)cuda_stream;
    return STMF_OK;
}

stmf_status stmf_maxplus(stmf_ctx *ctx, int m, int n, int r, const float *U, int ldu, const float *V, int ldv,
                         const uint32_t *mask, int ldm_words, float *P1, int ldp, uint8_t *A, int lda, float *P2)
{
    stmf_status s = check_common(ctx, m, n, r);
    if (s != STMF_OK) return s;
    if (!U || !V || !P1) return fail(ctx, STMF_ERR_INVALID, "U, V and P1 are required");
    if (ldu < r || ldv < n || ldp < n || (A && lda < n))
        return fail(ctx, STMF_ERR_INVALID, "leading dimension too small");
    if (mask && ldm_words < (n + 31) / 32) return fail(ctx, STMF_ERR_INVALID, "ldm_words < ceil(n/32)");
    CK(launch_maxplus(ctx->stream, m, n, r, U, ldu, V, ldv, mask, ldm_words, P1, ldp, A, lda, P2, nullptr, 0,
                      nullptr, nullptr));
    return STMF_OK;
}

stmf_status stmf_selection_stats(stmf_ctx *ctx, int m, int n, int r, const float *R, int ldr,
                                 const uint32_t *mask, int ldm_words, const float *U, int ldu, const float *V,
                                 int ldv, double *td_col, int32_t *colhist, double *f_host)
{
    stmf_status s = check_common(ctx, m, n, r);
    if (s != STMF_OK) return s;
    if (!R || !U || !V) return fail(ctx, STMF_ERR_INVALID, "R, U and V are required");
    if (ldr < n || ldu < r || ldv < n) return fail(ctx, STMF_ERR_INVALID, "leading dimension too small");
    if (mask && ldm_words < (n + 31) / 32) return fail(ctx, STMF_ERR_INVALID, "ldm_words < ceil(n/32)");
    const int nparts = planes_nparts(m);
    const size_t need = sizeof(double) * ((size_t)nparts * n + n + 1) + sizeof(int) * (size_t)nparts * n * r + 256;
    if (ctx->ws_bytes < need) {
        if (ctx->ws) cudaFree(ctx->ws);
        ctx->ws = nullptr; ctx->ws_bytes = 0;
        CK(cudaMalloc(&ctx->ws, need));
        ctx->ws_bytes = need;
    }
    double *tdpart = (double *)ctx->ws;
    double *tdtmp = tdpart + (size_t)nparts * n;
    double *fdev = tdtmp + n;
    int *chpart = (int *)(fdev + 1);
    cudaStream_t st = ctx->stream;
    CK(launch_maxplus(st, m, n, r, U, ldu, V, ldv, mask, ldm_words, nullptr, 0, nullptr, 0, nullptr, R, ldr,
                      tdpart, chpart));
    double *tdout = td_col ? td_col : tdtmp;
    CK(launch_td_finalize2(st, tdpart, chpart, nparts, n, n, r, tdout, colhist));
    if (f_host) {
        CK(launch_error_sum(st, tdout, n, fdev));
        CK(cudaMemcpyAsync(f_host, fdev, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return STMF_OK;
}

stmf_status stmf_rmse(stmf_ctx *ctx, int m, int n, int r, const float *R, int ldr, const uint32_t *mask,
                      int ldm_words, const float *U, int ldu, const float *V, int ldv, double *out_host)
{
    stmf_status s = check_common(ctx, m, n, r);
    if (s != STMF_OK) return s;
    if (!R || !U || !V || !out_host) return fail(ctx, STMF_ERR_INVALID, "R, U, V and out are required");
    if (ldr < n || ldu < r || ldv < n) return fail(ctx, STMF_ERR_INVALID, "leading dimension too small");
    if (mask && ldm_words < (n + 31) / 32) return fail(ctx, STMF_ERR_INVALID, "ldm_words < ceil(n/32)");
    const size_t need = sizeof(double) * (4 * (size_t)rmse_blocks(m, ctx->num_sms) + 4) + 256;
    if (ctx->ws_bytes < need) {
        if (ctx->ws) cudaFree(ctx->ws);
        ctx->ws = nullptr; ctx->ws_bytes = 0;
        CK(cudaMalloc(&ctx->ws, need));
        ctx->ws_bytes = need;
    }
    double *part = (double *)ctx->ws;
    double *out = part + 4 * (size_t)rmse_blocks(m, ctx->num_sms);
    cudaStream_t st = ctx->stream;
    CK(launch_rmse(st, ctx->num_sms, m, n, r, R, ldr, mask, ldm_words, U, ldu, V, ldv, part, out));
    CK(cudaMemcpyAsync(out_host, out, sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return STMF_OK;
}

stmf_status stmf_problem_create(stmf_ctx *ctx, int m, int n, int r, const float *R, int ldr, const uint32_t *mask,
                                int ldm_words, const float *U0, const stmf_options *opts, stmf_problem **out)
{
    if (!out) return fail(ctx, STMF_ERR_INVALID, "out is NULL");
    *out = nullptr;
    stmf_status s = check_common(ctx, m, n, r);
    if (s != STMF_OK) return s;
    if (!R) return fail(ctx, STMF_ERR_INVALID, "R is required");
    if (ldr < n) return fail(ctx, STMF_ERR_INVALID, "ldr < n");
    if (mask && ldm_words < (n + 31) / 32) return fail(ctx, STMF_ERR_INVALID, "ldm_words < ceil(n/32)");
    stmf_options o;
    if (opts) o = *opts; else stmf_default_options(&o);
    stmf_problem *P = nullptr;
    s = problem_alloc(ctx, m, n, r, STMF_WMAX, &P);
    if (s != STMF_OK) return s;
    int *d_bad = nullptr;
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaMalloc(&d_bad, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_pack(st, R, ldr, mask, ldm_words, m, n, P->R, P->np, P->mp, d_bad);
    int bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (d_bad) cudaFree(d_bad);
    if (e != cudaSuccess) { problem_free(P); return fail(ctx, STMF_ERR_CUDA, "pack: %s", cudaGetErrorString(e)); }
    if (bad) { problem_free(P); return fail(ctx, STMF_ERR_INVALID, "a given entry of R is not finite or has magnitude >= 2^60"); }
    s = problem_init(P, U0, o.acol_p, o.seed, o.picks);
    if (s != STMF_OK) { problem_free(P); return s; }
    s = read_ctl(P);
    if (s != STMF_OK) { problem_free(P); return s; }
    P->f_init = P->ctl_host->f;
    *out = P;
    return STMF_OK;
}

void stmf_problem_destroy(stmf_problem *P) { problem_free(P); }

stmf_status stmf_update_U(stmf_problem *P, int i, int j, int k, int commit_if_decreases, double *f_new, int *accepted)
{
    return update(P, i, j, k, 0, commit_if_decreases, f_new, accepted);
}

stmf_status stmf_update_V(stmf_problem *P, int i, int j, int k, int commit_if_decreases, double *f_new, int *accepted)
{
    return update(P, i, j, k, 1, commit_if_decreases, f_new, accepted);
}

stmf_status stmf_problem_get(stmf_problem *P, float *U, float *V, double *f)
{
    if (!P) return STMF_ERR_INVALID;
    stmf_ctx *ctx = P->ctx;
    cudaStream_t st = ctx->stream;
    CK(cudaSetDevice(ctx->device));
    if (U) CK(cudaMemcpyAsync(U, P->U, sizeof(float) * P->m * P->r, cudaMemcpyDeviceToDevice, st));
    if (V) CK(cudaMemcpy2DAsync(V, sizeof(float) * P->n, P->V, sizeof(float) * P->np, sizeof(float) * P->n, P->r,
                                cudaMemcpyDeviceToDevice, st));
    if (f) {
        stmf_status s = read_ctl(P);
        if (s != STMF_OK) return s;
        *f = P->ctl_host->f;
    }
    return STMF_OK;
}

stmf_status stmf_factorize_begin(stmf_ctx *ctx, int m, int n, int r, const float *R, int ldr, const uint32_t *mask,
                                 int ldm_words, const stmf_options *opts, stmf_problem **out)
{
    if (!out) return fail(ctx, STMF_ERR_INVALID, "out is NULL");
    return fastmf_begin(ctx, m, n, r, R, ldr, mask, ldm_words, opts, out);
}

stmf_status stmf_factorize_run(stmf_problem *P, int sweeps, double eps, stmf_report *report)
{
    if (!P) return STMF_ERR_INVALID;
    if (sweeps < 0) return fail(P->ctx, STMF_ERR_INVALID, "sweeps < 0");
    CK2(P->ctx, cudaSetDevice(P->ctx->device));
    stmf_status s = fastmf_run(P, sweeps, eps);
    if (s != STMF_OK) return s;
    fill_report(P, report);
    return STMF_OK;
}

stmf_status stmf_factorize_end(stmf_problem *P, float *U_out, float *V_out, int32_t *trace, int64_t trace_cap)
{
    if (!P) return STMF_ERR_INVALID;
    CK2(P->ctx, cudaSetDevice(P->ctx->device));
    return fastmf_end(P, U_out, V_out, trace, trace_cap);
}

stmf_status stmf_factorize(stmf_ctx *ctx, int m0, int n0, int r, const float *R, int ldr, const uint32_t *mask,
                           int ldm_words, const stmf_options *opts, float *U_out, float *V_out, stmf_report *rep)
{
    if (!U_out || !V_out) return fail(ctx, STMF_ERR_INVALID, "U_out and V_out are required");
    stmf_options o;
    if (opts) o = *opts; else stmf_default_options(&o);
    if (o.sweeps < 0) return fail(ctx, STMF_ERR_INVALID, "sweeps < 0");
    stmf_problem *P = nullptr;
    stmf_status s;
    {
        NvtxRange range("stmf prepare (orientation, init, planes)");
        s = fastmf_begin(ctx, m0, n0, r, R, ldr, mask, ldm_words, &o, &P);
    }
    if (s != STMF_OK) return s;
    s = fastmf_run(P, o.sweeps, o.eps);
    if (s == STMF_OK) s = fastmf_end(P, U_out, V_out, o.trace, o.trace_cap);
    if (s == STMF_OK) fill_report(P, rep);
    problem_free(P);
    return s;
}

stmf_status stmf_factorize_batched(stmf_ctx *ctx, int nprob, const stmf_batch_problem *probs,
                                   const stmf_options *opts, stmf_report *reports, int *tuned_windows)
{
    if (!ctx) return STMF_ERR_INVALID;
    if (nprob < 0 || (nprob > 0 && !probs)) return fail(ctx, STMF_ERR_INVALID, "bad problem list");
    if (nprob == 0) return STMF_OK;
    NvtxRange range("stmf batched factorization");
    return batched(ctx, nprob, probs, opts, reports, tuned_windows);
}

stmf_status stmf_peak_addmax(stmf_ctx *ctx, int mode, int iters, double *gops)
{
    if (!ctx || !gops || iters < 1 || mode < 0 || mode > 7) return fail(ctx, STMF_ERR_INVALID, "bad arguments");
    CK(cudaSetDevice(ctx->device));
    float *sink = nullptr;
    CK(cudaMalloc(&sink, 256 * sizeof(float)));
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    const int blocks = ctx->num_sms * 8;
    CK(launch_peak(ctx->stream, mode, iters / 10 + 1, blocks, sink));   // warm-up
    CK(cudaEventRecord(a, ctx->stream));
    CK(launch_peak(ctx->stream, mode, iters, blocks, sink));
    CK(cudaEventRecord(b, ctx->stream));
    CK(cudaEventSynchronize(b));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    *gops = peak_ops(mode, iters, blocks) / (ms * 1e-3) / 1e9;
    return STMF_OK;
}

}  // extern "C"
