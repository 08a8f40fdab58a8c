// Host side of the C ABI declared in include/stmf.h: argument validation,
// device workspaces, set-up of a problem, the F-ULF / F-URF single updates
// and the row loop of Algorithm 3 (FastSTMF).
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <chrono>
#include <vector>

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

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
cudaError_t dalloc(T **p, size_t count)
{
    return cudaMalloc((void **)p, sizeof(T) * (count ? count : 1));
}

void problem_free(stmf_problem *P)
{
    if (!P) return;
    void *ptrs[] = {P->R, P->RT, P->U, P->V, P->P1, P->P2, P->A, P->cmin1, P->cmin2, P->carg,
                    P->rmin1, P->rmin2, P->rarg, P->tdpart, P->chpart, P->tdcol, P->colhist,
                    P->rowhist, P->order, P->cand, P->Uc, P->Vc, P->part_ulf, P->part_urf, P->fc,
                    P->ctl};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (P->ctl_host) cudaFreeHost(P->ctl_host);
    delete P;
}

stmf_status problem_alloc(stmf_ctx *ctx, int m, int n, int r, int window, stmf_problem **out)
{
    stmf_problem *P = new stmf_problem();
    memset(P, 0, sizeof(*P));
    P->ctx = ctx;
    P->m = m; P->n = n; P->r = r;
    P->mp = stmf_roundup(m, STMF_PAD);
    P->np = stmf_roundup(n, STMF_PAD);
    P->window = window;
    P->dirty_k = -1;
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
    A(dalloc(&P->order, np)); A(dalloc(&P->cand, 8 * STMF_WMAX));
    A(dalloc(&P->Uc, (size_t)STMF_WMAX * mp)); A(dalloc(&P->Vc, (size_t)STMF_WMAX * np));
    A(dalloc(&P->part_ulf, (mp / 4) * STMF_WMAX)); A(dalloc(&P->part_urf, (np / 32) * STMF_WMAX));
    A(dalloc(&P->fc, STMF_WMAX)); A(dalloc(&P->ctl, 1));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&P->ctl_host, sizeof(stmf_ctl));
    if (e != cudaSuccess) {
        problem_free(P);
        cudaGetLastError();
        return fail(ctx, STMF_ERR_OOM, "device allocation for a %dx%d rank-%d problem failed: %s", m, n, r,
                    cudaGetErrorString(e));
    }
    cudaStream_t st = ctx->stream;
    e = cudaMemsetAsync(P->U, 0, sizeof(float) * mp * r, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->V, 0, sizeof(float) * r * np, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->ctl, 0, sizeof(stmf_ctl), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->P1, 0, sizeof(float) * mp * np, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->P2, 0, sizeof(float) * mp * np, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->A, 0, mp * np, st);
    if (e != cudaSuccess) { problem_free(P); return fail(ctx, STMF_ERR_CUDA, "memset: %s", cudaGetErrorString(e)); }
    *out = P;
    return STMF_OK;
}

// Statistics of component k (or of all components when k < 0):
//   column statistics from U_.k over RT, row statistics from V_k. over R.
stmf_status refresh_stats(stmf_problem *P, int k)
{
    stmf_ctx *ctx = P->ctx;
    cudaStream_t st = ctx->stream;
    const int k0 = k < 0 ? 0 : k, k1 = k < 0 ? P->r : k + 1;
    for (int l = k0; l < k1; ++l) {
        CK(launch_rowstat(st, P->RT, P->mp, P->n, P->m, P->U + l, P->r, P->cmin1 + (size_t)l * P->np,
                          P->cmin2 + (size_t)l * P->np, P->carg + (size_t)l * P->np));
        CK(launch_rowstat(st, P->R, P->np, P->m, P->n, P->V + (size_t)l * P->np, 1, P->rmin1 + (size_t)l * P->mp,
                          P->rmin2 + (size_t)l * P->mp, P->rarg + (size_t)l * P->mp));
    }
    return STMF_OK;
}

// Product planes, td_col, colhist, the column order and the current error.
stmf_status refresh_planes(stmf_problem *P)
{
    stmf_ctx *ctx = P->ctx;
    cudaStream_t st = ctx->stream;
    CK(launch_planes(st, P, P->chpart));
    CK(launch_td_finalize2(st, P->tdpart, P->chpart, planes_nparts(P->m), P->np, P->n, P->r, P->tdcol, P->colhist));
    CK(launch_order(st, P->tdcol, P->n, P->order));
    CK(launch_eval(st, P, 1));
    CK(launch_select(st, P, 2));
    P->refreshes++;
    return STMF_OK;
}

stmf_status refresh(stmf_problem *P, int k)
{
    stmf_status s = refresh_stats(P, k);
    if (s != STMF_OK) return s;
    return refresh_planes(P);
}

// After R (and RT) are packed: checks, U, V, statistics, planes, error.
stmf_status problem_init(stmf_problem *P, const float *U0, int acol_p, uint64_t seed, const int32_t *picks_in)
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
    // V = (-U)^T (x)* R: the column minima of component l are min1 of its
    // column statistics.
    stmf_status s = refresh_stats(P, -1);
    if (s != STMF_OK) return s;
    CK(launch_copy_rows(st, P->cmin1, P->np, P->V, P->np, P->r, P->n));
    s = refresh_stats(P, -1);   // row statistics of the new V
    if (s != STMF_OK) return s;
    s = refresh_planes(P);
    if (s != STMF_OK) return s;
    P->dirty_k = -2;
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
    CK(cudaMemcpyAsync(&rij, P->R + (size_t)i * P->np + j, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (rij != rij) return fail(ctx, STMF_ERR_INVALID, "R[%d][%d] is not given", i, j);
    cudaStream_t st = ctx->stream;
    CK(launch_single(st, P, i, j, k, type));
    CK(launch_seed(st, P, 1));
    CK(launch_eval(st, P, 0));
    CK(launch_select(st, P, 0));
    if (!commit_if_decreases) CK(launch_commit0(st, P));
    stmf_status s = read_ctl(P);
    if (s != STMF_OK) return s;
    const int kept = P->ctl_host->kept;
    const double fn = commit_if_decreases ? P->ctl_host->f_new : 0.0;
    double fval;
    CK(cudaMemcpyAsync(&fval, P->fc, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    (void)fn;
    if (f_new) *f_new = fval;
    if (accepted) *accepted = kept;
    if (kept) {
        s = refresh(P, k);
        if (s != STMF_OK) return s;
    }
    return STMF_OK;
}

void put_trace(const stmf_options *o, int64_t &nrec, int sweep, int i, int pos, int j, int k, int type, double f)
{
    if (!o || !o->trace || nrec >= o->trace_cap) return;
    int32_t *rec = o->trace + STMF_TRACE_INTS * nrec;
    rec[0] = sweep; rec[1] = i; rec[2] = pos; rec[3] = j; rec[4] = k; rec[5] = type;
    memcpy(rec + 6, &f, sizeof(double));
    ++nrec;
}

}  // namespace

extern "C" {

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
    const size_t need = sizeof(double) * ((size_t)nparts * n + n) + sizeof(int) * (size_t)nparts * n * r + 256;
    if (ctx->ws_bytes < need) {
        if (ctx->ws) cudaFree(ctx->ws);
        ctx->ws = nullptr; ctx->ws_bytes = 0;
        CK(cudaMalloc(&ctx->ws, need));
        ctx->ws_bytes = need;
    }
    double *tdpart = (double *)ctx->ws;
    double *tdtmp = tdpart + (size_t)nparts * n;
    int *chpart = (int *)(tdtmp + n);
    cudaStream_t st = ctx->stream;
    CK(launch_maxplus(st, m, n, r, U, ldu, V, ldv, mask, ldm_words, nullptr, 0, nullptr, 0, nullptr, R, ldr,
                      tdpart, chpart));
    double *tdout = td_col ? td_col : tdtmp;
    CK(launch_td_finalize2(st, tdpart, chpart, nparts, n, n, r, tdout, colhist));
    if (f_host) {
        std::vector<double> h(n);
        CK(cudaMemcpyAsync(h.data(), tdout, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        double f = 0.0;
        for (int t = 0; t < n; ++t) f += h[t];
        *f_host = f;
    }
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
    if (bad) { problem_free(P); return fail(ctx, STMF_ERR_INVALID, "a given entry of R is not finite"); }
    s = problem_init(P, U0, o.acol_p, o.seed, o.picks);
    if (s != STMF_OK) { problem_free(P); return s; }
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
        *f = P->ctl_host->f_ulf;
    }
    return STMF_OK;
}

stmf_status stmf_factorize(stmf_ctx *ctx, int m0, int n0, int r, const float *R, int ldr, const uint32_t *mask,
                           int ldm_words, const stmf_options *opts, float *U_out, float *V_out, stmf_report *rep)
{
    stmf_status s = check_common(ctx, m0, n0, r);
    if (s != STMF_OK) return s;
    if (!R || !U_out || !V_out) return fail(ctx, STMF_ERR_INVALID, "R, U_out and V_out are required");
    if (ldr < n0) return fail(ctx, STMF_ERR_INVALID, "ldr < n");
    if (mask && ldm_words < (n0 + 31) / 32) return fail(ctx, STMF_ERR_INVALID, "ldm_words < ceil(n/32)");
    stmf_options o;
    if (opts) o = *opts; else stmf_default_options(&o);
    if (o.sweeps < 0) return fail(ctx, STMF_ERR_INVALID, "sweeps < 0");
    if (o.window < 0 || o.window > STMF_WMAX) return fail(ctx, STMF_ERR_INVALID, "window outside [0, %d]", STMF_WMAX);
    if (o.precision != 0) return fail(ctx, STMF_ERR_INVALID, "precision mode %d is not available", o.precision);
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
    } else {
        random_permutation(m, o.seed, perm);
    }
    const int window = o.window ? (o.window + 1) / 2 * 2 : STMF_WMAX;
    stmf_problem *P = nullptr;
    s = problem_alloc(ctx, m, n, r, window, &P);
    if (s != STMF_OK) return s;
    struct Guard { stmf_problem *P; ~Guard() { problem_free(P); } } guard{P};
    cudaStream_t st = ctx->stream;
    int *d_perm = nullptr, *d_bad = nullptr;
    CK(cudaMalloc(&d_perm, sizeof(int) * m));
    struct Guard2 { int *a; ~Guard2() { if (a) cudaFree(a); } } g2{d_perm};
    CK(cudaMalloc(&d_bad, sizeof(int)));
    struct Guard3 { int *a; ~Guard3() { if (a) cudaFree(a); } } g3{d_bad};
    CK(cudaMemcpyAsync(d_perm, perm.data(), sizeof(int) * m, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
    CK(launch_pack_oriented(st, R, ldr, mask, ldm_words, m, n, tr, d_perm, P->R, P->np, P->mp, d_bad));
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (bad) return fail(ctx, STMF_ERR_INVALID, "a given entry of R is not finite");
    s = problem_init(P, o.U0, o.acol_p, o.seed, o.picks);
    if (s != STMF_OK) return s;

    s = read_ctl(P);
    if (s != STMF_OK) return s;
    const double f_init = P->ctl_host->f_ulf;
    double f = f_init;
    int64_t nrec = 0;
    int sweeps_done = 0;
    long long accepted = 0;
    const int wj0 = 2;
    auto t0 = std::chrono::steady_clock::now();
    for (int sw = 0; sw < o.sweeps; ++sw) {
        const double f_prev = f;
        for (int i = 0; i < m; ++i) {
            if (P->dirty_k != -2) {
                s = refresh(P, P->dirty_k);
                if (s != STMF_OK) return s;
                P->dirty_k = -2;
            }
            CK(launch_begin_row(st, P, i, wj0));
            while (true) {
                CK(launch_window(st, P));
                CK(launch_seed(st, P, P->window));
                CK(launch_eval(st, P, 0));
                CK(launch_select(st, P, o.select == 1 ? 1 : 0));
                s = read_ctl(P);
                if (s != STMF_OK) return s;
                const stmf_ctl &c = *P->ctl_host;
                if (c.kept) {
                    f = c.f_new;
                    P->dirty_k = c.kept_k;
                    ++accepted;
                    put_trace(&o, nrec, sw, i, c.kept_pos, c.kept_j, c.kept_k, c.kept_type, f);
                    break;
                }
                if (c.row_done) {
                    put_trace(&o, nrec, sw, i, -1, -1, -1, -1, f);
                    break;
                }
            }
        }
        ++sweeps_done;
        if (o.eps > 0.0 && (f_prev - f < o.eps && f - f_prev < o.eps)) break;
    }
    if (P->dirty_k != -2) {
        s = refresh(P, P->dirty_k);
        if (s != STMF_OK) return s;
        P->dirty_k = -2;
    }
    CK(cudaStreamSynchronize(st));
    auto t1 = std::chrono::steady_clock::now();
    CK(launch_unorient(st, P, tr, d_perm, U_out, V_out));
    s = read_ctl(P);
    if (s != STMF_OK) return s;
    if (rep) {
        memset(rep, 0, sizeof(*rep));
        rep->f_init = f_init;
        rep->f_final = P->ctl_host->f_ulf;
        rep->sweeps_done = sweeps_done;
        rep->transposed = tr;
        rep->candidates_tried = P->ctl_host->tried;
        rep->candidates_issued = P->ctl_host->issued;
        rep->accepted = accepted;
        rep->refreshes = P->refreshes;
        rep->seconds = std::chrono::duration<double>(t1 - t0).count();
    }
    return STMF_OK;
}

stmf_status stmf_peak_addmax(stmf_ctx *ctx, int mode, int iters, double *gops)
{
    if (!ctx || !gops || iters < 1 || mode < 0 || mode > 3) return fail(ctx, STMF_ERR_INVALID, "bad arguments");
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
    const double lane_ops = (double)blocks * 256.0 * iters * 8.0 * 2.0 * (mode == 3 ? 2.0 : 1.0);
    *gops = lane_ops / (ms * 1e-3) / 1e9;
    return STMF_OK;
}

}  // extern "C"
