// Learned initialisation of U (an addition to the paper, which initialises
// with Random Acol).  A row of R is summarised by a 32-quantile sketch of its
// given entries, centred on the row median; an MLP 32 -> 128 -> 128 -> r
// (ReLU) maps the sketch to the row of U minus the median.  Weights are held
// in BF16 for the forward pass and in FP32 (master copy) for Adam; every
// product accumulates in FP32.  Kernels here: the row sketch, forward,
// backward (deterministic: every gradient element is one thread's fixed-order
// sum over the batch), Adam and the BF16 refresh.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"

#define SK 32          // sketch length
#define HID 128        // hidden width

namespace {

// ---------------------------------------------------------------- sketch
// One block per row: the given entries are sorted in shared memory (bitonic,
// padded with +inf), then sketch[q] = v[floor((q + 0.5) * cnt / 32)] - median,
// median = v[floor(cnt / 2)]  (nearest-rank quantiles).
__global__ void __launch_bounds__(1024) k_row_sketch(const float *__restrict__ R, int ldr,
                                                     const uint32_t *__restrict__ mask, int ldm, int m, int n,
                                                     int npow2, float *__restrict__ sketch, float *__restrict__ med)
{
    extern __shared__ float sv[];
    __shared__ int scnt;
    const int s = blockIdx.x;
    if (threadIdx.x == 0) scnt = 0;
    __syncthreads();
    // compact the given entries (order irrelevant: they are sorted next)
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const float v = R[(size_t)s * ldr + t];
        const bool given = mask ? ((mask[(size_t)s * ldm + (t >> 5)] >> (t & 31)) & 1u) : v == v;
        if (given) {
            const int p = atomicAdd(&scnt, 1);
            sv[p] = v;
        }
    }
    __syncthreads();
    const int cnt = scnt;
    for (int t = cnt + threadIdx.x; t < npow2; t += blockDim.x) sv[t] = INFINITY;
    __syncthreads();
    for (int k = 2; k <= npow2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < npow2; t += blockDim.x) {
                const int p = t ^ j;
                if (p > t) {
                    const bool up = (t & k) == 0;
                    const float a = sv[t], b = sv[p];
                    if ((a > b) == up) { sv[t] = b; sv[p] = a; }
                }
            }
            __syncthreads();
        }
    if (cnt == 0) {
        if (threadIdx.x < SK) sketch[(size_t)s * SK + threadIdx.x] = 0.f;
        if (threadIdx.x == 0) med[s] = 0.f;
        return;
    }
    const float md = sv[cnt / 2];
    if (threadIdx.x < SK) {
        const int idx = (int)(((double)threadIdx.x + 0.5) * cnt / SK);
        sketch[(size_t)s * SK + threadIdx.x] = sv[min(idx, cnt - 1)] - md;
    }
    if (threadIdx.x == 0) med[s] = md;
}

// ---------------------------------------------------------------- forward
// 32 rows of the batch per block, one thread per hidden unit.  Stores the
// hidden activations for the backward pass (H1, H2 may be NULL at inference).
__global__ void __launch_bounds__(HID) k_mlp_fwd(int B, int r, const float *__restrict__ X,
                                                 const __nv_bfloat16 *__restrict__ W1, const float *__restrict__ b1,
                                                 const __nv_bfloat16 *__restrict__ W2, const float *__restrict__ b2,
                                                 const __nv_bfloat16 *__restrict__ W3, const float *__restrict__ b3,
                                                 float *__restrict__ H1, float *__restrict__ H2, float *__restrict__ Y)
{
    __shared__ float sx[32][SK];
    __shared__ float sh1[32][HID + 1];
    __shared__ float sh2[32][HID + 1];
    const int j = threadIdx.x, row0 = blockIdx.x * 32;
    const int nr = min(32, B - row0);
    for (int e = j; e < 32 * SK; e += HID) {
        const int a = e / SK, c = e % SK;
        sx[a][c] = a < nr ? X[(size_t)(row0 + a) * SK + c] : 0.f;
    }
    __syncthreads();
    float w[SK];
#pragma unroll
    for (int i = 0; i < SK; ++i) w[i] = __bfloat162float(W1[i * HID + j]);
    for (int a = 0; a < nr; ++a) {
        float acc = b1[j];
#pragma unroll
        for (int i = 0; i < SK; ++i) acc = fmaf(sx[a][i], w[i], acc);
        acc = fmaxf(acc, 0.f);
        sh1[a][j] = acc;
        if (H1) H1[(size_t)(row0 + a) * HID + j] = acc;
    }
    __syncthreads();
    for (int a = 0; a < nr; ++a) {
        float acc = b2[j];
        for (int i = 0; i < HID; ++i) acc = fmaf(sh1[a][i], __bfloat162float(W2[i * HID + j]), acc);
        acc = fmaxf(acc, 0.f);
        sh2[a][j] = acc;
        if (H2) H2[(size_t)(row0 + a) * HID + j] = acc;
    }
    __syncthreads();
    for (int e = j; e < nr * r; e += HID) {
        const int a = e / r, o = e % r;
        float acc = b3[o];
        for (int i = 0; i < HID; ++i) acc = fmaf(sh2[a][i], __bfloat162float(W3[i * r + o]), acc);
        Y[(size_t)(row0 + a) * r + o] = acc;
    }
}

// ---------------------------------------------------------------- backward
// dY = 2 (Y - T) / (B r) (mean squared error); loss partials per row.
__global__ void k_mse(int B, int r, const float *__restrict__ Y, const float *__restrict__ T, float *__restrict__ dY,
                      double *__restrict__ rowloss)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= B) return;
    double l = 0.0;
    for (int o = 0; o < r; ++o) {
        const float d = Y[(size_t)a * r + o] - T[(size_t)a * r + o];
        dY[(size_t)a * r + o] = 2.f * d / (float)(B * r);
        l += (double)d * d;
    }
    rowloss[a] = l / (double)(B * r);
}

// dH[a][i] = (H[a][i] > 0) * sum_o dOut[a][o] * W[i][o]   (W: in x out, BF16)
__global__ void k_back_act(int B, int in, int out, const float *__restrict__ dOut, const __nv_bfloat16 *__restrict__ W,
                           const float *__restrict__ H, float *__restrict__ dH)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= B * in) return;
    const int a = e / in, i = e % in;
    float acc = 0.f;
    for (int o = 0; o < out; ++o) acc = fmaf(dOut[(size_t)a * out + o], __bfloat162float(W[(size_t)i * out + o]), acc);
    dH[e] = H[e] > 0.f ? acc : 0.f;
}

// gW[i][o] = sum_a In[a][i] * dOut[a][o];  gb[o] = sum_a dOut[a][o]  (fixed order over a)
__global__ void k_back_w(int B, int in, int out, const float *__restrict__ In, const float *__restrict__ dOut,
                         float *__restrict__ gW, float *__restrict__ gb)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < in * out) {
        const int i = e / out, o = e % out;
        float acc = 0.f;
        for (int a = 0; a < B; ++a) acc = fmaf(In[(size_t)a * in + i], dOut[(size_t)a * out + o], acc);
        gW[e] = acc;
    } else if (e < in * out + out) {
        const int o = e - in * out;
        float acc = 0.f;
        for (int a = 0; a < B; ++a) acc += dOut[(size_t)a * out + o];
        gb[o] = acc;
    }
}

// Adam (Kingma and Ba) on the FP32 master parameters, then the BF16 copy.
__global__ void k_adam(int np, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m1,
                       float *__restrict__ m2, float lr, float b1, float b2, float eps, float c1, float c2,
                       __nv_bfloat16 *__restrict__ pb, int nbf)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= np) return;
    const float gi = g[e];
    const float a = b1 * m1[e] + (1.f - b1) * gi;
    const float b = b2 * m2[e] + (1.f - b2) * gi * gi;
    m1[e] = a;
    m2[e] = b;
    const float v = p[e] - lr * (a / c1) / (sqrtf(b / c2) + eps);
    p[e] = v;
    if (e < nbf) pb[e] = __float2bfloat16_rn(v);
}

__global__ void k_to_bf16(int n, const float *__restrict__ p, __nv_bfloat16 *__restrict__ pb)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) pb[e] = __float2bfloat16_rn(p[e]);
}

}  // namespace

// Parameter layout (FP32 master, and BF16 copy of the weights in the same order):
//   W1 [SK x HID] | W2 [HID x HID] | W3 [HID x r] | b1 [HID] | b2 [HID] | b3 [r]
struct stmf_mlp {
    stmf_ctx *ctx;
    int r, np, nw;     // parameters, weights (the BF16 part)
    float *p, *g, *m1, *m2;
    __nv_bfloat16 *pb;
    int step;
    int cap;           // batch capacity of the work buffers
    float *H1, *H2, *Y, *dY, *dH2, *dH1;
    double *rowloss;
};

namespace {

int mlp_nw(int r) { return SK * HID + HID * HID + HID * r; }
int mlp_np(int r) { return mlp_nw(r) + HID + HID + r; }

stmf_status mfail(stmf_ctx *ctx, stmf_status st, const char *msg)
{
    if (ctx) snprintf(ctx->err, sizeof(ctx->err), "%s", msg);
    return st;
}

void mlp_free_work(stmf_mlp *M)
{
    void *q[] = {M->H1, M->H2, M->Y, M->dY, M->dH2, M->dH1, M->rowloss};
    for (void *x : q)
        if (x) cudaFree(x);
    M->H1 = M->H2 = M->Y = M->dY = M->dH2 = M->dH1 = nullptr;
    M->rowloss = nullptr;
    M->cap = 0;
}

cudaError_t mlp_reserve(stmf_mlp *M, int B)
{
    if (B <= M->cap) return cudaSuccess;
    mlp_free_work(M);
    cudaError_t e = cudaMalloc(&M->H1, sizeof(float) * (size_t)B * HID);
    if (e == cudaSuccess) e = cudaMalloc(&M->H2, sizeof(float) * (size_t)B * HID);
    if (e == cudaSuccess) e = cudaMalloc(&M->Y, sizeof(float) * (size_t)B * M->r);
    if (e == cudaSuccess) e = cudaMalloc(&M->dY, sizeof(float) * (size_t)B * M->r);
    if (e == cudaSuccess) e = cudaMalloc(&M->dH2, sizeof(float) * (size_t)B * HID);
    if (e == cudaSuccess) e = cudaMalloc(&M->dH1, sizeof(float) * (size_t)B * HID);
    if (e == cudaSuccess) e = cudaMalloc(&M->rowloss, sizeof(double) * (size_t)B);
    if (e == cudaSuccess) M->cap = B;
    return e;
}

void launch_fwd(stmf_mlp *M, int B, const float *X, float *H1, float *H2, float *Y)
{
    const __nv_bfloat16 *W1 = M->pb, *W2 = W1 + SK * HID, *W3 = W2 + HID * HID;
    const float *b1 = M->p + M->nw, *b2 = b1 + HID, *b3 = b2 + HID;
    k_mlp_fwd<<<(B + 31) / 32, HID, 0, M->ctx->stream>>>(B, M->r, X, W1, b1, W2, b2, W3, b3, H1, H2, Y);
}

// U0[s][l] = Y[s][l] + median[s]
__global__ void k_add_median(const float *__restrict__ Y, const float *__restrict__ med, int m, int r,
                             float *__restrict__ U0)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m * r) U0[e] = Y[e] + med[e / r];
}

}  // namespace

// Learned initial rows of a problem (the addition to Algorithm 3's Random
// Acol start): U0[s] = MLP(sketch of row s) + median of row s, with the row's
// given entries those of R that are not NaN.  Runs on ctx's stream, which must
// be the MLP's.
stmf_status mlp_predict_rows(stmf_ctx *ctx, stmf_mlp *M, int m, int n, const float *R, int ldr, float *U0)
{
    if (M->ctx != ctx) return mfail(ctx, STMF_ERR_INVALID, "the MLP was created on another context");
    if (n > 12288) return mfail(ctx, STMF_ERR_INVALID, "learned initialisation needs n <= 12288 (row sketch)");
    float *buf = nullptr;
    const size_t nsk = (size_t)m * SK, nmd = (size_t)m, ny = (size_t)m * M->r;
    cudaError_t e = cudaMalloc(&buf, sizeof(float) * (nsk + nmd + ny));
    if (e != cudaSuccess) return mfail(ctx, STMF_ERR_OOM, cudaGetErrorString(e));
    float *sk = buf, *md = buf + nsk, *Y = md + nmd;
    int np2 = 1;
    while (np2 < n) np2 <<= 1;
    const size_t smem = sizeof(float) * np2;
    if (smem > 48 * 1024)
        e = cudaFuncSetAttribute(k_row_sketch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        k_row_sketch<<<m, 1024, smem, ctx->stream>>>(R, ldr, nullptr, 0, m, n, np2, sk, md);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        launch_fwd(M, m, sk, nullptr, nullptr, Y);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_add_median<<<(unsigned)((ny + 255) / 256), 256, 0, ctx->stream>>>(Y, md, m, M->r, U0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(buf);
    return e == cudaSuccess ? STMF_OK : mfail(ctx, STMF_ERR_CUDA, cudaGetErrorString(e));
}

int mlp_rank(const stmf_mlp *M) { return M->r; }

extern "C" {

stmf_status stmf_row_sketch(stmf_ctx *ctx, int m, int n, const float *R, int ldr, const uint32_t *mask,
                            int ldm_words, float *sketch, float *median)
{
    if (!ctx) return STMF_ERR_INVALID;
    if (m < 1 || n < 1 || n > 12288) return mfail(ctx, STMF_ERR_INVALID, "sketch needs 1 <= n <= 12288");
    if (!R || !sketch || !median || ldr < n) return mfail(ctx, STMF_ERR_INVALID, "bad sketch arguments");
    if (mask && ldm_words < (n + 31) / 32) return mfail(ctx, STMF_ERR_INVALID, "ldm_words < ceil(n/32)");
    int np2 = 1;
    while (np2 < n) np2 <<= 1;
    const size_t smem = sizeof(float) * np2;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess && smem > 48 * 1024)
        e = cudaFuncSetAttribute(k_row_sketch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        k_row_sketch<<<m, 1024, smem, ctx->stream>>>(R, ldr, mask, ldm_words, m, n, np2, sketch, median);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return mfail(ctx, STMF_ERR_CUDA, cudaGetErrorString(e));
    return STMF_OK;
}

stmf_status stmf_mlp_create(stmf_ctx *ctx, int r, const float *params_host, stmf_mlp **out)
{
    if (!ctx || !out || r < 1 || r > STMF_MAX_RANK || !params_host)
        return mfail(ctx, STMF_ERR_INVALID, "bad MLP arguments");
    stmf_mlp *M = new stmf_mlp();
    memset(M, 0, sizeof(*M));
    M->ctx = ctx; M->r = r; M->np = mlp_np(r); M->nw = mlp_nw(r);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaMalloc(&M->p, sizeof(float) * M->np);
    if (e == cudaSuccess) e = cudaMalloc(&M->g, sizeof(float) * M->np);
    if (e == cudaSuccess) e = cudaMalloc(&M->m1, sizeof(float) * M->np);
    if (e == cudaSuccess) e = cudaMalloc(&M->m2, sizeof(float) * M->np);
    if (e == cudaSuccess) e = cudaMalloc(&M->pb, sizeof(__nv_bfloat16) * M->nw);
    if (e == cudaSuccess) e = cudaMemcpyAsync(M->p, params_host, sizeof(float) * M->np, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(M->m1, 0, sizeof(float) * M->np, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(M->m2, 0, sizeof(float) * M->np, ctx->stream);
    if (e == cudaSuccess) {
        k_to_bf16<<<(M->nw + 255) / 256, 256, 0, ctx->stream>>>(M->nw, M->p, M->pb);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        stmf_mlp_destroy(M);
        return mfail(ctx, e == cudaErrorMemoryAllocation ? STMF_ERR_OOM : STMF_ERR_CUDA, cudaGetErrorString(e));
    }
    *out = M;
    return STMF_OK;
}

void stmf_mlp_destroy(stmf_mlp *M)
{
    if (!M) return;
    mlp_free_work(M);
    void *q[] = {M->p, M->g, M->m1, M->m2, M->pb};
    for (void *x : q)
        if (x) cudaFree(x);
    delete M;
}

int stmf_mlp_param_count(int r) { return (r < 1 || r > STMF_MAX_RANK) ? -1 : mlp_np(r); }

stmf_status stmf_mlp_get_params(stmf_mlp *M, float *params_host)
{
    if (!M || !params_host) return STMF_ERR_INVALID;
    cudaError_t e = cudaMemcpyAsync(params_host, M->p, sizeof(float) * M->np, cudaMemcpyDeviceToHost, M->ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(M->ctx->stream);
    return e == cudaSuccess ? STMF_OK : mfail(M->ctx, STMF_ERR_CUDA, cudaGetErrorString(e));
}

stmf_status stmf_mlp_forward(stmf_mlp *M, int B, const float *X, float *Y)
{
    if (!M || B < 1 || !X || !Y) return STMF_ERR_INVALID;
    cudaError_t e = cudaSetDevice(M->ctx->device);
    if (e == cudaSuccess) {
        launch_fwd(M, B, X, nullptr, nullptr, Y);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? STMF_OK : mfail(M->ctx, STMF_ERR_CUDA, cudaGetErrorString(e));
}

stmf_status stmf_mlp_gradient(stmf_mlp *M, int B, const float *X, const float *T, double *loss, float *grad_host)
{
    if (!M || B < 1 || !X || !T) return STMF_ERR_INVALID;
    stmf_ctx *ctx = M->ctx;
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = mlp_reserve(M, B);
    if (e != cudaSuccess) return mfail(ctx, STMF_ERR_OOM, cudaGetErrorString(e));
    const int r = M->r;
    const __nv_bfloat16 *W2 = M->pb + SK * HID, *W3 = W2 + HID * HID;
    float *gW1 = M->g, *gW2 = gW1 + SK * HID, *gW3 = gW2 + HID * HID;
    float *gb1 = M->g + M->nw, *gb2 = gb1 + HID, *gb3 = gb2 + HID;
    launch_fwd(M, B, X, M->H1, M->H2, M->Y);
    k_mse<<<(B + 255) / 256, 256, 0, st>>>(B, r, M->Y, T, M->dY, M->rowloss);
    k_back_w<<<(HID * r + r + 255) / 256, 256, 0, st>>>(B, HID, r, M->H2, M->dY, gW3, gb3);
    k_back_act<<<(B * HID + 255) / 256, 256, 0, st>>>(B, HID, r, M->dY, W3, M->H2, M->dH2);
    k_back_w<<<(HID * HID + HID + 255) / 256, 256, 0, st>>>(B, HID, HID, M->H1, M->dH2, gW2, gb2);
    k_back_act<<<(B * HID + 255) / 256, 256, 0, st>>>(B, HID, HID, M->dH2, W2, M->H1, M->dH1);
    k_back_w<<<(SK * HID + HID + 255) / 256, 256, 0, st>>>(B, SK, HID, X, M->dH1, gW1, gb1);
    e = cudaGetLastError();
    if (e == cudaSuccess && loss) {
        std::vector<double> h(B);
        e = cudaMemcpyAsync(h.data(), M->rowloss, sizeof(double) * B, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        double l = 0.0;
        for (int a = 0; a < B; ++a) l += h[a];
        *loss = l;
    }
    if (e == cudaSuccess && grad_host) {
        e = cudaMemcpyAsync(grad_host, M->g, sizeof(float) * M->np, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    return e == cudaSuccess ? STMF_OK : mfail(ctx, STMF_ERR_CUDA, cudaGetErrorString(e));
}

stmf_status stmf_mlp_train_step(stmf_mlp *M, int B, const float *X, const float *T, float lr, double *loss)
{
    stmf_status s = stmf_mlp_gradient(M, B, X, T, loss, nullptr);
    if (s != STMF_OK) return s;
    M->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)M->step), c2 = 1.f - powf(b2, (float)M->step);
    k_adam<<<(M->np + 255) / 256, 256, 0, M->ctx->stream>>>(M->np, M->p, M->g, M->m1, M->m2, lr, b1, b2, 1e-8f, c1,
                                                            c2, M->pb, M->nw);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? STMF_OK : mfail(M->ctx, STMF_ERR_CUDA, cudaGetErrorString(e));
}

}  // extern "C"
