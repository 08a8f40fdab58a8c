// Learned initialisation of U (an addition to the paper, which initialises
// with Random Acol).  A row of R is summarised by a 32-quantile sketch of its
// given entries, centred on the row median; an MLP 32 -> 128 -> 128 -> r
// (ReLU) maps the sketch to the row of U minus the median.  Weights are held
// in BF16 for the products and in FP32 (master copy) for Adam.  Every matrix
// product of the forward and backward passes runs on the tensor cores
// (mma.sync, BF16 operands, FP32 accumulation, fixed order: reproducible).
// Kernels here: the row sketch, the GEMM with its epilogues, the loss, the
// bias gradients, Adam and the BF16 refresh.
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

// ------------------------------------------------------- tensor-core GEMM
// C[M x N] = A[M x K] * B[K x N] on the tensor cores (mma.sync m16n8k16,
// BF16 operands, FP32 accumulation), for every product of the network's
// forward and backward passes.  A(i, k) = A[i*sai + k*sak] and
// B(k, j) = B[k*sbk + j*sbj] are FP32 (activations, gradients: rounded to
// BF16 to nearest even when staged) or BF16 (weights).  Block: 4 warps, a
// 64 x 32 tile of C; warp w owns rows 16w..16w+15 of it, four 8-column MMA
// tiles; K in chunks of 32 through shared memory (rows padded to 40 BF16 so
// the fragment loads are free of bank conflicts).  Epilogues:
//   EPI_STORE     C = acc
//   EPI_BIAS_RELU C = max(acc + bias[j], 0)
//   EPI_BIAS      C = acc + bias[j]
//   EPI_MASK      C = H(i, j) > 0 ? acc : 0   (ReLU derivative, H FP32)
// The summation order is fixed, so the results are reproducible.
enum { EPI_STORE = 0, EPI_BIAS_RELU = 1, EPI_BIAS = 2, EPI_MASK = 3 };
constexpr int GBM = 64, GBN = 32, GBK = 32, GPAD = 40;

__device__ __forceinline__ __nv_bfloat16 to_bf16(float x) { return __float2bfloat16_rn(x); }
__device__ __forceinline__ __nv_bfloat16 to_bf16(__nv_bfloat16 x) { return x; }

template <class TA, class TB, int EPI>
__global__ void __launch_bounds__(128) k_gemm_bf16(int M, int N, int K, const TA *__restrict__ A, int sai, int sak,
                                                   const TB *__restrict__ B, int sbk, int sbj,
                                                   const float *__restrict__ bias, const float *__restrict__ H,
                                                   int ldh, float *__restrict__ C, int ldc)
{
    __shared__ __align__(16) __nv_bfloat16 As[GBM][GPAD];     // [row][k]
    __shared__ __align__(16) __nv_bfloat16 Bs[GBN][GPAD];     // [col][k] (transposed: k pairs adjacent)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = lane >> 2, tig = lane & 3;
    const int i0 = blockIdx.y * GBM, j0 = blockIdx.x * GBN;
    float acc[4][4];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[t][q] = 0.f;
    for (int k0 = 0; k0 < K; k0 += GBK) {
        __syncthreads();
        // stage A (64 x 32) and B (32 x 32); the index that is contiguous in
        // memory runs fastest across threads
        for (int e = tid; e < GBM * GBK; e += 128) {
            const int r = sak == 1 ? e / GBK : e % GBM, c = sak == 1 ? e % GBK : e / GBM;
            const int i = i0 + r, k = k0 + c;
            As[r][c] = (i < M && k < K) ? to_bf16(A[(size_t)i * sai + (size_t)k * sak]) : __float2bfloat16_rn(0.f);
        }
        for (int e = tid; e < GBK * GBN; e += 128) {
            const int c = sbj == 1 ? e % GBN : e / GBK, kk = sbj == 1 ? e / GBN : e % GBK;
            const int j = j0 + c, k = k0 + kk;
            Bs[c][kk] = (j < N && k < K) ? to_bf16(B[(size_t)k * sbk + (size_t)j * sbj]) : __float2bfloat16_rn(0.f);
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < GBK; ks += 16) {
            const int ra = warp * 16 + grp;
            uint32_t a[4];
            a[0] = *reinterpret_cast<const uint32_t *>(&As[ra][ks + 2 * tig]);
            a[1] = *reinterpret_cast<const uint32_t *>(&As[ra + 8][ks + 2 * tig]);
            a[2] = *reinterpret_cast<const uint32_t *>(&As[ra][ks + 2 * tig + 8]);
            a[3] = *reinterpret_cast<const uint32_t *>(&As[ra + 8][ks + 2 * tig + 8]);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int cb = t * 8 + grp;
                const uint32_t b0 = *reinterpret_cast<const uint32_t *>(&Bs[cb][ks + 2 * tig]);
                const uint32_t b1 = *reinterpret_cast<const uint32_t *>(&Bs[cb][ks + 2 * tig + 8]);
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                    "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
                    : "+f"(acc[t][0]), "+f"(acc[t][1]), "+f"(acc[t][2]), "+f"(acc[t][3])
                    : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
            }
        }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + warp * 16 + grp + (q >= 2 ? 8 : 0);
            const int j = j0 + t * 8 + 2 * tig + (q & 1);
            if (i >= M || j >= N) continue;
            float v = acc[t][q];
            if (EPI == EPI_BIAS_RELU) v = fmaxf(v + bias[j], 0.f);
            if (EPI == EPI_BIAS) v = v + bias[j];
            if (EPI == EPI_MASK) v = H[(size_t)i * ldh + j] > 0.f ? v : 0.f;
            C[(size_t)i * ldc + j] = v;
        }
}

template <class TA, class TB, int EPI>
void gemm(cudaStream_t st, int M, int N, int K, const TA *A, int sai, int sak, const TB *B, int sbk, int sbj,
          const float *bias, const float *H, int ldh, float *C, int ldc)
{
    dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM);
    k_gemm_bf16<TA, TB, EPI><<<grid, 128, 0, st>>>(M, N, K, A, sai, sak, B, sbk, sbj, bias, H, ldh, C, ldc);
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

// gb[o] = sum over a of dOut[a][o] in batch order (the bias gradients)
__global__ void k_colsum(int B, int out, const float *__restrict__ dOut, float *__restrict__ gb)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= out) return;
    float acc = 0.f;
    for (int a = 0; a < B; ++a) acc += dOut[(size_t)a * out + o];
    gb[o] = acc;
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

// Forward pass: H1 = relu(X W1 + b1), H2 = relu(H1 W2 + b2), Y = H2 W3 + b3
// (H1, H2: the buffers kept for the backward pass, or scratch).
void launch_fwd(stmf_mlp *M, int B, const float *X, float *H1, float *H2, float *Y)
{
    const __nv_bfloat16 *W1 = M->pb, *W2 = W1 + SK * HID, *W3 = W2 + HID * HID;
    const float *b1 = M->p + M->nw, *b2 = b1 + HID, *b3 = b2 + HID;
    cudaStream_t st = M->ctx->stream;
    gemm<float, __nv_bfloat16, EPI_BIAS_RELU>(st, B, HID, SK, X, SK, 1, W1, HID, 1, b1, nullptr, 0, H1, HID);
    gemm<float, __nv_bfloat16, EPI_BIAS_RELU>(st, B, HID, HID, H1, HID, 1, W2, HID, 1, b2, nullptr, 0, H2, HID);
    gemm<float, __nv_bfloat16, EPI_BIAS>(st, B, M->r, HID, H2, HID, 1, W3, M->r, 1, b3, nullptr, 0, Y, M->r);
}

// U0[s][l] = Y[s][l] + median[s]
__global__ void k_add_median(const float *__restrict__ Y, const float *__restrict__ med, int m, int r,
                             float *__restrict__ U0)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m * r) U0[e] = Y[e] + med[e / r];
}

// ------------------------------------------------------------ targets
// The gauge of a factorization: U (x) V is unchanged by U_.l + c, V_l. - c
// for any c per component, and by any order of the components.  Training
// targets fix it: c_l = max over t < n of V_lt (so that max_t V'_lt = 0), and
// the components go in decreasing order of their sum over rows of U_sl + c_l
// (FP64, rows in index order; equal sums keep the smaller l first).
__global__ void __launch_bounds__(256) k_tgt_colmax(int n, const float *__restrict__ V, int ldv,
                                                    float *__restrict__ c)
{
    __shared__ float red[8];
    const int l = blockIdx.x;
    float x = -INFINITY;
    for (int t = threadIdx.x; t < n; t += 256) x = fmaxf(x, V[(size_t)l * ldv + t]);
#pragma unroll
    for (int o = 16; o; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) x = fmaxf(x, red[w]);
        c[l] = x;
    }
}

// One warp: lane l sums its component in row order, then the lanes rank the
// sums; order[p] = the component at position p.
__global__ void k_tgt_order(int m, int r, const float *__restrict__ U, int ldu, const float *__restrict__ c,
                            int *__restrict__ order)
{
    const int l = threadIdx.x;
    double key = -INFINITY;
    if (l < r) {
        key = 0.0;
        for (int s = 0; s < m; ++s) key += (double)(U[(size_t)s * ldu + l] + c[l]);
    }
    int pos = 0;
    for (int q = 0; q < r; ++q) {
        const double kq = __shfl_sync(0xffffffffu, key, q);
        pos += (kq > key || (kq == key && q < l)) ? 1 : 0;
    }
    if (l < r) order[pos] = l;
}

// Rank of lane l's value x among the r lanes, in decreasing order (equal
// values: the smaller lane first).
__device__ __forceinline__ int desc_rank(float x, int l, int r)
{
    int pos = 0;
    for (int q = 0; q < r; ++q) {
        const float xq = __shfl_sync(0xffffffffu, x, q);
        pos += (xq > x || (xq == x && q < l)) ? 1 : 0;
    }
    return pos;
}

// One warp per row: T[s][p] = (U_s,order[p] + c_order[p]) - median[s]
// (canonical), or the row's values U_sl + c_l in decreasing order, minus the
// median (sorted).  FP32.
__global__ void __launch_bounds__(256) k_tgt_rows(int m, int r, const float *__restrict__ U, int ldu,
                                                  const float *__restrict__ c, const int *__restrict__ order,
                                                  const float *__restrict__ median, int sorted,
                                                  float *__restrict__ T)
{
    const int s = blockIdx.x * 8 + (threadIdx.x >> 5), l = threadIdx.x & 31;
    if (s >= m) return;
    const int comp = sorted ? l : (l < r ? order[l] : 0);
    const float x = l < r ? U[(size_t)s * ldu + comp] + c[comp] : -INFINITY;
    const int p = sorted ? desc_rank(x, l, r) : l;
    if (l < r) T[(size_t)s * r + p] = x - median[s];
}

// One warp per row: out[s][l] = the value of Y[s] whose rank (decreasing)
// equals the rank of U_ref[s][l] in its row (decreasing; equal values: the
// smaller index first).
__global__ void __launch_bounds__(256) k_assign_by_rank(int m, int r, const float *__restrict__ Y, int ldy,
                                                        const float *__restrict__ Uref, int ldu,
                                                        float *__restrict__ out, int ldo)
{
    __shared__ float sv[8][32];
    const int w = threadIdx.x >> 5, s = blockIdx.x * 8 + w, l = threadIdx.x & 31;
    if (s >= m) return;               // whole warps leave together
    const float y = l < r ? Y[(size_t)s * ldy + l] : -INFINITY;
    const float u = l < r ? Uref[(size_t)s * ldu + l] : -INFINITY;
    const int ry = desc_rank(y, l, r), ru = desc_rank(u, l, r);
    if (l < r) sv[w][ry] = y;
    __syncwarp();
    if (l < r) out[(size_t)s * ldo + l] = sv[w][ru];
}

}  // namespace

// Learned initial rows of a problem (the addition to Algorithm 3's Random
// Acol start): U0[s] = MLP(sketch of row s) + median of row s, with the row's
// given entries those the mask marks (mask NULL: those of R that are not
// NaN).  Runs on ctx's stream, which must be the MLP's.
stmf_status mlp_predict_rows(stmf_ctx *ctx, stmf_mlp *M, int m, int n, const float *R, int ldr,
                             const uint32_t *mask, int ldm_words, float *U0)
{
    if (M->ctx != ctx) return mfail(ctx, STMF_ERR_INVALID, "the MLP was created on another context");
    if (n > 12288) return mfail(ctx, STMF_ERR_INVALID, "learned initialisation needs n <= 12288 (row sketch)");
    float *buf = nullptr;
    const size_t nsk = (size_t)m * SK, nmd = (size_t)m, ny = (size_t)m * M->r;
    cudaError_t e = cudaMalloc(&buf, sizeof(float) * (nsk + nmd + ny));
    if (e != cudaSuccess) return mfail(ctx, STMF_ERR_OOM, cudaGetErrorString(e));
    float *sk = buf, *md = buf + nsk, *Y = md + nmd;
    if (e == cudaSuccess) e = mlp_reserve(M, m);     // hidden activations of the forward pass
    int np2 = 1;
    while (np2 < n) np2 <<= 1;
    const size_t smem = sizeof(float) * np2;
    if (e == cudaSuccess && smem > 48 * 1024)
        e = cudaFuncSetAttribute(k_row_sketch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        k_row_sketch<<<m, 1024, smem, ctx->stream>>>(R, ldr, mask, ldm_words, m, n, np2, sk, md);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        launch_fwd(M, m, sk, M->H1, M->H2, Y);
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
    if (e == cudaSuccess) e = mlp_reserve(M, B);
    if (e == cudaSuccess) {
        launch_fwd(M, B, X, M->H1, M->H2, Y);
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
    // forward, then per layer: weight gradient In^T dOut, bias gradient (the
    // column sums of dOut) and the gradient of the layer's input
    // (dOut W^T masked by the ReLU derivative), all GEMMs on the tensor cores
    launch_fwd(M, B, X, M->H1, M->H2, M->Y);
    k_mse<<<(B + 255) / 256, 256, 0, st>>>(B, r, M->Y, T, M->dY, M->rowloss);
    gemm<float, float, EPI_STORE>(st, HID, r, B, M->H2, 1, HID, M->dY, r, 1, nullptr, nullptr, 0, gW3, r);
    k_colsum<<<1, 128, 0, st>>>(B, r, M->dY, gb3);
    gemm<float, __nv_bfloat16, EPI_MASK>(st, B, HID, r, M->dY, r, 1, W3, 1, r, nullptr, M->H2, HID, M->dH2, HID);
    gemm<float, float, EPI_STORE>(st, HID, HID, B, M->H1, 1, HID, M->dH2, HID, 1, nullptr, nullptr, 0, gW2, HID);
    k_colsum<<<1, 128, 0, st>>>(B, HID, M->dH2, gb2);
    gemm<float, __nv_bfloat16, EPI_MASK>(st, B, HID, HID, M->dH2, HID, 1, W2, 1, HID, nullptr, M->H1, HID, M->dH1,
                                         HID);
    gemm<float, float, EPI_STORE>(st, SK, HID, B, X, 1, SK, M->dH1, HID, 1, nullptr, nullptr, 0, gW1, HID);
    k_colsum<<<1, 128, 0, st>>>(B, HID, M->dH1, gb1);
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

stmf_status stmf_mlp_predict(stmf_mlp *M, int m, int n, const float *R, int ldr, const uint32_t *mask,
                             int ldm_words, float *U0)
{
    if (!M) return STMF_ERR_INVALID;
    stmf_ctx *ctx = M->ctx;
    if (m < 1 || n < 1 || !R || !U0 || ldr < n) return mfail(ctx, STMF_ERR_INVALID, "bad prediction arguments");
    if (mask && ldm_words < (n + 31) / 32) return mfail(ctx, STMF_ERR_INVALID, "ldm_words < ceil(n/32)");
    const cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return mfail(ctx, STMF_ERR_CUDA, cudaGetErrorString(e));
    return mlp_predict_rows(ctx, M, m, n, R, ldr, mask, ldm_words, U0);
}

stmf_status stmf_mlp_targets(stmf_ctx *ctx, int m, int n, int r, const float *U, int ldu, const float *V, int ldv,
                             const float *median, int sorted, float *T)
{
    if (!ctx) return STMF_ERR_INVALID;
    if (m < 1 || n < 1 || r < 1 || r > STMF_MAX_RANK || ldu < r || ldv < n || !U || !V || !median || !T)
        return mfail(ctx, STMF_ERR_INVALID, "bad target arguments");
    cudaStream_t st = ctx->stream;
    void *buf = nullptr;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaMalloc(&buf, sizeof(float) * STMF_MAX_RANK + sizeof(int) * STMF_MAX_RANK);
    if (e != cudaSuccess) return mfail(ctx, STMF_ERR_OOM, cudaGetErrorString(e));
    float *c = static_cast<float *>(buf);
    int *order = reinterpret_cast<int *>(c + STMF_MAX_RANK);
    k_tgt_colmax<<<r, 256, 0, st>>>(n, V, ldv, c);
    k_tgt_order<<<1, 32, 0, st>>>(m, r, U, ldu, c, order);
    k_tgt_rows<<<(m + 7) / 8, 256, 0, st>>>(m, r, U, ldu, c, order, median, sorted ? 1 : 0, T);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the scratch lives until the kernels end
    cudaFree(buf);
    return e == cudaSuccess ? STMF_OK : mfail(ctx, STMF_ERR_CUDA, cudaGetErrorString(e));
}

stmf_status stmf_assign_by_rank(stmf_ctx *ctx, int m, int r, const float *Y, int ldy, const float *U_ref, int ldu,
                                float *out, int ldo)
{
    if (!ctx) return STMF_ERR_INVALID;
    if (m < 1 || r < 1 || r > STMF_MAX_RANK || ldy < r || ldu < r || ldo < r || !Y || !U_ref || !out || out == Y)
        return mfail(ctx, STMF_ERR_INVALID, "bad rank-assignment arguments");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) {
        k_assign_by_rank<<<(m + 7) / 8, 256, 0, ctx->stream>>>(m, r, Y, ldy, U_ref, ldu, out, ldo);
        e = cudaGetLastError();
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
