// Masked max-plus product with top-2 tracking and the ByRow / TD_A selection
// statistics fused into its epilogue.
//
//   P1_ij = max_l (U_il + V_lj)        tropical product (Section "Related work")
//   A_ij  = smallest argmax l          f(i,j) (Section "The ByRow strategy")
//   P2_ij = max over l != A_ij         runner-up: max_{l != k} = (A == k ? P2 : P1)
//   td_col[j]   = sum_i |R_ij - P1_ij|  over given entries (FP64)
//   colhist[j,l]= #{given i : A_ij = l}
//
// (max,+) is not a ring, so this is FADD + FMNMX work on the CUDA cores; the
// tensor cores have no (max,+) mode.  One CTA computes a 128 x 128 block as
// four 32 x 128 tiles; each thread owns a 4 x 4 register tile, U and V tiles
// are staged in shared memory (U broadcast along a warp, V read as float4).
#include "common.cuh"

#define QNAN __int_as_float(0x7fffffff)

namespace {

// Compensated FP32 accumulation (TwoSum, Knuth): s + c carries the running sum
// to about u^2 relative accuracy, with FP32 adds only (FP64 is slow on GB300).
__device__ __forceinline__ void two_sum_add(float &s, float &c, float x)
{
    const float t = s + x;
    const float bp = t - s;
    const float e = (s - (t - bp)) + (x - bp);
    s = t;
    c += e;
}

constexpr int TR = 32;     // rows per tile
constexpr int TC = 128;    // columns per tile
constexpr int TILES = 4;   // tiles per CTA (rows of a CTA = TR * TILES)

template <bool STATS, bool MASKED>
__global__ void __launch_bounds__(256)
k_maxplus(int m, int n, int r, const float *__restrict__ U, int ldu,
          const float *__restrict__ V, int ldv, const uint32_t *__restrict__ mask, int ldm,
          float *__restrict__ P1, int ldp, uint8_t *__restrict__ A, int lda,
          float *__restrict__ P2, const float *__restrict__ R, int ldr,
          double *__restrict__ tdpart, int *__restrict__ chpart)
{
    __shared__ float sU[TR][STMF_MAX_RANK + 1];
    __shared__ __align__(16) float sV[STMF_MAX_RANK][TC];
    __shared__ double sTd[8][TC];
    __shared__ int sHist[STATS ? TC * STMF_MAX_RANK : 1];

    const int tid = threadIdx.x, rg = tid >> 5, cl = tid & 31;
    const int col0 = blockIdx.x * TC;
    const int part = blockIdx.y;
    const int c = col0 + cl * 4;

    for (int e = tid; e < r * TC; e += 256) {
        int l = e / TC, b = e % TC, t = col0 + b;
        sV[l][b] = t < n ? V[(size_t)l * ldv + t] : 0.f;
    }
    if (STATS)
        for (int e = tid; e < TC * r; e += 256) sHist[e] = 0;
    double td_acc[4] = {0.0, 0.0, 0.0, 0.0};

    for (int tile = 0; tile < TILES; ++tile) {
        const int row0 = (part * TILES + tile) * TR;
        if (row0 >= m) break;
        __syncthreads();
        for (int e = tid; e < TR * r; e += 256) {
            int a = e / r, l = e % r, s = row0 + a;
            sU[a][l] = s < m ? U[(size_t)s * ldu + l] : 0.f;
        }
        __syncthreads();

        float p1[4][4], p2[4][4];
        int am[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) { p1[i][jj] = -INFINITY; p2[i][jj] = -INFINITY; am[i][jj] = 0; }

        for (int l = 0; l < r; ++l) {
            float u[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) u[i] = sU[rg * 4 + i][l];
            const float4 v4 = *reinterpret_cast<const float4 *>(&sV[l][cl * 4]);
            const float v[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const float s = u[i] + v[jj];
                    // new runner-up = max(old runner-up, min(old max, s)); strict
                    // '>' keeps the smaller l as argmax on ties
                    p2[i][jj] = fmaxf(p2[i][jj], fminf(p1[i][jj], s));
                    am[i][jj] = s > p1[i][jj] ? l : am[i][jj];
                    p1[i][jj] = fmaxf(p1[i][jj], s);
                }
        }

#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int s = row0 + rg * 4 + i;
            if (s >= m) continue;
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int t = c + jj;
                if (t >= n) continue;
                bool given = true;
                if (MASKED && mask) given = (mask[(size_t)s * ldm + (t >> 5)] >> (t & 31)) & 1u;
                float q1 = p1[i][jj], q2 = p2[i][jj];
                int qa = am[i][jj];
                if (STATS) {
                    const float rv = R[(size_t)s * ldr + t];
                    if (MASKED ? given : (rv == rv)) {
                        td_acc[jj] += (double)fabsf(rv - q1);
                        atomicAdd(&sHist[(cl * 4 + jj) * r + qa], 1);
                    }
                } else {
                    if (MASKED && !given) { q1 = QNAN; q2 = QNAN; qa = 255; }
                    if (P1) P1[(size_t)s * ldp + t] = q1;
                    if (P2) P2[(size_t)s * ldp + t] = q2;
                    if (A) A[(size_t)s * lda + t] = (uint8_t)qa;
                }
            }
        }
    }

    if (STATS) {
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) sTd[rg][cl * 4 + jj] = td_acc[jj];
        __syncthreads();
        if (tid < TC) {
            double s = 0.0;
#pragma unroll
            for (int g = 0; g < 8; ++g) s += sTd[g][tid];
            const int t = col0 + tid;
            if (t < n) tdpart[(size_t)part * n + t] = s;
        }
        for (int e = tid; e < TC * r; e += 256) {
            const int t = col0 + e / r;
            if (t < n) chpart[((size_t)part * n + t) * r + e % r] = sHist[e];
        }
    }
}

// Planes for the internal layout (no mask, vector stores), with td_col and
// colhist partials per 128-row part.  The column sums of td are accumulated
// in compensated FP32 per thread and combined in FP64; the histogram lives in
// shared memory as [l][4][32] so the 32 lanes of a warp always hit 32
// different banks.  HALF (FP16 screening) also writes R, P1, P2 rounded to
// nearest half at given entries (a quiet NaN elsewhere) and raises the
// running maxima of |R| and of the finite |P1|, |P2| over given entries.
struct HalfPlanes {
    __half *Rh, *P1h, *P2h;
    unsigned *mr, *mp;
};

__device__ __forceinline__ unsigned pack_halves(__half a, __half b)
{
    return (unsigned)__half_as_ushort(a) | ((unsigned)__half_as_ushort(b) << 16);
}

template <bool HALF>
__global__ void __launch_bounds__(256)
k_maxplus_planes(int m, int n, int r, const float *__restrict__ U, const float *__restrict__ V,
                 int ld, float *__restrict__ P1, uint8_t *__restrict__ A, float *__restrict__ P2,
                 const float *__restrict__ R, double *__restrict__ tdpart, int *__restrict__ chpart,
                 HalfPlanes H)
{
    float hmr = 0.f, hmp = 0.f;
    __shared__ float sU[TR][STMF_MAX_RANK + 1];
    __shared__ __align__(16) float sV[STMF_MAX_RANK][TC];
    __shared__ double sTd[8][TC];
    __shared__ int sHist[STMF_MAX_RANK][4][32];

    const int tid = threadIdx.x, rg = tid >> 5, cl = tid & 31;
    const int col0 = blockIdx.x * TC;
    const int part = blockIdx.y;
    const int c = col0 + cl * 4;

    for (int e = tid; e < r * TC; e += 256) {
        int l = e / TC, b = e % TC;
        sV[l][b] = V[(size_t)l * ld + col0 + b];
    }
    for (int e = tid; e < r * 128; e += 256) (&sHist[0][0][0])[e] = 0;
    float ts[4] = {0.f, 0.f, 0.f, 0.f}, tc[4] = {0.f, 0.f, 0.f, 0.f};

    for (int tile = 0; tile < TILES; ++tile) {
        const int row0 = (part * TILES + tile) * TR;
        if (row0 >= m) break;
        __syncthreads();
        for (int e = tid; e < TR * r; e += 256) {
            int a = e / r, l = e % r;
            sU[a][l] = U[(size_t)(row0 + a) * r + l];
        }
        __syncthreads();

        float p1[4][4], p2[4][4];
        int am[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) { p1[i][jj] = -INFINITY; p2[i][jj] = -INFINITY; am[i][jj] = 0; }

        for (int l = 0; l < r; ++l) {
            float u[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) u[i] = sU[rg * 4 + i][l];
            const float4 v4 = *reinterpret_cast<const float4 *>(&sV[l][cl * 4]);
            const float v[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const float s = u[i] + v[jj];
                    p2[i][jj] = fmaxf(p2[i][jj], fminf(p1[i][jj], s));
                    am[i][jj] = s > p1[i][jj] ? l : am[i][jj];
                    p1[i][jj] = fmaxf(p1[i][jj], s);
                }
        }

#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const size_t off = (size_t)(row0 + rg * 4 + i) * ld + c;
            const float4 r4 = *reinterpret_cast<const float4 *>(R + off);
            const float rv[4] = {r4.x, r4.y, r4.z, r4.w};
            float q1[4], q2[4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const bool given = rv[jj] == rv[jj];
                q1[jj] = given ? p1[i][jj] : STMF_SENTINEL;
                q2[jj] = given ? p2[i][jj] : STMF_SENTINEL;
            }
            *reinterpret_cast<float4 *>(P1 + off) = make_float4(q1[0], q1[1], q1[2], q1[3]);
            *reinterpret_cast<float4 *>(P2 + off) = make_float4(q2[0], q2[1], q2[2], q2[3]);
            const uint32_t packed = (uint32_t)am[i][0] | ((uint32_t)am[i][1] << 8) |
                                    ((uint32_t)am[i][2] << 16) | ((uint32_t)am[i][3] << 24);
            *reinterpret_cast<uint32_t *>(A + off) = packed;
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                if (rv[jj] == rv[jj]) {   // given entry (not NaN)
                    two_sum_add(ts[jj], tc[jj], fabsf(rv[jj] - p1[i][jj]));
                    atomicAdd(&sHist[am[i][jj]][jj][cl], 1);
                }
            }
            if (HALF) {
                __half hr[4], h1[4], h2[4];
                const __half qnan = __ushort_as_half((unsigned short)0x7e00);
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const bool given = rv[jj] == rv[jj];
                    hr[jj] = given ? __float2half_rn(rv[jj]) : qnan;
                    h1[jj] = given ? __float2half_rn(p1[i][jj]) : qnan;
                    h2[jj] = given ? __float2half_rn(p2[i][jj]) : qnan;
                    if (given) {
                        hmr = fmaxf(hmr, fabsf(rv[jj]));
                        hmp = fmaxf(hmp, fabsf(p1[i][jj]));
                        if (fabsf(p2[i][jj]) < INFINITY) hmp = fmaxf(hmp, fabsf(p2[i][jj]));
                    }
                }
                *reinterpret_cast<uint2 *>(H.Rh + off) = make_uint2(pack_halves(hr[0], hr[1]), pack_halves(hr[2], hr[3]));
                *reinterpret_cast<uint2 *>(H.P1h + off) = make_uint2(pack_halves(h1[0], h1[1]), pack_halves(h1[2], h1[3]));
                *reinterpret_cast<uint2 *>(H.P2h + off) = make_uint2(pack_halves(h2[0], h2[1]), pack_halves(h2[2], h2[3]));
            }
        }
    }
    if (HALF) {
        // non-negative floats order like their bit patterns
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            hmr = fmaxf(hmr, __shfl_xor_sync(0xffffffffu, hmr, o));
            hmp = fmaxf(hmp, __shfl_xor_sync(0xffffffffu, hmp, o));
        }
        if (cl == 0) {
            atomicMax(H.mr, __float_as_uint(hmr));
            atomicMax(H.mp, __float_as_uint(hmp));
        }
    }
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) sTd[rg][cl * 4 + jj] = (double)ts[jj] + (double)tc[jj];
    __syncthreads();
    if (tid < TC) {
        double s = 0.0;
#pragma unroll
        for (int g = 0; g < 8; ++g) s += sTd[g][tid];
        tdpart[(size_t)part * ld + col0 + tid] = s;
    }
    for (int e = tid; e < TC * r; e += 256) {
        const int b = e / r, l = e % r;          // column b of the tile = lane b/4, slot b%4
        chpart[((size_t)part * ld + col0 + b) * r + l] = sHist[l][b & 3][b >> 2];
    }
}

// td_col[t] = sum over parts (fixed order); colhist likewise.  Also clears
// the rank counters of the column order (when rank != nullptr).
__global__ void k_td_finalize(const double *__restrict__ tdpart, const int *__restrict__ chpart,
                              int nparts, int ldpart, int n, int r, double *__restrict__ tdcol,
                              int *__restrict__ colhist, int *__restrict__ rank)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) s += tdpart[(size_t)p * ldpart + t];
    if (tdcol) tdcol[t] = s;
    if (colhist)
        for (int l = 0; l < r; ++l) {
            int h = 0;
            for (int p = 0; p < nparts; ++p) h += chpart[((size_t)p * ldpart + t) * r + l];
            colhist[(size_t)t * r + l] = h;
        }
    if (rank) rank[t] = 0;
}

// Column order of Algorithm 3: decreasing td_col, equal values keep the
// smaller j first.  rank_j = #{e : td_e > td_j} + #{e < j : td_e = td_j},
// counted over a 2-D grid (columns x key chunks held in shared memory) so
// the O(n^2) comparisons spread over every SM.  td_col >= 0, so its IEEE bit
// pattern orders like the value and compares as a 64-bit integer.
constexpr int RANK_CHUNK = 512;
__global__ void __launch_bounds__(256) k_rank(const double *__restrict__ tdcol, int n, int *__restrict__ rank)
{
    __shared__ unsigned long long sk[RANK_CHUNK];
    const int j = blockIdx.x * 256 + threadIdx.x;
    const int base = blockIdx.y * RANK_CHUNK;
    const int len = min(RANK_CHUNK, n - base);
    for (int e = threadIdx.x; e < len; e += 256) sk[e] = (unsigned long long)__double_as_longlong(tdcol[base + e]);
    __syncthreads();
    if (j >= n) return;
    const unsigned long long kj = (unsigned long long)__double_as_longlong(tdcol[j]);
    const int jl = j - base;   // chunk-local index of j (may be outside the chunk)
    int cnt = 0;
    for (int e = 0; e < len; ++e) {
        const unsigned long long x = sk[e];
        cnt += (x > kj) | ((x == kj) & (e < jl));
    }
    if (cnt) atomicAdd(&rank[j], cnt);
}

// order[rank_j] = j, and the current error f = sum_j td_col[j] (fixed order:
// strided per thread, then a fixed tree), written to the control block.
__global__ void __launch_bounds__(1024) k_scatter_f(const double *__restrict__ tdcol, const int *__restrict__ rank,
                                                    int n, int *__restrict__ order, stmf_ctl *ctl)
{
    __shared__ double red[1024];
    double s = 0.0;
    for (int j = threadIdx.x; j < n; j += 1024) {
        order[rank[j]] = j;
        s += tdcol[j];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 512; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && ctl) {
        ctl->f = red[0];
        ctl->dirty_k = -2;
        ctl->refreshes += 1;
    }
}

// f = sum_j td_col[j] with k_scatter_f's fixed order (strided per thread,
// then a fixed tree), written to *out: the error of stmf_selection_stats and
// of its allocation-free form, equal bit for bit to the factorization's.
__global__ void __launch_bounds__(1024) k_error_sum(const double *__restrict__ tdcol, int n, double *__restrict__ out)
{
    __shared__ double red[1024];
    double s = 0.0;
    for (int j = threadIdx.x; j < n; j += 1024) s += tdcol[j];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 512; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// RMSE-A / RMSE-P (Section "Evaluation metrics"): squared residuals of the
// approximation over the given entries and over the held-out entries with a
// known value (R not NaN).  P = max_l (U_sl + V_lt) and d = R - P in FP32, as
// in the factorization; d^2 and the sums in FP64.  Block b takes rows b,
// b + grid, ...; each thread's columns in order, then a fixed tree over the
// block: part[4 b + {0, 1, 2, 3}] = (sum_A, sum_P, |S_A|, |S_P|).
constexpr int RMSE_THREADS = 256;
__global__ void __launch_bounds__(RMSE_THREADS) k_rmse_part(int m, int n, int r, const float *__restrict__ R, int ldr,
                                                            const uint32_t *__restrict__ mask, int ldm,
                                                            const float *__restrict__ U, int ldu,
                                                            const float *__restrict__ V, int ldv,
                                                            double *__restrict__ part)
{
    __shared__ float su[STMF_MAX_RANK];
    __shared__ double red[4][RMSE_THREADS];
    const int tid = threadIdx.x;
    double sa = 0.0, sp = 0.0, na = 0.0, np = 0.0;
    for (int s = blockIdx.x; s < m; s += gridDim.x) {
        __syncthreads();
        if (tid < r) su[tid] = U[(size_t)s * ldu + tid];
        __syncthreads();
        for (int t = tid; t < n; t += RMSE_THREADS) {
            const float x = R[(size_t)s * ldr + t];
            const bool given = mask ? ((mask[(size_t)s * ldm + (t >> 5)] >> (t & 31)) & 1u) : true;
            if (!given && x != x) continue;
            float p = -INFINITY;
            for (int l = 0; l < r; ++l) p = fmaxf(p, su[l] + V[(size_t)l * ldv + t]);
            const double d = (double)(x - p);
            if (given) { sa += d * d; na += 1.0; }
            else { sp += d * d; np += 1.0; }
        }
    }
    red[0][tid] = sa; red[1][tid] = sp; red[2][tid] = na; red[3][tid] = np;
    __syncthreads();
    for (int o = RMSE_THREADS / 2; o; o >>= 1) {
        if (tid < o)
#pragma unroll
            for (int q = 0; q < 4; ++q) red[q][tid] += red[q][tid + o];
        __syncthreads();
    }
    if (tid < 4) part[4 * (size_t)blockIdx.x + tid] = red[tid][0];
}

// Sums the block partials in block order; out = (RMSE-A, RMSE-P, |S_A|, |S_P|).
__global__ void k_rmse_final(const double *__restrict__ part, int nb, double *__restrict__ out)
{
    if (threadIdx.x != 0) return;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = 0; b < nb; ++b)
        for (int q = 0; q < 4; ++q) a[q] += part[4 * (size_t)b + q];
    out[0] = a[2] > 0.0 ? sqrt(a[0] / a[2]) : (double)NAN;
    out[1] = a[3] > 0.0 ? sqrt(a[1] / a[3]) : (double)NAN;
    out[2] = a[2];
    out[3] = a[3];
}

// TD selection (Section "The ByRow strategy"): the key of column t for row
// i = ctl->i is its tropical distance td(i,t) = |R_it - P1_it| where R_it is
// given, else 0 (the window skips those columns).  Ranked like the column
// order: decreasing key, equal keys keep the smaller t first, so the given
// columns come out in the selection's order.
__global__ void k_row_keys(const float *__restrict__ R, const float *__restrict__ P1, int np, int n,
                           const stmf_ctl *__restrict__ ctl, double *__restrict__ key, int *__restrict__ rank)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const size_t e = (size_t)ctl->i * np + t;
    const float x = R[e];
    key[t] = x == x ? (double)fabsf(x - P1[e]) : 0.0;
    rank[t] = 0;
}

__global__ void k_row_scatter(const int *__restrict__ rank, int n, int *__restrict__ order)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) order[rank[t]] = t;
}

// TD_B selection (Section "The ByRow strategy"): i0 of every column t, the
// row of the largest td(s,t) over given s (the smaller s on ties).  A block
// covers 32 columns; its 32 warps stride over the rows, each warp reading 32
// consecutive columns of one row.
__global__ void __launch_bounds__(1024) k_col_tdmax(const float *__restrict__ R, const float *__restrict__ P1,
                                                    int np, int m, int n, int *__restrict__ colarg)
{
    __shared__ unsigned long long red[32][33];
    const int c = threadIdx.x & 31, q = threadIdx.x >> 5;
    const int t = blockIdx.x * 32 + c;
    unsigned long long best = 0ull;
    if (t < n)
        for (int s = q; s < m; s += 32) {
            const size_t e = (size_t)s * np + t;
            const float x = R[e];
            if (x == x) {
                const unsigned long long k = td_argmax_key(fabsf(x - P1[e]), s);
                best = k > best ? k : best;
            }
        }
    red[q][c] = best;
    __syncthreads();
    if (q == 0 && t < n) {
        for (int z = 1; z < 32; ++z) best = red[z][c] > best ? red[z][c] : best;
        colarg[t] = best ? td_argmax_index(best) : 0;   // every column has a given entry (checked at set-up)
    }
}

}  // namespace

cudaError_t launch_row_order(cudaStream_t st, stmf_problem *P)
{
    const int nb = (P->n + 255) / 256;
    k_row_keys<<<nb, 256, 0, st>>>(P->R, P->P1, P->np, P->n, P->ctl, P->rowkey, P->rowrank);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 grid((P->n + 255) / 256, (P->n + RANK_CHUNK - 1) / RANK_CHUNK);
    k_rank<<<grid, 256, 0, st>>>(P->rowkey, P->n, P->rowrank);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_row_scatter<<<nb, 256, 0, st>>>(P->rowrank, P->n, P->roworder);
    return cudaGetLastError();
}

cudaError_t launch_maxplus(cudaStream_t st, int m, int n, int r, const float *U, int ldu,
                           const float *V, int ldv, const uint32_t *mask, int ldm,
                           float *P1, int ldp, uint8_t *A, int lda, float *P2,
                           const float *R, int ldr, double *tdpart, int *colhist)
{
    dim3 grid((n + TC - 1) / TC, (m + TR * TILES - 1) / (TR * TILES));
    if (R)
        k_maxplus<true, true><<<grid, 256, 0, st>>>(m, n, r, U, ldu, V, ldv, mask, ldm, P1, ldp, A,
                                                    lda, P2, R, ldr, tdpart, colhist);
    else
        k_maxplus<false, true><<<grid, 256, 0, st>>>(m, n, r, U, ldu, V, ldv, mask, ldm, P1, ldp, A,
                                                     lda, P2, R, ldr, tdpart, colhist);
    return cudaGetLastError();
}

cudaError_t launch_planes(cudaStream_t st, stmf_problem *P, int *chpart)
{
    dim3 grid(P->np / TC, (P->m + TR * TILES - 1) / (TR * TILES));
    if (P->precision == 1) {
        const HalfPlanes H{P->Rh, P->P1h, P->P2h, &P->ctl->scr_mr, &P->ctl->scr_mp};
        k_maxplus_planes<true><<<grid, 256, 0, st>>>(P->m, P->n, P->r, P->U, P->V, P->np, P->P1, P->A, P->P2,
                                                     P->R, P->tdpart, chpart, H);
    } else {
        k_maxplus_planes<false><<<grid, 256, 0, st>>>(P->m, P->n, P->r, P->U, P->V, P->np, P->P1, P->A, P->P2,
                                                      P->R, P->tdpart, chpart, HalfPlanes{});
    }
    return cudaGetLastError();
}

int planes_nparts(int m) { return (m + TR * TILES - 1) / (TR * TILES); }

cudaError_t launch_td_finalize2(cudaStream_t st, const double *tdpart, const int *chpart, int nparts,
                                int ldpart, int n, int r, double *tdcol, int *colhist)
{
    k_td_finalize<<<(n + 255) / 256, 256, 0, st>>>(tdpart, chpart, nparts, ldpart, n, r, tdcol, colhist, nullptr);
    return cudaGetLastError();
}

int rmse_blocks(int m, int num_sms) { return m < 4 * num_sms ? m : 4 * num_sms; }

cudaError_t launch_rmse(cudaStream_t st, int num_sms, int m, int n, int r, const float *R, int ldr,
                        const uint32_t *mask, int ldm, const float *U, int ldu, const float *V, int ldv,
                        double *part, double *out)
{
    const int nb = rmse_blocks(m, num_sms);
    k_rmse_part<<<nb, RMSE_THREADS, 0, st>>>(m, n, r, R, ldr, mask, ldm, U, ldu, V, ldv, part);
    k_rmse_final<<<1, 32, 0, st>>>(part, nb, out);
    return cudaGetLastError();
}

cudaError_t launch_error_sum(cudaStream_t st, const double *tdcol, int n, double *out)
{
    k_error_sum<<<1, 1024, 0, st>>>(tdcol, n, out);
    return cudaGetLastError();
}

// Product planes, statistics, column order and error of a problem (and, for
// the TD_B selection, every column's i0).
cudaError_t launch_refresh_planes(cudaStream_t st, stmf_problem *P)
{
    cudaError_t e = launch_planes(st, P, P->chpart);
    if (e != cudaSuccess) return e;
    k_td_finalize<<<(P->n + 255) / 256, 256, 0, st>>>(P->tdpart, P->chpart, planes_nparts(P->m), P->np, P->n, P->r,
                                                      P->tdcol, P->colhist, P->rank);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dim3 grid((P->n + 255) / 256, (P->n + RANK_CHUNK - 1) / RANK_CHUNK);
    k_rank<<<grid, 256, 0, st>>>(P->tdcol, P->n, P->rank);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_scatter_f<<<1, 1024, 0, st>>>(P->tdcol, P->rank, P->n, P->order, P->ctl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (P->sel == STMF_SEL_TD_B) k_col_tdmax<<<(P->n + 31) / 32, 1024, 0, st>>>(P->R, P->P1, P->np, P->m, P->n, P->colarg);
    return cudaGetLastError();
}
