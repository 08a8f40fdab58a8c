// FP32 add+max issue-rate microbenchmark.  Every thread runs 8 independent
// dependency chains so the issue slots, not the latencies, bound the rate.
//   mode 0: FADD, FMNMX alternating (1:1, the mix of a max-plus inner loop)
//   mode 1: FADD only        mode 2: FMNMX only
//   mode 3: packed half2 HADD2 / HMNMX2 alternating (2 operations per lane)
//   mode 4: packed FP32x2 adds only (add.rn.f32x2: 2 operations per lane)
//   mode 5: one packed FP32x2 add then two scalar FMNMX (the add:max = 1:1
//           mix of a max-plus loop with its additions packed)
//   mode 6: the instruction mix of the error-change pass (k_delta) per two
//           entries of a candidate: x = u + v (packed add), the two maxima
//           max(E, x) (FMNMX), the change P1 - max (packed sub) and its
//           accumulation (packed add)
//   mode 7: the instruction mix of the residuation pass (k_res) per two
//           entries of a candidate: two subtractions R - w (FADD) and one
//           three-input minimum that folds both into the running minimum
// Operations counted: modes 0-5, one per FP32 lane operation (two per packed
// instruction); modes 6 and 7, the algorithmic operations of the pass they
// mirror per entry and candidate (4 for mode 6: add, max, sub, accumulate;
// 2 for mode 7: sub, min), so that a kernel's achieved rate in those units
// divides by them directly.  Every chain is loop-carried, so no instruction
// can be hoisted out of the loop.
#include <cuda_fp16.h>

#include "common.cuh"

namespace {

template <int MODE>
__global__ void __launch_bounds__(256) k_peak(int iters, float b, float c, float *sink)
{
    float x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = (float)(threadIdx.x + q) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (MODE == 0) { x[q] = x[q] + b; x[q] = fmaxf(x[q], c); }
            if (MODE == 1) { x[q] = x[q] + b; x[q] = x[q] - c; }
            if (MODE == 2) { x[q] = fmaxf(x[q], b); x[q] = fminf(x[q], c); }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += x[q];
    if (s == 12345.678f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_half2(int iters, float b, float c, float *sink)
{
    __half2 x[8];
    const __half2 hb = __float2half2_rn(b), hc = __float2half2_rn(c);
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = __float2half2_rn((float)(threadIdx.x + q) * 1e-3f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            x[q] = __hadd2(x[q], hb);
            x[q] = __hmax2(x[q], hc);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += __low2float(x[q]) + __high2float(x[q]);
    if (s == 12345.678f) sink[threadIdx.x] = s;
}

template <int MIX>
__global__ void __launch_bounds__(256) k_peak_f32x2(int iters, float b, float c, float *sink)
{
    float2 x[8];
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = make_float2((float)(threadIdx.x + q) * 1e-3f, (float)q * 1e-3f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (MIX) {
                x[q] = __fadd2_rn(x[q], b2);
                x[q].x = fmaxf(x[q].x, c);
                x[q].y = fmaxf(x[q].y, c);
            } else {
                x[q] = __fadd2_rn(x[q], b2);
                x[q] = __fadd2_rn(x[q], c2);
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += x[q].x + x[q].y;
    if (s == 12345.678f) sink[threadIdx.x] = s;
}

// mode 6: 8 independent chains; each step is the per-pair sequence of the
// error-change pass, with the running sum fed back as the next step's u.
__global__ void __launch_bounds__(256) k_peak_delta(int iters, float e0, float *sink)
{
    unsigned long long acc[8], C, Pp;
    const float E0 = e0 + threadIdx.x * 1e-6f, E1 = e0 - 1e-3f;
    asm volatile("mov.b64 %0, {%1, %2};" : "=l"(C) : "f"(1e-7f), "f"(-1e-7f));
    asm volatile("mov.b64 %0, {%1, %2};" : "=l"(Pp) : "f"(2.0f), "f"(3.0f));
#pragma unroll
    for (int q = 0; q < 8; ++q)
        asm volatile("mov.b64 %0, {%1, %2};" : "=l"(acc[q]) : "f"(0.1f * q), "f"(-0.1f * q));
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            unsigned long long x, mp, d;
            float lo, hi;
            asm volatile("add.rn.f32x2 %0, %1, %2;" : "=l"(x) : "l"(acc[q]), "l"(C));
            asm volatile("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x));
            asm volatile("max.f32 %0, %1, %2;" : "=f"(lo) : "f"(lo), "f"(E0));
            asm volatile("max.f32 %0, %1, %2;" : "=f"(hi) : "f"(hi), "f"(E1));
            asm volatile("mov.b64 %0, {%1, %2};" : "=l"(mp) : "f"(lo), "f"(hi));
            asm volatile("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(Pp), "l"(mp));
            asm volatile("add.rn.f32x2 %0, %1, %2;" : "=l"(acc[q]) : "l"(acc[q]), "l"(d));
        }
    }
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        float a, b;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(acc[q]));
        t += a + b;
    }
    if (t == 12345.678f) sink[threadIdx.x] = t;
}

// mode 7: 8 independent running minima; each step subtracts two values from
// the running minimum and folds both back with one three-input minimum.
__global__ void __launch_bounds__(256) k_peak_res(int iters, float w0, float *sink)
{
    float acc[8];
    const float wa = w0 + threadIdx.x * 1e-9f, wb = w0 * 0.5f;
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 1e3f + q;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            float d0, d1;
            asm volatile("sub.f32 %0, %1, %2;" : "=f"(d0) : "f"(acc[q]), "f"(wa));
            asm volatile("sub.f32 %0, %1, %2;" : "=f"(d1) : "f"(acc[q]), "f"(wb));
            asm volatile("min.f32 %0, %1, %2, %3;" : "=f"(acc[q]) : "f"(acc[q]), "f"(d0), "f"(d1));
        }
    }
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += acc[q];
    if (t == 12345.678f) sink[threadIdx.x] = t;
}

}  // namespace

// Lane operations (modes 0-5) or algorithmic operations (modes 6, 7) that one
// launch of `blocks` x 256 threads performs.
double peak_ops(int mode, int iters, int blocks)
{
    const double th = (double)blocks * 256.0 * iters;
    if (mode == 6) return th * 8.0 * 2.0 * 4.0;    // 8 chains x 2 entries x 4 ops
    if (mode == 7) return th * 8.0 * 2.0 * 2.0;    // 8 chains x 2 entries x 2 ops
    return th * 8.0 * 2.0 * (mode >= 3 ? 2.0 : 1.0);
}

cudaError_t launch_peak(cudaStream_t st, int mode, int iters, int blocks, float *sink)
{
    // b, c chosen so the chains neither overflow nor become constant
    const float b = 1e-7f, c = -1e30f;
    switch (mode) {
    case 0: k_peak<0><<<blocks, 256, 0, st>>>(iters, b, c, sink); break;
    case 1: k_peak<1><<<blocks, 256, 0, st>>>(iters, b, b, sink); break;
    case 2: k_peak<2><<<blocks, 256, 0, st>>>(iters, -1e30f, 1e30f, sink); break;
    case 3: k_peak_half2<<<blocks, 256, 0, st>>>(iters, 1e-3f, -60000.f, sink); break;
    case 4: k_peak_f32x2<0><<<blocks, 256, 0, st>>>(iters, b, -b, sink); break;
    case 5: k_peak_f32x2<1><<<blocks, 256, 0, st>>>(iters, b, c, sink); break;
    case 6: k_peak_delta<<<blocks, 256, 0, st>>>(iters, 1.0f, sink); break;
    default: k_peak_res<<<blocks, 256, 0, st>>>(iters, 1e-30f, sink); break;
    }
    return cudaGetLastError();
}
