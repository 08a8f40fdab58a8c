// FP32 add+max issue-rate microbenchmark.  Every thread runs 8 independent
// dependency chains so the issue slots, not the latencies, bound the rate.
//   mode 0: FADD, FMNMX alternating (1:1, the mix of a max-plus inner loop)
//   mode 1: FADD only        mode 2: FMNMX only
//   mode 3: packed half2 HADD2 / HMNMX2 alternating (2 operations per lane)
//   mode 4: packed FP32x2 adds only (add.rn.f32x2: 2 operations per lane)
//   mode 5: one packed FP32x2 add then two scalar FMNMX (the add:max = 1:1
//           mix of a max-plus loop with its additions packed)
// Operations counted: one per FP32 lane operation (two per packed instruction).
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

}  // namespace

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
    default: k_peak_f32x2<1><<<blocks, 256, 0, st>>>(iters, b, c, sink); break;
    }
    return cudaGetLastError();
}
