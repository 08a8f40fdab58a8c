// FP16 screening of a window's candidates (precision 1).
//
// After phase 1 has written every candidate's U'_.k and V'_k. (Uc, Vc), the
// screen evaluates each candidate's change of the b-norm error
//   Delta_c = sum over given (s,t) of ( |R_st - P'_st| - |R_st - P1_st| ),
//   P'_st = max(E_st, U'_sk + V'_kt),  E = (A == k ? P2 : P1)
// with packed half2 arithmetic on half copies of R, P1, P2, and proves some
// candidates non-improving: a candidate is dropped only when the half value
// exceeds a rigorous bound on the difference between it and the value the
// FP32 evaluation would compute, so the FP32 evaluation of every dropped
// candidate is >= 0 and the first-improving choice (and the best-of-window
// choice) over the kept candidates is the FP32 path's choice.
//
// Why the bound holds (u_h = 2^-11 and u = 2^-24 the unit roundoffs, M the
// candidate's magnitude bound max|R| + max(max|P1|,|P2|, max|U'| + max|V'|)):
//  * x = fl32(U'_sk + V'_kt) is computed exactly as the FP32 path does and
//    rounded to nearest half.  Rounding to nearest is monotone, so
//    max(rn(E), rn(x)) = rn(max(E, x)) = rn(P'): the half P' is the rounded
//    FP32 P', and an entry the candidate leaves unchanged (P' = P1) gives
//    exactly 0 in both precisions.
//  * A term can be non-zero (in either precision) only at a given entry with
//    A = k or rn(x) >= rn(E); the screen counts these entries, |S|.
//  * Per entry of S: half term error <= 6.01 u_h M + 2^-22, the depth-3 half
//    sum of 8 rows adds <= 6.05 u_h M, the FP32 accumulation of the screen
//    <= 2.03 D_s u M and the FP32 path's own term and sum errors
//    <= (4.02 + 2.03 D_32) u M (D = the number of FP32 additions a term
//    passes through).  The FP32 path forms its terms as P1 - P' (exact
//    when P1, P' <= R, which residuation keeps up to rounding): a value at
//    most 3 u M above R moves a term by at most 12 u M more.
//  * Drop iff Delta_half > 1.01 |S| W, W the per-entry sum of the above; no
//    dropping at all when M > 16384 (half overflow).  The block and grid sums
//    of both paths are float-float (relative error below 2^-44 over their
//    depth), far inside the 1% margin.
#include <cuda_fp16.h>

#include "common.cuh"

namespace {

constexpr unsigned FULLM = 0xffffffffu;
constexpr unsigned QNAN2 = 0x7e007e00u;
constexpr int VB = 8;          // candidates whose V' pairs are loaded together

__device__ __forceinline__ __half2 as_h2(unsigned u)
{
    __half2 h;
    *reinterpret_cast<unsigned *>(&h) = u;
    return h;
}

__device__ __forceinline__ unsigned as_u(__half2 h) { return *reinterpret_cast<unsigned *>(&h); }

// half2 mask of the halves of a pair whose byte of A equals k
__device__ __forceinline__ unsigned pair_mask(unsigned a16, int k)
{
    return ((a16 & 0xffu) == (unsigned)k ? 0x0000ffffu : 0u) | ((a16 >> 8) == (unsigned)k ? 0xffff0000u : 0u);
}

// half2 mask of the given (not NaN) halves
__device__ __forceinline__ unsigned given_mask(unsigned r2)
{
    return ((r2 & 0x7fffu) <= 0x7c00u ? 0x0000ffffu : 0u) | (((r2 >> 16) & 0x7fffu) <= 0x7c00u ? 0xffff0000u : 0u);
}

// Grid: the first `wmax` blocks compute max |U'| over s < m and max |V'| over
// t < n of one candidate slot each; the others own SCR_ROWS rows x all
// columns (thread = column pair) and accumulate every candidate's half change
// and the count |S| per thread in shared memory.
__global__ void __launch_bounds__(SCR_THREADS) k_screen(stmf_problem P, int wmax, int nblk)
{
    extern __shared__ float2 sacc[];                 // [candidate][SCR_THREADS]: (change, count)
    __shared__ float su[STMF_WMAX][SCR_ROWS];
    __shared__ int sslot[STMF_WMAX], sk[STMF_WMAX];
    __shared__ float red[2][SCR_THREADS / 32];
    const stmf_win *win = P.win;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nu = win->nu, nv = win->nv, nc = win->nc;

    if ((int)blockIdx.x < wmax) {
        const int c = blockIdx.x;
        if (c >= nc) return;
        float um = 0.f, vm = 0.f;
        for (int s = tid; s < P.m; s += SCR_THREADS) um = fmaxf(um, fabsf(P.Uc[(size_t)c * P.mp + s]));
        for (int t = tid; t < P.n; t += SCR_THREADS) vm = fmaxf(vm, fabsf(P.Vc[(size_t)c * P.np + t]));
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            um = fmaxf(um, __shfl_xor_sync(FULLM, um, o));
            vm = fmaxf(vm, __shfl_xor_sync(FULLM, vm, o));
        }
        if (lane == 0) { red[0][warp] = um; red[1][warp] = vm; }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < SCR_THREADS / 32; ++w) { um = fmaxf(um, red[0][w]); vm = fmaxf(vm, red[1][w]); }
            P.scr_umax[c] = um;
            P.scr_vmax[c] = vm;
        }
        return;
    }

    const int b = blockIdx.x - wmax;
    const int s0 = b * SCR_ROWS;
    const int rows = min(SCR_ROWS, P.m - s0);
    // F-ULF candidates then F-URF candidates, each list grouped by k
    if (tid < nu + nv) {
        const int slot = tid < nu ? win->ulist[tid] : win->vlist[tid - nu];
        sslot[tid] = slot;
        sk[tid] = P.cand[8 * slot + 1];
    }
    __syncthreads();
    const int ncl = nu + nv;
    for (int e = tid; e < ncl * SCR_ROWS; e += SCR_THREADS) {
        const int c = e / SCR_ROWS, i = e % SCR_ROWS;
        su[c][i] = i < rows ? P.Uc[(size_t)sslot[c] * P.mp + s0 + i] : 0.f;
    }
    for (int c = 0; c < ncl; ++c) sacc[c * SCR_THREADS + tid] = make_float2(0.f, 0.f);
    __syncthreads();

    const int npair = P.np >> 1;
    const __half2 zero2 = __float2half2_rn(0.f);
    for (int p = tid; p < npair; p += SCR_THREADS) {
        // the pair's R, P1, P2, A of the block's rows stay in registers; E
        // and the A = k indicator are rebuilt from them when k changes
        __half2 r2[SCR_ROWS], t02[SCR_ROWS], e2[SCR_ROWS], k2[SCR_ROWS];
        unsigned p1[SCR_ROWS], p2[SCR_ROWS], a16[SCR_ROWS];
#pragma unroll
        for (int i = 0; i < SCR_ROWS; ++i) {
            if (i < rows) {
                const size_t off = (size_t)(s0 + i) * P.np + 2 * p;
                r2[i] = *reinterpret_cast<const __half2 *>(P.Rh + off);
                p1[i] = *reinterpret_cast<const unsigned *>(P.P1h + off);
                p2[i] = *reinterpret_cast<const unsigned *>(P.P2h + off);
                a16[i] = *reinterpret_cast<const unsigned short *>(P.A + off);
            } else {
                r2[i] = as_h2(QNAN2);
                p1[i] = p2[i] = QNAN2;
                a16[i] = 0xffffu;
            }
            t02[i] = __hmax2(__habs2(__hsub2(r2[i], as_h2(p1[i]))), zero2);
            e2[i] = as_h2(QNAN2);
            k2[i] = zero2;
        }
        int kcur = -1;
        // candidates in groups of VB: the group's V' pairs are loaded together
        for (int c0 = 0; c0 < ncl; c0 += VB) {
            float2 vb[VB];
#pragma unroll
            for (int g = 0; g < VB; ++g)
                vb[g] = c0 + g < ncl ? *reinterpret_cast<const float2 *>(P.Vc + (size_t)sslot[c0 + g] * P.np + 2 * p)
                                     : make_float2(0.f, 0.f);
#pragma unroll
            for (int g = 0; g < VB; ++g) {
                const int c = c0 + g;
                if (c >= ncl) break;
                const int k = sk[c];
                if (k != kcur) {
                    kcur = k;
#pragma unroll
                    for (int i = 0; i < SCR_ROWS; ++i) {
                        const unsigned mk = pair_mask(a16[i], k);
                        e2[i] = as_h2((p2[i] & mk) | (p1[i] & ~mk));
                        k2[i] = as_h2(mk & given_mask(as_u(r2[i])) & 0x3c003c00u);   // 1.0 where A = k, given
                    }
                }
                const float2 v = vb[g];
                __half2 d[SCR_ROWS], q[SCR_ROWS];
#pragma unroll
                for (int i = 0; i < SCR_ROWS; ++i) {
                    const float u = su[c][i];
                    const __half2 x = __floats2half2_rn(u + v.x, u + v.y);
                    const __half2 pp = __hmax2(e2[i], x);
                    d[i] = __hsub2(__hmax2(__habs2(__hsub2(r2[i], pp)), zero2), t02[i]);
                    q[i] = __hmax2(__hge2(x, e2[i]), k2[i]);
                }
#pragma unroll
                for (int w = SCR_ROWS / 2; w; w >>= 1)
#pragma unroll
                    for (int i = 0; i < w; ++i) { d[i] = __hadd2(d[i], d[i + w]); q[i] = __hadd2(q[i], q[i + w]); }
                const float2 fd = __half22float2(d[0]), fq = __half22float2(q[0]);
                float2 a = sacc[c * SCR_THREADS + tid];
                a.x += fd.x + fd.y;
                a.y += fq.x + fq.y;
                sacc[c * SCR_THREADS + tid] = a;
            }
        }
    }
    __syncthreads();
    for (int c = warp; c < ncl; c += SCR_THREADS / 32) {
        stmf_ff x = {0.f, 0.f}, y = {0.f, 0.f};
        for (int t = lane; t < SCR_THREADS; t += 32) {
            const float2 a = sacc[c * SCR_THREADS + t];
            x = ff_add(x, {a.x, 0.f});
            y = ff_add(y, {a.y, 0.f});
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            x = ff_add(x, {__shfl_xor_sync(FULLM, x.hi, o), __shfl_xor_sync(FULLM, x.lo, o)});
            y = ff_add(y, {__shfl_xor_sync(FULLM, y.hi, o), __shfl_xor_sync(FULLM, y.lo, o)});
        }
        if (lane == 0) {
            P.scr_sum[(size_t)sslot[c] * nblk + b] = make_float2(x.hi, x.lo);
            P.scr_cnt[(size_t)sslot[c] * nblk + b] = make_float2(y.hi, y.lo);
        }
    }
}

// Sums the blocks' values of every candidate (fixed order), drops the
// candidates the bound proves non-improving, keeps the others in the
// evaluation lists in their order, and re-opens the evaluation queue.
__global__ void __launch_bounds__(1024) k_screen_select(stmf_problem P, int nblk, double depth)
{
    __shared__ double sd[STMF_WMAX], sn[STMF_WMAX];
    const stmf_ctl *ctl = P.ctl;
    stmf_win *win = P.win;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nc = win->nc;
    for (int c = warp; c < nc; c += 32) {
        stmf_ff x = {0.f, 0.f}, y = {0.f, 0.f};
        for (int b = lane; b < nblk; b += 32) {
            const float2 p = P.scr_sum[(size_t)c * nblk + b], q = P.scr_cnt[(size_t)c * nblk + b];
            x = ff_add(x, {p.x, p.y});
            y = ff_add(y, {q.x, q.y});
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            x = ff_add(x, {__shfl_xor_sync(FULLM, x.hi, o), __shfl_xor_sync(FULLM, x.lo, o)});
            y = ff_add(y, {__shfl_xor_sync(FULLM, y.hi, o), __shfl_xor_sync(FULLM, y.lo, o)});
        }
        if (lane == 0) {
            sd[c] = (double)x.hi + (double)x.lo;
            sn[c] = (double)y.hi + (double)y.lo;
        }
    }
    __syncthreads();
    if (tid != 0) return;
    const double uh = 1.0 / 2048.0, u32 = 1.0 / 16777216.0;
    const double coef = (6.01 + 6.05) * uh + (4.02 + 12.0 + 2.03 * depth) * u32;
    const double mr = (double)__uint_as_float(ctl->scr_mr), mp = (double)__uint_as_float(ctl->scr_mp);
    int dropped = 0;
    for (int c = 0; c < nc; ++c) {
        const double M = mr + fmax(mp, (double)P.scr_umax[c] + (double)P.scr_vmax[c]);
        int drop = 0;
        if (M <= 16384.0) {
            const double W = M * coef + 1.0 / 4194304.0;
            drop = sd[c] > 1.01 * sn[c] * W;     // false for a NaN sum
        }
        P.cand[8 * c + 4] = drop;
        dropped += drop;
    }
    int nu2 = 0, nv2 = 0;
    for (int a = 0; a < win->nu; ++a) {
        const int slot = win->ulist[a];
        if (!P.cand[8 * slot + 4]) win->ulist[nu2++] = slot;
    }
    for (int a = 0; a < win->nv; ++a) {
        const int slot = win->vlist[a];
        if (!P.cand[8 * slot + 4]) win->vlist[nv2++] = slot;
    }
    int na2 = 0;
    for (int a = 0; a < win->na; ++a) {
        const int slot = win->alist[a];
        if (!P.cand[8 * slot + 4]) win->alist[na2++] = slot;
    }
    win->na = na2;
    win->nu = nu2;
    win->nv = nv2;
    win->screened = dropped;
}

size_t screen_smem(int wmax) { return sizeof(float2) * (size_t)wmax * SCR_THREADS; }

}  // namespace

// Host set-up of a problem's screen (before any capture): shared-memory
// limit of the screen kernel.
cudaError_t screen_prepare(stmf_problem *P)
{
    P->scr_blocks = (P->m + SCR_ROWS - 1) / SCR_ROWS;
    return cudaFuncSetAttribute(k_screen, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)screen_smem(STMF_WMAX));
}

cudaError_t launch_screen(cudaStream_t st, stmf_problem *P)
{
    const int wmax = P->ctl_host->wmax;
    const int nblk = P->scr_blocks;
    k_screen<<<wmax + nblk, SCR_THREADS, screen_smem(wmax), st>>>(*P, wmax, nblk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // FP32 additions a term passes through: the screen's per-thread sums
    // (one per column-pair step, plus the pair sum) and the FP32 path's
    // (tile tree plus one per tile of a phase-2 block)
    const double ds = 2.0 + (P->np / 2 + SCR_THREADS - 1) / SCR_THREADS;
    const double d32 = 1.0 + delta_depth(P);
    k_screen_select<<<1, 1024, 0, st>>>(*P, nblk, ds + d32);
    return cudaGetLastError();
}
