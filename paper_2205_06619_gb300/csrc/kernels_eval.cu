// Evaluation of a window of F-ULF / F-URF candidates (Algorithms 1 and 2),
// in two launches.
//
// Phase 1 (k_res) completes every candidate's factor pair:
//   F-ULF slot c:  U'_sc = min over given t of (R_st - V'_ct)   (row residuation)
//   F-URF slot c:  V'_ct = min over given s of (R_st - U'_sc)   (column residuation)
// where the other factor (V'_c for F-ULF, U'_c for F-URF) is the seed that
// k_seed wrote.  Phase 2 (k_delta) sums, for every candidate, the change of
// the b-norm terms over all entries
//   Delta_c = sum over given (s,t) of ( |R_st - max(E_st, U'_sc + V'_ct)| - |R_st - P1_st| ),
//   E = max over l != k of (U_sl + V_lt) = (A == k ? P2 : P1),
// per entry, so a candidate that changes nothing gives exactly 0.
#include "common.cuh"

namespace {

constexpr unsigned FULLM = 0xffffffffu;
constexpr int NCT = STMF_WMAX / 2;    // candidates of one type in a window

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Atomic minimum of a float slot that starts at +inf.  Non-negative floats
// order like their bit patterns as signed integers, negative ones in reverse
// as unsigned integers; -0 is first made +0 so that it orders as zero.
__device__ __forceinline__ void atomic_min_float(float *addr, float v)
{
    v = v + 0.0f;
    if (v >= 0.f) atomicMin(reinterpret_cast<int *>(addr), __float_as_int(v));
    else atomicMax(reinterpret_cast<unsigned *>(addr), __float_as_uint(v));
}

// ------------------------------------------------------------------ phase 1
// Task = (type, RES_THREADS x RES_RPT rows of X, a chunk of columns): type 0
// runs over the rows of R with the F-ULF candidates' V'_c, type 1 over the
// rows of R^T with the F-URF candidates' U'_c.  The candidates' values of the
// chunk are staged in shared memory and read as warp-wide broadcasts; each
// thread owns two rows (every broadcast feeds both) and keeps their running
// minima of all the type's candidates in registers (no cross-thread
// reduction).  The candidate loop is unrolled for a compile-time count
// NB >= cnt (4, 8, 16 or 32, picked per block) so the minima of different
// candidates interleave; the slots above cnt compute on whatever the staging
// area holds and are never stored.  Chunks combine through atomic minima,
// which are exact in any order.  NaN entries (not given, padding) drop out of
// fminf.
constexpr int RES_THREADS = 128;
constexpr int RES_CHUNK_MAX = 128;   // columns per task: a multiple of 8 up to this, chosen per launch
constexpr int RES_RPT = 2;           // rows per thread

__device__ __forceinline__ float min8(float4 a, float4 b, float4 w0, float4 w1)
{
    const float m0 = fminf(fminf(a.x - w0.x, a.y - w0.y), fminf(a.z - w0.z, a.w - w0.w));
    const float m1 = fminf(fminf(b.x - w1.x, b.y - w1.y), fminf(b.z - w1.z, b.w - w1.w));
    return fminf(m0, m1);
}

template <int NB>
__device__ __forceinline__ void res_rows(const float4 *x4a, const float4 *x4b, bool has_b,
                                         const float (*sW)[RES_CHUNK_MAX], int nq, const int *sslot, int cnt,
                                         float *OUT, size_t ldo, int row)
{
    float acc[NB], accb[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) { acc[c] = INFINITY; accb[c] = INFINITY; }
#pragma unroll 1
    for (int q = 0; q < nq; q += 2) {
        const float4 a = x4a[q], b = x4a[q + 1];
        const float4 a2 = x4b[q], b2 = x4b[q + 1];
#pragma unroll
        for (int c = 0; c < NB; ++c) {
            const float4 w0 = reinterpret_cast<const float4 *>(sW[c])[q];
            const float4 w1 = reinterpret_cast<const float4 *>(sW[c])[q + 1];
            acc[c] = fminf(acc[c], min8(a, b, w0, w1));
            accb[c] = fminf(accb[c], min8(a2, b2, w0, w1));
        }
    }
#pragma unroll
    for (int c = 0; c < NB; ++c) {
        if (c < cnt && acc[c] < INFINITY) atomic_min_float(OUT + sslot[c] * ldo + row, acc[c]);
        if (has_b && c < cnt && accb[c] < INFINITY) atomic_min_float(OUT + sslot[c] * ldo + row + RES_THREADS, accb[c]);
    }
}

__global__ void __launch_bounds__(RES_THREADS) k_res(stmf_problem P, int ntask0, int nch0, int nch1, int chunk)
{
    __shared__ __align__(16) float sW[NCT][RES_CHUNK_MAX];
    __shared__ int sslot[NCT];
    stmf_win *win = P.win;
    const int tid = threadIdx.x;
    // the window evaluation's span (this launch's start to the end of
    // phase 2) is recorded with the global nanosecond timer: inside a CUDA
    // graph no event can bracket single nodes
    if (tid == 0) atomicMin(&win->ev_t0, global_ns());
    int task = blockIdx.x;
    const int type = task >= ntask0;
    if (type) task -= ntask0;
    const int cnt = type ? win->nv : win->nu;
    if (cnt == 0) return;
    const int nch = type ? nch1 : nch0;
    const int rb = task / nch, c0 = (task % nch) * chunk;
    const float *X = type ? P.RT : P.R;
    const size_t ldx = type ? P.mp : P.np;
    const int nq = min(chunk, (int)ldx - c0) >> 2;      // float4 columns of this task (rows are padded to 256)
    const int nrows = type ? P.n : P.m;
    const float *W = type ? P.Uc : P.Vc;
    float *OUT = type ? P.Vc : P.Uc;
    const size_t ldw = type ? P.mp : P.np;
    const size_t ldo = type ? P.np : P.mp;

    if (tid < cnt) sslot[tid] = type ? win->vlist[tid] : win->ulist[tid];
    __syncthreads();
    for (int e = tid; e < cnt * nq; e += RES_THREADS) {
        const int c = e / nq, q = e % nq;
        reinterpret_cast<float4 *>(sW[c])[q] = reinterpret_cast<const float4 *>(W + sslot[c] * ldw + c0)[q];
    }
    __syncthreads();
    const int row = rb * RES_THREADS * RES_RPT + tid;
    if (row < nrows) {
        const bool has_b = row + RES_THREADS < nrows;
        const float4 *x4 = reinterpret_cast<const float4 *>(X + row * ldx + c0);
        const float4 *x4b = has_b ? reinterpret_cast<const float4 *>(X + (row + RES_THREADS) * ldx + c0) : x4;
        if (cnt <= 4) res_rows<4>(x4, x4b, has_b, sW, nq, sslot, cnt, OUT, ldo, row);
        else if (cnt <= 8) res_rows<8>(x4, x4b, has_b, sW, nq, sslot, cnt, OUT, ldo, row);
        else if (cnt <= 16) res_rows<16>(x4, x4b, has_b, sW, nq, sslot, cnt, OUT, ldo, row);
        else res_rows<32>(x4, x4b, has_b, sW, nq, sslot, cnt, OUT, ldo, row);
    }
    __syncthreads();
    if (tid == 0) atomicMax(&win->ev_r1, global_ns());
}

// ------------------------------------------------------------------ phase 2
// Tiles of 4 rows x DEL_COLS columns (a thread owns 4 rows x one float4
// column) cover the matrix and are dealt to the blocks round-robin, so every
// block's share is fixed and the sums are reproducible.  A thread keeps its
// tile of P1, P2 and A in registers and runs through all the window's
// candidates (grouped by k, so E is rebuilt only when k changes); V'_c is
// read from global memory two candidates ahead, U'_c of the tile's rows from
// shared memory.
constexpr int DEL_THREADS = 128;
constexpr int DEL_COLS = 4 * DEL_THREADS;
constexpr int DEL_BLOCKS_PER_SM = 5;
static_assert(DEL_BLOCKS_PER_SM <= STMF_DELTA_MAX_BLOCKS_PER_SM, "phase-2 partials buffer too small");

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }


// Change of the b-norm terms of a 4 x 4 tile for one candidate.  Every
// factorization the method holds satisfies U (x) V <= R on the given entries
// (Acol and both updates end with a residuation), and so does every
// candidate's U' (x) V'.  With P1 <= R and P' <= R the term
// |R - P'| - |R - P1| is P1 - P', P' = max(E, u_i + v_j): R is not needed.
// (FP32 rounding can put a value an ulp above R; the term then differs from
// the literal one by a few ulps, far inside the error tolerance.)  Entries
// not given hold P1 = P2 = STMF_SENTINEL, so P' = STMF_SENTINEL (every
// finite x is far below it) and the term is exactly 0,
// as it is for every entry a candidate leaves unchanged.  Packed FP32x2
// additions; the tile sum is a fixed tree of depth 4.
__device__ __forceinline__ float tile_change(const float (&p1)[4][4], const float (&E)[4][4], const float4 u,
                                             const float4 v)
{
    const float uu[4] = {u.x, u.y, u.z, u.w};
    const float2 v01 = f2(v.x, v.y), v23 = f2(v.z, v.w);
    float2 q[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 ui = f2(uu[i], uu[i]);
        const float2 x01 = __fadd2_rn(ui, v01), x23 = __fadd2_rn(ui, v23);
        const float2 n01 = f2(-fmaxf(E[i][0], x01.x), -fmaxf(E[i][1], x01.y));
        const float2 n23 = f2(-fmaxf(E[i][2], x23.x), -fmaxf(E[i][3], x23.y));
        const float2 d01 = __fadd2_rn(f2(p1[i][0], p1[i][1]), n01);
        const float2 d23 = __fadd2_rn(f2(p1[i][2], p1[i][3]), n23);
        q[i] = __fadd2_rn(d01, d23);
    }
    const float2 s = __fadd2_rn(__fadd2_rn(q[0], q[1]), __fadd2_rn(q[2], q[3]));
    return s.x + s.y;
}

__global__ void __launch_bounds__(DEL_THREADS, DEL_BLOCKS_PER_SM) k_delta(stmf_problem P, int ntiles, int nct)
{
    __shared__ float sacc[STMF_WMAX][DEL_THREADS];
    __shared__ __align__(16) float su[STMF_WMAX][4];
    __shared__ int sslot[STMF_WMAX], sk[STMF_WMAX];
    stmf_win *win = P.win;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) atomicMin(&win->ev_d0, global_ns());
    const int na = win->na;
    if (tid < na) {
        const int slot = win->alist[tid];
        sslot[tid] = slot;
        sk[tid] = P.cand[8 * slot + 1];
    }
    for (int c = 0; c < na; ++c) sacc[c][tid] = 0.f;
    const int nf4 = P.np >> 2;
    for (int tile = blockIdx.x; tile < ntiles && na > 0; tile += gridDim.x) {
        const int s0 = (tile / nct) * 4;
        const int f = (tile % nct) * DEL_THREADS + tid;
        __syncthreads();
        for (int e = tid; e < 4 * na; e += DEL_THREADS)
            su[e >> 2][e & 3] = P.Uc[(size_t)sslot[e >> 2] * P.mp + s0 + (e & 3)];
        __syncthreads();
        if (f >= nf4) continue;

        float p1[4][4], p2[4][4], E[4][4];
        uint32_t aw[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const size_t o4 = (size_t)(s0 + i) * nf4 + f;
            const float4 y = reinterpret_cast<const float4 *>(P.P1)[o4];
            const float4 z = reinterpret_cast<const float4 *>(P.P2)[o4];
            aw[i] = reinterpret_cast<const uint32_t *>(P.A)[o4];
            p1[i][0] = y.x; p1[i][1] = y.y; p1[i][2] = y.z; p1[i][3] = y.w;
            p2[i][0] = z.x; p2[i][1] = z.y; p2[i][2] = z.z; p2[i][3] = z.w;
        }
        const float4 *Vc4 = reinterpret_cast<const float4 *>(P.Vc) + f;
        const size_t ldv4 = (size_t)nf4;
        float4 vn0 = Vc4[sslot[0] * ldv4];
        float4 vn1 = na > 1 ? Vc4[sslot[1] * ldv4] : vn0;
        int kcur = -1;
#pragma unroll 1
        for (int c = 0; c < na; ++c) {
            const float4 v4 = vn0;
            vn0 = vn1;
            if (c + 2 < na) vn1 = Vc4[sslot[c + 2] * ldv4];
            const int k = sk[c];
            if (k != kcur) {
                kcur = k;
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj)
                        E[i][jj] = ((aw[i] >> (8 * jj)) & 0xffu) == (uint32_t)k ? p2[i][jj] : p1[i][jj];
            }
            const float4 u4 = *reinterpret_cast<const float4 *>(su[c]);
            sacc[c][tid] += tile_change(p1, E, u4, v4);
        }
    }
    __syncthreads();
    // block partial of every candidate, fixed order, float-float
    for (int c = warp; c < na; c += DEL_THREADS / 32) {
        stmf_ff x = {0.f, 0.f};
        for (int t = lane; t < DEL_THREADS; t += 32) x = ff_add(x, {sacc[c][t], 0.f});
#pragma unroll
        for (int o = 16; o; o >>= 1)
            x = ff_add(x, {__shfl_xor_sync(FULLM, x.hi, o), __shfl_xor_sync(FULLM, x.lo, o)});
        if (lane == 0) P.part[(size_t)sslot[c] * gridDim.x + blockIdx.x] = make_float2(x.hi, x.lo);
    }
    if (tid == 0) atomicMax(&win->ev_t1, global_ns());
}

// Phase 2 with tiles of 8 rows x DEL_COLS columns (a thread owns 8 rows x
// one float4 column): the per-candidate costs (the V' load, the U' loads,
// the accumulator update, the loop and the k test) spread over 32 entries
// instead of 16, and each V' load feeds twice the entries.  P1 and E stay in
// registers; P2 and A of the thread's entries go to its own slots of dynamic
// shared memory (never shared, so no barrier) and are read only when k
// changes.  Per entry the term is tile_change's P1 - max(E, x), formed as
// min(P1 - E, P1 - x): rounding is monotone, so fl(P1 - max(E, x)) =
// min(fl(P1 - E), fl(P1 - x)) bit for bit, and P1 - E (0 where A != k) is
// rebuilt per k-group in place of E; no negation is needed.  The tile sum is
// a fixed tree of depth 5.
constexpr int DEL8_ROWS = 8;
constexpr int DEL8_MAX_BLOCKS_PER_SM = 4;   // at 4 the kernel spills about 35 registers; at 3 it fits in 163
constexpr size_t DEL8_SMEM = (size_t)DEL8_ROWS * DEL_THREADS * (sizeof(float4) + sizeof(uint32_t));

__device__ __forceinline__ float tile_change8(const float (&p1)[8][4], const float (&B)[8][4], const float4 u0,
                                              const float4 u1, const float4 v)
{
    const float uu[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
    const float2 v01 = f2(v.x, v.y), v23 = f2(v.z, v.w);
    float2 q[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float2 ui = f2(uu[i], uu[i]);
        const float2 x01 = __fadd2_rn(ui, v01), x23 = __fadd2_rn(ui, v23);
        // P1 - x with one rounding: fma(-1, x, P1)
        const float2 y01 = __ffma2_rn(x01, f2(-1.f, -1.f), f2(p1[i][0], p1[i][1]));
        const float2 y23 = __ffma2_rn(x23, f2(-1.f, -1.f), f2(p1[i][2], p1[i][3]));
        const float2 d01 = f2(fminf(B[i][0], y01.x), fminf(B[i][1], y01.y));
        const float2 d23 = f2(fminf(B[i][2], y23.x), fminf(B[i][3], y23.y));
        q[i] = __fadd2_rn(d01, d23);
    }
    const float2 s = __fadd2_rn(__fadd2_rn(__fadd2_rn(q[0], q[1]), __fadd2_rn(q[2], q[3])),
                                __fadd2_rn(__fadd2_rn(q[4], q[5]), __fadd2_rn(q[6], q[7])));
    return s.x + s.y;
}

template <int MINB>
__global__ void __launch_bounds__(DEL_THREADS, MINB) k_delta8(stmf_problem P, int ntiles, int nct)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    float4 *sP2 = reinterpret_cast<float4 *>(dsm);                                   // [8][DEL_THREADS]
    uint32_t *sA = reinterpret_cast<uint32_t *>(dsm + sizeof(float4) * DEL8_ROWS * DEL_THREADS);   // [8][DEL_THREADS]
    __shared__ float sacc[STMF_WMAX][DEL_THREADS];
    __shared__ __align__(16) float su[STMF_WMAX][DEL8_ROWS];
    __shared__ int sslot[STMF_WMAX], sk[STMF_WMAX];
    stmf_win *win = P.win;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) atomicMin(&win->ev_d0, global_ns());
    const int na = win->na;
    if (tid < na) {
        const int slot = win->alist[tid];
        sslot[tid] = slot;
        sk[tid] = P.cand[8 * slot + 1];
    }
    for (int c = 0; c < na; ++c) sacc[c][tid] = 0.f;
    const int nf4 = P.np >> 2;
    for (int tile = blockIdx.x; tile < ntiles && na > 0; tile += gridDim.x) {
        const int s0 = (tile / nct) * DEL8_ROWS;
        const int f = (tile % nct) * DEL_THREADS + tid;
        __syncthreads();
        for (int e = tid; e < DEL8_ROWS * na; e += DEL_THREADS)
            su[e >> 3][e & 7] = P.Uc[(size_t)sslot[e >> 3] * P.mp + s0 + (e & 7)];
        __syncthreads();
        if (f >= nf4) continue;

        float p1[8][4], B[8][4];   // B = P1 - E of the current k (0 where A != k)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const size_t o4 = (size_t)(s0 + i) * nf4 + f;
            const float4 y = reinterpret_cast<const float4 *>(P.P1)[o4];
            sP2[i * DEL_THREADS + tid] = reinterpret_cast<const float4 *>(P.P2)[o4];
            sA[i * DEL_THREADS + tid] = reinterpret_cast<const uint32_t *>(P.A)[o4];
            p1[i][0] = y.x; p1[i][1] = y.y; p1[i][2] = y.z; p1[i][3] = y.w;
        }
        const float4 *Vc4 = reinterpret_cast<const float4 *>(P.Vc) + f;
        const size_t ldv4 = (size_t)nf4;
        float4 vn0 = Vc4[sslot[0] * ldv4];
        float4 vn1 = na > 1 ? Vc4[sslot[1] * ldv4] : vn0;
        int kcur = -1;
#pragma unroll 1
        for (int c = 0; c < na; ++c) {
            const float4 v4 = vn0;
            vn0 = vn1;
            if (c + 2 < na) vn1 = Vc4[sslot[c + 2] * ldv4];
            const int k = sk[c];
            if (k != kcur) {
                kcur = k;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float4 z = sP2[i * DEL_THREADS + tid];
                    const uint32_t a = sA[i * DEL_THREADS + tid];
                    const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj)
                        B[i][jj] = ((a >> (8 * jj)) & 0xffu) == (uint32_t)k ? p1[i][jj] - zz[jj] : 0.f;
                }
            }
            const float4 u0 = *reinterpret_cast<const float4 *>(&su[c][0]);
            const float4 u1 = *reinterpret_cast<const float4 *>(&su[c][4]);
            sacc[c][tid] += tile_change8(p1, B, u0, u1, v4);
        }
    }
    __syncthreads();
    // block partial of every candidate, fixed order, float-float
    for (int c = warp; c < na; c += DEL_THREADS / 32) {
        stmf_ff x = {0.f, 0.f};
        for (int t = lane; t < DEL_THREADS; t += 32) x = ff_add(x, {sacc[c][t], 0.f});
#pragma unroll
        for (int o = 16; o; o >>= 1)
            x = ff_add(x, {__shfl_xor_sync(FULLM, x.hi, o), __shfl_xor_sync(FULLM, x.lo, o)});
        if (lane == 0) P.part[(size_t)sslot[c] * gridDim.x + blockIdx.x] = make_float2(x.hi, x.lo);
    }
    if (tid == 0) atomicMax(&win->ev_t1, global_ns());
}

int res_blocks(int rows) { return (rows + RES_THREADS * RES_RPT - 1) / (RES_THREADS * RES_RPT); }

// Phase-1 tasks all have the same size, so a launch takes as many waves as
// the tasks need slots; the column chunk (a multiple of 8 up to 128) is the
// one that minimises waves x chunk.  Two slots are left to the decision
// block (1024 threads x 32 registers) that runs beside the evaluation, so
// that it never pushes a task into another wave.
int res_chunk_heuristic(const stmf_problem *P)
{
    static int per_sm = 0;
    if (!per_sm && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_res, RES_THREADS, 0) != cudaSuccess)
        per_sm = 1;
    long long slots = (long long)per_sm * P->ctx->num_sms - 2;
    if (slots < 1) slots = 1;
    int best = RES_CHUNK_MAX;
    long long best_cost = -1;
    for (int c = 32; c <= RES_CHUNK_MAX; c += 8) {
        const long long tasks = (long long)res_blocks(P->m) * ((P->n + c - 1) / c) +
                                (long long)res_blocks(P->n) * ((P->m + c - 1) / c);
        const long long cost = (tasks + slots - 1) / slots * c;
        if (best_cost < 0 || cost <= best_cost) { best_cost = cost; best = c; }
    }
    return best;
}

}  // namespace

int res_chunk(const stmf_problem *P)
{
    const int c = P->res_chunk_sel;
    return (c >= 32 && c <= RES_CHUNK_MAX && c % 8 == 0) ? c : res_chunk_heuristic(P);
}

// Phase 2's thread-tile height: 4 (k_delta) or 8 (k_delta8).  By default 8
// where the 8-row tiles still give every resident block (3 per SM) one,
// else 4: measured on the 1000 x 5000 workload, k_delta8 at 3 blocks per SM
// takes 69.3 us per 64-candidate window against 73.8 us for k_delta at 5 (at
// 4 blocks per SM it spills and takes 82.3 us).
int delta_rows(const stmf_problem *P)
{
    if (P->delta_rows_sel == 4 || P->delta_rows_sel == DEL8_ROWS) return P->delta_rows_sel;
    const long long t8 = (long long)((P->m + DEL8_ROWS - 1) / DEL8_ROWS) * ((P->np + DEL_COLS - 1) / DEL_COLS);
    return t8 >= 3LL * P->ctx->num_sms ? DEL8_ROWS : 4;
}

int delta_tiles(const stmf_problem *P)
{
    const int tr = delta_rows(P);
    return ((P->m + tr - 1) / tr) * ((P->np + DEL_COLS - 1) / DEL_COLS);
}

int delta_bps(const stmf_problem *P)
{
    const int cap = delta_rows(P) == DEL8_ROWS ? DEL8_MAX_BLOCKS_PER_SM : DEL_BLOCKS_PER_SM;
    const int def = delta_rows(P) == DEL8_ROWS ? 3 : DEL_BLOCKS_PER_SM;
    return (P->delta_bps_sel >= 1 && P->delta_bps_sel <= cap) ? P->delta_bps_sel : def;
}

int delta_grid(const stmf_problem *P)
{
    const int ntiles = delta_tiles(P);
    const int cap = delta_bps(P) * P->ctx->num_sms;
    return ntiles < cap ? ntiles : cap;
}

int delta_parts(const stmf_problem *P) { return delta_grid(P); }

bool delta_fills_gpu(const stmf_problem *P)
{
    const int ntiles = ((P->m + 3) / 4) * ((P->np + DEL_COLS - 1) / DEL_COLS);
    return ntiles >= DEL_BLOCKS_PER_SM * P->ctx->num_sms;
}

int delta_depth(const stmf_problem *P)
{
    const int ntiles = delta_tiles(P);
    const int g = delta_grid(P);
    // per term: the change, the tile tree (4 levels for 4 rows, 5 for 8),
    // the pair sum, and one addition per tile a block takes
    return (delta_rows(P) == DEL8_ROWS ? 6 : 5) + (ntiles + g - 1) / g;
}

// Set-up before any capture: the dynamic shared memory of the 8-row kernel.
cudaError_t delta_prepare()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_delta8<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DEL8_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_delta8<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DEL8_SMEM);
    if (e == cudaSuccess) done = true;
    return e;
}

cudaError_t launch_res(cudaStream_t st, stmf_problem *P)
{
    const int chunk = res_chunk(P);
    const int nch0 = (P->n + chunk - 1) / chunk, nch1 = (P->m + chunk - 1) / chunk;
    const int ntask0 = res_blocks(P->m) * nch0, ntask1 = res_blocks(P->n) * nch1;
    k_res<<<ntask0 + ntask1, RES_THREADS, 0, st>>>(*P, ntask0, nch0, nch1, chunk);
    return cudaGetLastError();
}

cudaError_t launch_delta(cudaStream_t st, stmf_problem *P)
{
    const int nct = (P->np + DEL_COLS - 1) / DEL_COLS;
    const int ntiles = delta_tiles(P), grid = delta_grid(P);
    if (delta_rows(P) == DEL8_ROWS) {
        if (delta_bps(P) >= 4) k_delta8<4><<<grid, DEL_THREADS, DEL8_SMEM, st>>>(*P, ntiles, nct);
        else k_delta8<3><<<grid, DEL_THREADS, DEL8_SMEM, st>>>(*P, ntiles, nct);
    } else {
        k_delta<<<grid, DEL_THREADS, 0, st>>>(*P, ntiles, nct);
    }
    return cudaGetLastError();
}
