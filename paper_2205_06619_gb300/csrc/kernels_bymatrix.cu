// The global order of the ByMatrix strategy (STMF_ByMatrix_NoPerm_TD_W;
// Section "The ByMatrix strategy" and its pseudocode in the Supplement).  At
// the start of every iteration each given element (i, j) gets
//   err(i,j) = td_row(i) + td_col(j) - td(i,j),   td = |R - P1| (FP32),
// with td_row and td_col summed in FP64 in index order, and err evaluated as
// (td_row + td_col) - td in FP64.  The elements are sorted by decreasing err,
// equal err keeping the smaller q = i*n + j first; the iteration's windows
// then walk that order.
//
// Sort: a bitonic network over the pairs (key, q) of the given elements,
// key = 0x7fff...f - the FP64 bits of err (err >= 0, so its bits order like
// its value, and a larger err gives a smaller key).  The pairs take slots in
// any order (atomic counter) and the rest up to a power of two holds
// UINT64_MAX keys.  The given pairs are unique, so the sorted sequence is the
// one total order, whatever the network and the slots.  Tiles of
// SORT_TILE pairs run their stages in shared memory; larger strides are
// global passes, one launch each.
#include "common.cuh"

namespace {

constexpr int SORT_TILE = 2048;
constexpr int SORT_THREADS = 1024;
constexpr unsigned long long KEY_NONE = ~0ull;

// td_row(s): sequential FP64 sum over t of the given |R_st - P1_st| (one
// thread per row, index order).
__global__ void k_td_rowsum_seq(const float *__restrict__ R, const float *__restrict__ P1, int ld, int m, int n,
                                double *__restrict__ tdr)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= m) return;
    const float *Rs = R + (size_t)s * ld, *Ps = P1 + (size_t)s * ld;
    double acc = 0.0;
    for (int t = 0; t < n; ++t) {
        const float x = Rs[t];
        if (x == x) acc += (double)fabsf(x - Ps[t]);
    }
    tdr[s] = acc;
}

// td_col(t): sequential FP64 sum over s (one thread per column, index order;
// the threads of a warp read consecutive columns of one row).
__global__ void k_td_colsum_seq(const float *__restrict__ R, const float *__restrict__ P1, int ld, int m, int n,
                                double *__restrict__ tdc)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double acc = 0.0;
    for (int s = 0; s < m; ++s) {
        const size_t e = (size_t)s * ld + t;
        const float x = R[e];
        if (x == x) acc += (double)fabsf(x - P1[e]);
    }
    tdc[t] = acc;
}

// Every slot empty (UINT64_MAX) and the slot counter at 0.
__global__ void k_clear_keys(size_t nsort, unsigned long long *__restrict__ key, unsigned long long *__restrict__ cnt)
{
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nsort) key[q] = KEY_NONE;
    if (q == 0) *cnt = 0ull;
}

// One pair per given element, in the next free slot (one atomic per warp).
__global__ void k_err_keys(const float *__restrict__ R, const float *__restrict__ P1, int ld, int m, int n,
                           const double *__restrict__ tdr, const double *__restrict__ tdc,
                           unsigned long long *__restrict__ key, unsigned *__restrict__ val,
                           unsigned long long *__restrict__ cnt)
{
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool given = false;
    unsigned long long k = KEY_NONE;
    if (q < (size_t)m * n) {
        const int i = (int)(q / n), j = (int)(q - (size_t)i * n);
        const size_t e = (size_t)i * ld + j;
        const float x = R[e];
        if (x == x) {
            const double err = (tdr[i] + tdc[j]) - (double)fabsf(x - P1[e]);
            k = 0x7fffffffffffffffull - (unsigned long long)__double_as_longlong(err);
            given = true;
        }
    }
    const unsigned b = __ballot_sync(0xffffffffu, given);
    if (!b) return;
    const int leader = __ffs(b) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(cnt, (unsigned long long)__popc(b));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (given) {
        const unsigned long long slot = base + __popc(b & ((1u << lane) - 1u));
        key[slot] = k;
        val[slot] = (unsigned)q;
    }
}

__device__ __forceinline__ bool pair_after(unsigned long long ka, unsigned va, unsigned long long kb, unsigned vb)
{
    return ka > kb || (ka == kb && va > vb);
}

// Compare-exchange of positions e < l of the bitonic network at stage k:
// ascending where the global index e has bit k clear, descending otherwise.
__device__ __forceinline__ void cmp_swap(unsigned long long &ke, unsigned &ve, unsigned long long &kl, unsigned &vl,
                                         bool up)
{
    if (pair_after(ke, ve, kl, vl) == up) {
        const unsigned long long tk = ke; ke = kl; kl = tk;
        const unsigned tv = ve; ve = vl; vl = tv;
    }
}

// Stages k = kmin..kmax (all strides j < SORT_TILE of each) on one tile in
// shared memory.  kmin = 2, kmax = SORT_TILE sorts the tile; kmin = kmax = K
// finishes stage K after its global passes.
__global__ void __launch_bounds__(SORT_THREADS) k_bitonic_tile(unsigned long long *__restrict__ key,
                                                              unsigned *__restrict__ val, size_t kmin, size_t kmax)
{
    __shared__ unsigned long long sk[SORT_TILE];
    __shared__ unsigned sv[SORT_TILE];
    const size_t base = (size_t)blockIdx.x * SORT_TILE;
    for (int e = threadIdx.x; e < SORT_TILE; e += SORT_THREADS) { sk[e] = key[base + e]; sv[e] = val[base + e]; }
    __syncthreads();
    for (size_t k = kmin; k <= kmax; k <<= 1) {
        const int j0 = (int)(k >> 1) < SORT_TILE / 2 ? (int)(k >> 1) : SORT_TILE / 2;
        for (int j = j0; j > 0; j >>= 1) {
            // thread x owns the pair (e, e + j), e = the x-th index with bit j clear
            const int x = threadIdx.x;
            const int e = ((x / j) * 2 * j) + (x % j), l = e + j;
            const bool up = ((base + e) & k) == 0;
            cmp_swap(sk[e], sv[e], sk[l], sv[l], up);
            __syncthreads();
        }
    }
    for (int e = threadIdx.x; e < SORT_TILE; e += SORT_THREADS) { key[base + e] = sk[e]; val[base + e] = sv[e]; }
}

// One global pass of stage k at stride j >= SORT_TILE: pair p of the
// nsort / 2 pairs is (e, e + j), e = the p-th index with bit j clear.
__global__ void k_bitonic_global(unsigned long long *__restrict__ key, unsigned *__restrict__ val, size_t nsort,
                                 size_t k, size_t j)
{
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nsort / 2) return;
    const size_t e = (p / j) * 2 * j + (p % j), l = e + j;
    unsigned long long ke = key[e], kl = key[l];
    unsigned ve = val[e], vl = val[l];
    const bool up = (e & k) == 0;
    if (pair_after(ke, ve, kl, vl) == up) {
        key[e] = kl; key[l] = ke;
        val[e] = vl; val[l] = ve;
    }
}

}  // namespace

// Padded length of the ByMatrix sort: the next power of two >= the number of
// given entries, at least one tile.
size_t matrix_sort_len(long long ngiven)
{
    size_t len = SORT_TILE;
    while (len < (size_t)ngiven) len <<= 1;
    return len;
}

// td sums, keys and the sort of one ByMatrix iteration (before its first
// window).  P->skey / P->sval hold the order afterwards: the first ngiven
// values are the given elements q in the method's order.
cudaError_t launch_matrix_order(cudaStream_t st, stmf_problem *P)
{
    k_td_rowsum_seq<<<(P->m + 127) / 128, 128, 0, st>>>(P->R, P->P1, P->np, P->m, P->n, P->tdr_seq);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_td_colsum_seq<<<(P->n + 127) / 128, 128, 0, st>>>(P->R, P->P1, P->np, P->m, P->n, P->tdc_seq);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t ns = P->nsort, cells = (size_t)P->m * P->n;
    k_clear_keys<<<(unsigned)((ns + 255) / 256), 256, 0, st>>>(ns, P->skey, P->scnt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_err_keys<<<(unsigned)((cells + 255) / 256), 256, 0, st>>>(P->R, P->P1, P->np, P->m, P->n, P->tdr_seq,
                                                                P->tdc_seq, P->skey, P->sval, P->scnt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const unsigned tiles = (unsigned)(ns / SORT_TILE);
    k_bitonic_tile<<<tiles, SORT_THREADS, 0, st>>>(P->skey, P->sval, 2, SORT_TILE);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (size_t k = 2 * (size_t)SORT_TILE; k <= ns; k <<= 1) {
        for (size_t j = k >> 1; j >= (size_t)SORT_TILE; j >>= 1) {
            k_bitonic_global<<<(unsigned)((ns / 2 + 255) / 256), 256, 0, st>>>(P->skey, P->sval, ns, k, j);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        k_bitonic_tile<<<tiles, SORT_THREADS, 0, st>>>(P->skey, P->sval, k, k);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

namespace {
__global__ void k_count_given(const float *__restrict__ R, int ld, int m, int n, unsigned long long *__restrict__ cnt)
{
    unsigned long long c = 0;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < (size_t)m * n;
         q += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(q / n), j = (int)(q - (size_t)i * n);
        const float x = R[(size_t)i * ld + j];
        c += x == x;
    }
    c = __reduce_add_sync(0xffffffffu, (unsigned)c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}
}  // namespace

// Number of given entries of the packed R (ByMatrix: the length of its order).
cudaError_t launch_count_given(cudaStream_t st, const stmf_problem *P, unsigned long long *d_cnt)
{
    k_count_given<<<4 * P->ctx->num_sms, 256, 0, st>>>(P->R, P->np, P->m, P->n, d_cnt);
    return cudaGetLastError();
}
