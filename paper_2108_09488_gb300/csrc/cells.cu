// cells.cu -- cell-linked list on the GPU: cell keys, stable LSD radix sort by key, sorted
// particle copy and the cell start table.
//
// The neighbour sum of Eq. 4 (Sec. 2.2) runs over particles inside the kernel support; the
// cell list restricts the candidates to the cells around each particle.  Keys are computed from
// fixed-point positions with integer arithmetic only, cell = (xq * nc) >> 32 per axis and
// key = (cz * ncy + cy) * ncx + cx, and the sort is stable with the caller's order as the input
// order, so the permutation is (key, caller index)-ordered and identical on every run.
//
// Sort pass structure (digit-major histogram layout hist[digit * nblocks + block]):
//   hist   -- per-block digit histogram (pass 0 also computes the keys)
//   scan   -- exclusive scan of the whole histogram, one block
//   scatter-- per-block stable ranking with warp match, then scatter to the global slot
// HBM traffic per pass and particle: read key + index (8 B), write key + index (8 B), re-read the
// keys for the histogram (4 B).
#include "ade_internal.h"

namespace ade {

namespace {

__device__ __forceinline__ uint32_t cell_key(const uint32_t *__restrict__ xq, int n, int i,
                                             int dim, int ncx, int ncy, int ncz)
{
    uint32_t cx = __umulhi(__ldg(xq + i), (uint32_t)ncx);
    uint32_t cy = __umulhi(__ldg(xq + n + i), (uint32_t)ncy);
    uint32_t cz = dim == 3 ? __umulhi(__ldg(xq + 2 * (size_t)n + i), (uint32_t)ncz) : 0u;
    return (cz * (uint32_t)ncy + cy) * (uint32_t)ncx + cx;
}

// Pass 0: compute keys (and the identity index) and the block histogram of the first digit.
__global__ __launch_bounds__(kSortThreads) void k_hash_hist(const uint32_t *__restrict__ xq, int n,
                                                            int dim, int ncx, int ncy, int ncz,
                                                            uint32_t *__restrict__ keys,
                                                            uint32_t *__restrict__ idx,
                                                            uint32_t *__restrict__ hist,
                                                            int nblocks, int bits)
{
    __shared__ uint32_t sh[256];
    const int radix = 1 << bits;
    const uint32_t mask = (uint32_t)radix - 1u;
    for (int t = threadIdx.x; t < radix; t += blockDim.x) sh[t] = 0u;
    __syncthreads();
    const int base = blockIdx.x * kSortTile;
    for (int k = 0; k < kSortItems; ++k) {
        int i = base + k * kSortThreads + threadIdx.x;
        if (i < n) {
            uint32_t key = cell_key(xq, n, i, dim, ncx, ncy, ncz);
            keys[i] = key;
            idx[i] = (uint32_t)i;
            atomicAdd(&sh[key & mask], 1u);
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < radix; t += blockDim.x) hist[(size_t)t * nblocks + blockIdx.x] = sh[t];
}

__global__ __launch_bounds__(kSortThreads) void k_hist(const uint32_t *__restrict__ keys, int n,
                                                       int shift, int bits,
                                                       uint32_t *__restrict__ hist, int nblocks)
{
    __shared__ uint32_t sh[256];
    const int radix = 1 << bits;
    const uint32_t mask = (uint32_t)radix - 1u;
    for (int t = threadIdx.x; t < radix; t += blockDim.x) sh[t] = 0u;
    __syncthreads();
    const int base = blockIdx.x * kSortTile;
    for (int k = 0; k < kSortItems; ++k) {
        int i = base + k * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&sh[(__ldg(keys + i) >> shift) & mask], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < radix; t += blockDim.x) hist[(size_t)t * nblocks + blockIdx.x] = sh[t];
}

// Exclusive scan of hist[0..total) in place, one block of 1024 threads.
constexpr int kScanThreads = 1024;
__global__ __launch_bounds__(kScanThreads) void k_scan(uint32_t *__restrict__ hist, int total)
{
    __shared__ uint32_t warp_sums[32];
    const int chunk = (total + kScanThreads - 1) / kScanThreads;
    const int lo = threadIdx.x * chunk;
    const int hi = min(lo + chunk, total);
    uint32_t s = 0u;
    for (int i = lo; i < hi; ++i) s += hist[i];
    // block-wide exclusive scan of s
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint32_t v = warp_sums[lane];
        uint32_t vi = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) vi += y;
        }
        warp_sums[lane] = vi - v;
    }
    __syncthreads();
    uint32_t run = warp_sums[wid] + incl - s;
    for (int i = lo; i < hi; ++i) {
        uint32_t c = hist[i];
        hist[i] = run;
        run += c;
    }
}

// Stable scatter of one digit.  Warp w of a block owns tile elements
// [w*32*kSortItems, (w+1)*32*kSortItems); round j handles element w*32*kSortItems + 32 j + lane,
// so (warp, round, lane) order equals element order and the ranks below are stable.
__global__ __launch_bounds__(kSortThreads) void k_scatter(const uint32_t *__restrict__ keys_in,
                                                          const uint32_t *__restrict__ idx_in,
                                                          uint32_t *__restrict__ keys_out,
                                                          uint32_t *__restrict__ idx_out, int n,
                                                          int shift, int bits,
                                                          const uint32_t *__restrict__ hist,
                                                          int nblocks)
{
    constexpr int kWarps = kSortThreads / 32;
    __shared__ uint32_t wcnt[kWarps][256];
    const int radix = 1 << bits;
    const uint32_t mask = (uint32_t)radix - 1u;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < kWarps * 256; t += blockDim.x) (&wcnt[0][0])[t] = 0u;
    __syncthreads();

    const uint32_t lt_mask = (1u << lane) - 1u;
    const int base = blockIdx.x * kSortTile + wid * 32 * kSortItems;
    uint32_t key[kSortItems], rank[kSortItems];
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        int i = base + 32 * j + lane;
        bool valid = i < n;
        uint32_t k = valid ? __ldg(keys_in + i) : 0u;
        uint32_t d = valid ? ((k >> shift) & mask) : 0xffffffffu;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = __popc(peers & lt_mask);
        uint32_t cnt = valid ? wcnt[wid][d] : 0u;
        __syncwarp();
        if (valid && before == 0u) wcnt[wid][d] = cnt + __popc(peers);
        __syncwarp();
        key[j] = k;
        rank[j] = cnt + before;
    }
    __syncthreads();
    // exclusive prefix over warps, per digit
    for (int t = threadIdx.x; t < radix; t += blockDim.x) {
        uint32_t run = 0u;
        for (int w = 0; w < kWarps; ++w) {
            uint32_t c = wcnt[w][t];
            wcnt[w][t] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        int i = base + 32 * j + lane;
        if (i < n) {
            uint32_t d = (key[j] >> shift) & mask;
            uint32_t pos = __ldg(hist + (size_t)d * nblocks + blockIdx.x) + wcnt[wid][d] + rank[j];
            if (pos < (uint32_t)n) {  // always true for a consistent histogram; guards the write
                keys_out[pos] = key[j];
                idx_out[pos] = __ldg(idx_in + i);
            }
        }
    }
}

// Sorted particle copy P[k] = {x, y, z, C} of caller particle perm[k], and the cell start table:
// cell_start[c] = number of particles with key < c, for c = 0..ncells.
__global__ void k_reorder_cells(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ perm,
                                const uint32_t *__restrict__ xq, const float *__restrict__ C, int n,
                                int dim, int ncells, uint32_t *__restrict__ cell_start,
                                uint4 *__restrict__ P)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    long long cur = (i < n) ? (long long)__ldg(keys + i) : (long long)ncells;
    long long prev = (i > 0) ? (long long)__ldg(keys + i - 1) : -1ll;
    for (long long c = prev + 1; c <= cur; ++c) cell_start[c] = (uint32_t)i;
    if (i < n) {
        uint32_t a = __ldg(perm + i);
        uint4 p;
        p.x = __ldg(xq + a);
        p.y = __ldg(xq + n + a);
        p.z = dim == 3 ? __ldg(xq + 2 * (size_t)n + a) : 0u;
        p.w = __float_as_uint(__ldg(C + a));
        P[i] = p;
    }
}

}  // namespace

cudaError_t launch_build_cells(int dim, const uint32_t *xq, const float *C, int n, const int *nc,
                               int ncells, int passes, int digit_bits, const Work &w,
                               int sort_blocks, int *final_buf, cudaStream_t s)
{
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        int shift = p * digit_bits;
        int bits = digit_bits;
        if (p == 0) {
            k_hash_hist<<<sort_blocks, kSortThreads, 0, s>>>(xq, n, dim, nc[0], nc[1], nc[2], w.keys[0],
                                                             w.idx[0], w.hist, sort_blocks, bits);
        } else {
            k_hist<<<sort_blocks, kSortThreads, 0, s>>>(w.keys[cur], n, shift, bits, w.hist, sort_blocks);
        }
        k_scan<<<1, kScanThreads, 0, s>>>(w.hist, (1 << bits) * sort_blocks);
        k_scatter<<<sort_blocks, kSortThreads, 0, s>>>(w.keys[cur], w.idx[cur], w.keys[cur ^ 1],
                                                       w.idx[cur ^ 1], n, shift, bits, w.hist, sort_blocks);
        cur ^= 1;
    }
    int threads = 256;
    int blocks = (n + 1 + threads - 1) / threads;
    k_reorder_cells<<<blocks, threads, 0, s>>>(w.keys[cur], w.idx[cur], xq, C, n, dim, ncells,
                                               w.cell_start, w.P0);
    *final_buf = cur;
    return cudaGetLastError();
}

}  // namespace ade
