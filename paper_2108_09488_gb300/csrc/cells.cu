// cells.cu -- cell-linked list on the GPU: cell keys, a one-digit radix (counting) sort by key,
// the cell start table and the cell-sorted particle copy.
//
// The neighbour sum of Eq. 4 (Sec. 2.2) runs over particles inside the kernel support; the cell
// list restricts the candidates to the cells around each particle.  Keys come from fixed-point
// positions with integer arithmetic only: cell = (xq * nc) >> 32 per axis and
// key = (cz * ncy + cy) * ncx + cx.  The sort uses the whole key as one digit (radix = number of
// cells), which is cheaper than several 8-bit passes because the key space is about the size of
// the particle set:
//   k_count   key of every particle; atomic count per cell (the returned slot is a provisional
//             rank of the particle inside its cell)
//   scan      exclusive scan of the counts -> cell_start[0..ncells]: one launch over tiles of 4096
//             cells whose totals k_count accumulated (two or three launches without them)
//   k_place   provisional position cell_start[key] + rank
//   k_order   one thread per cell sorts its segment by caller index (insertion sort; cells hold a
//             handful of particles) and writes the sorted copy {x, y, z, C}; cells of more than
//             kSmallCell particles (wide kernels: hundreds to thousands per cell) are ordered by
//             the whole warp instead, each element placed at its rank among the cell's indices;
//             grids averaging 16 or more particles per cell use k_order_block (one block per cell,
//             the same ranking spread over 256 threads)
//             and, for the trimmed interaction walks, reduces the bounding box of every pencil
//             (the cells of one (cy, cz) row along x) over the transverse positions of its
//             particles, as fractions of a cell (FP32, so a walk bounds its distance to the row
//             with FP32 arithmetic and no periodic wrap): a warp reduces its cells by pencil and
//             the first lane of each pencil segment merges the result with atomic min / max on the
//             bit patterns (non-negative floats order like their bits); k_count resets the boxes
// The result is the stable order (key, caller index) regardless of the order the atomics took,
// so the permutation and cell table are identical on every run and bit-exact against a stable
// counting sort.
// HBM traffic per particle: xq read twice (8 or 12 B each), key and rank write + read (16 B),
// provisional and final permutation (12 B), gather of xq and C (12-16 B), sorted copy write
// (16 B); per cell: count, start and cursor words (about 16 B).
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

constexpr int kThreads = 256;
constexpr uint32_t kInfBits = 0x7f800000u;   // +inf: the lower bound of an empty pencil box
constexpr int kTileItems = 16;                        // cells per thread of the one-pass scan
constexpr int kTileCells = kThreads * kTileItems;     // cells per tile (one scan block): 4096
constexpr int kTileStride = 32;   // words between two tile totals: one 128-byte line each, so the
                                  // totals' atomics spread over the L2 slices
constexpr int kTileWindow = 8;    // tiles a block aggregates in shared memory (from its lowest)

// Adds the block's particles to their tiles' totals (tile = key / kTileCells, 0xffffffff for no
// particle).  Every thread of the block must call it.
__device__ __forceinline__ void add_tile_totals(uint32_t tile, uint32_t *__restrict__ tile_sums)
{
    // Every particle also counts toward its tile's total.  Particles of a block mostly fall in a
    // few neighbouring tiles: a warp whose particles share one tile adds once, the block sums
    // tiles [t0, t0 + kTileWindow) in shared memory (t0 its lowest tile) and adds each once.
    __shared__ uint32_t s_win[kTileWindow], s_t0;
    const int lane = threadIdx.x & 31;
    uint32_t lo = tile;
    for (int o = 16; o > 0; o >>= 1) lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    if (threadIdx.x < kTileWindow) s_win[threadIdx.x] = 0u;
    if (threadIdx.x == 0) s_t0 = 0xffffffffu;
    __syncthreads();
    if (lane == 0) atomicMin(&s_t0, lo);
    __syncthreads();
    const uint32_t t0 = s_t0;
    const bool one = __all_sync(0xffffffffu, tile == lo || tile == 0xffffffffu);
    if (one) {
        const uint32_t cnt = (uint32_t)__popc(__ballot_sync(0xffffffffu, tile != 0xffffffffu));
        if (lane == 0 && cnt) {
            if (lo - t0 < (uint32_t)kTileWindow) atomicAdd(&s_win[lo - t0], cnt);
            else atomicAdd(tile_sums + (size_t)lo * kTileStride, cnt);
        }
    } else if (tile != 0xffffffffu) {
        if (tile - t0 < (uint32_t)kTileWindow) atomicAdd(&s_win[tile - t0], 1u);
        else atomicAdd(tile_sums + (size_t)tile * kTileStride, 1u);
    }
    __syncthreads();
    if (threadIdx.x < kTileWindow && s_win[threadIdx.x])
        atomicAdd(tile_sums + (size_t)(t0 + threadIdx.x) * kTileStride, s_win[threadIdx.x]);
}

__global__ __launch_bounds__(kThreads) void k_count(const uint32_t *__restrict__ xq, int n, int dim,
                                                    int ncx, int ncy, int ncz,
                                                    uint32_t *__restrict__ keys,
                                                    uint32_t *__restrict__ rank,
                                                    uint32_t *__restrict__ count,
                                                    uint4 *__restrict__ pencil, int npencils,
                                                    uint32_t *__restrict__ tile_sums)
{
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * kThreads + threadIdx.x;
    if (pencil)   // empty boxes {min y, max y, min z, max z} = {+inf, 0, +inf, 0}: k_order merges into them
        for (int q = i; q < npencils; q += gridDim.x * kThreads) pencil[q] = make_uint4(kInfBits, 0u, kInfBits, 0u);
    uint32_t tile = 0xffffffffu;
    if (i < n) {
        const uint32_t key = cell_key(xq, n, i, dim, ncx, ncy, ncz);
        keys[i] = key;
        rank[i] = atomicAdd(count + key, 1u);
        tile = key / (uint32_t)kTileCells;
    }
    if (tile_sums) add_tile_totals(tile, tile_sums);
}

// Three-launch exclusive scan of count[0..m) into start[0..m] (start[m] = total).
constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;   // elements per scan block
static_assert(kScanTile == kScanTileCells, "scan tile size is shared with the workspace layouts");

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total)
{
    __shared__ uint32_t warp_sums[kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < kThreads / 32 ? warp_sums[lane] : 0u;
        uint32_t si = s;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += y;
        }
        if (lane < kThreads / 32) warp_sums[lane] = si - s;
        if (lane == kThreads / 32 - 1) *total = si;
    }
    __syncthreads();
    uint32_t r = warp_sums[wid] + incl - v;
    __syncthreads();
    return r;
}

__global__ __launch_bounds__(kThreads) void k_scan_blocks(const uint32_t *__restrict__ count, int m,
                                                          uint32_t *__restrict__ block_sums)
{
    pdl_wait();
    pdl_trigger();
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint32_t s = 0u;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < m) s += __ldg(count + base + k);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ uint32_t ws[kThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0u;
        for (int w = 0; w < kThreads / 32; ++w) t += ws[w];
        block_sums[blockIdx.x] = t;
    }
}

// One block: exclusive scan of the block sums in place, kScanTile at a time with a carry.
__global__ __launch_bounds__(kThreads) void k_scan_top(uint32_t *__restrict__ block_sums, int nb)
{
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t total;
    uint32_t carry = 0u;
    for (int chunk = 0; chunk < nb; chunk += kScanTile) {
        const int base = chunk + threadIdx.x * kScanItems;
        uint32_t v[kScanItems];
        uint32_t s = 0u;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            v[k] = base + k < nb ? block_sums[base + k] : 0u;
            s += v[k];
        }
        uint32_t run = block_exclusive_scan(s, &total) + carry;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (base + k < nb) block_sums[base + k] = run;
            run += v[k];
        }
        carry += total;
        __syncthreads();
    }
}

// Also clears count (each entry is read here once, by one thread), so the next build finds it zero.
// SUMS: block_off holds the blocks' plain sums (k_scan_top did not run) and every block adds up the
// sums of the blocks before it itself -- one launch less, for grids of up to kScanFoldBlocks blocks.
constexpr int kScanFoldBlocks = 1024;

template <bool SUMS>
__global__ __launch_bounds__(kThreads) void k_scan_apply(uint32_t *__restrict__ count, int m,
                                                         const uint32_t *__restrict__ block_off,
                                                         uint32_t *__restrict__ start)
{
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t total;
    uint32_t off = 0u;
    if (SUMS) {
        uint32_t part = 0u;
        for (int b = threadIdx.x; b < (int)blockIdx.x; b += kThreads) part += __ldg(block_off + b);
        block_exclusive_scan(part, &total);
        off = total;                      // read after the scan's closing barrier
        __syncthreads();                  // total is reused below
    } else {
        off = __ldg(block_off + blockIdx.x);
    }
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0u;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = 0u;
        if (base + k < m) {
            v[k] = count[base + k];
            count[base + k] = 0u;
        }
        s += v[k];
    }
    uint32_t run = block_exclusive_scan(s, &total) + off;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < m) start[base + k] = run;
        run += v[k];
    }
    if (base <= m - 1 && m - 1 < base + kScanItems) start[m] = run;  // holder of the last element
}

// One-pass exclusive scan of count[0..m) into start[0..m] (start[m] = total), replacing
// k_scan_blocks + k_scan_apply where the workspace holds the tile totals.  k_count has already
// added every particle to the total of its key's tile of kTileCells cells (tile_sums), so a block
// needs no other block: it sums the totals of the tiles before its own (its offset), scans its
// tile's counts and writes their starts.  No block waits on another.  Also clears count, like
// k_scan_apply; k_place clears the tile totals once every block has read them.
__global__ __launch_bounds__(kThreads) void k_scan_tiles(uint32_t *__restrict__ count, int m,
                                                         uint32_t *__restrict__ start,
                                                         const uint32_t *__restrict__ tile_sums)
{
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t s_part[kThreads / 32], total;
    const int b = blockIdx.x;
    uint32_t off = 0u;
    for (int q = threadIdx.x; q < b; q += kThreads) off += tile_sums[(size_t)q * kTileStride];
    for (int o = 16; o > 0; o >>= 1) off += __shfl_down_sync(0xffffffffu, off, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = off;
    const int base = b * kTileCells + threadIdx.x * kTileItems;
    uint32_t v[kTileItems];
    const bool whole = base + kTileItems <= m;   // vector loads and stores (16-byte aligned)
    if (whole) {
        uint4 *c4 = reinterpret_cast<uint4 *>(count + base);
#pragma unroll
        for (int q = 0; q < kTileItems / 4; ++q) {
            const uint4 t = c4[q];
            v[4 * q] = t.x;
            v[4 * q + 1] = t.y;
            v[4 * q + 2] = t.z;
            v[4 * q + 3] = t.w;
            c4[q] = make_uint4(0u, 0u, 0u, 0u);
        }
    } else {
#pragma unroll
        for (int k = 0; k < kTileItems; ++k) {
            v[k] = 0u;
            if (base + k < m) {
                v[k] = count[base + k];
                count[base + k] = 0u;
            }
        }
    }
    uint32_t sum = 0u;
#pragma unroll
    for (int k = 0; k < kTileItems; ++k) sum += v[k];
    uint32_t run = block_exclusive_scan(sum, &total);   // its barriers also publish s_part
    uint32_t boff = 0u;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) boff += s_part[w];
    run += boff;
    if (whole) {
        uint4 *s4 = reinterpret_cast<uint4 *>(start + base);
#pragma unroll
        for (int q = 0; q < kTileItems / 4; ++q) {
            uint4 t;
            t.x = run;
            run += v[4 * q];
            t.y = run;
            run += v[4 * q + 1];
            t.z = run;
            run += v[4 * q + 2];
            t.w = run;
            run += v[4 * q + 3];
            s4[q] = t;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kTileItems; ++k) {
            if (base + k < m) start[base + k] = run;
            run += v[k];
        }
    }
    if (base <= m - 1 && m - 1 < base + kTileItems) start[m] = run;  // holder of the last element
}

__global__ __launch_bounds__(kThreads) void k_place(const uint32_t *__restrict__ keys,
                                                    const uint32_t *__restrict__ rank, int n,
                                                    const uint32_t *__restrict__ start,
                                                    uint32_t *__restrict__ perm_tmp,
                                                    uint32_t *__restrict__ tile_sums, int ntiles)
{
    pdl_wait();
    pdl_trigger();
    if (tile_sums && blockIdx.x == 0)   // the scan has read them: clear for the next build
        for (int q = threadIdx.x; q < ntiles; q += kThreads) tile_sums[(size_t)q * kTileStride] = 0u;
    const int i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const uint32_t pos = __ldg(start + __ldg(keys + i)) + __ldg(rank + i);
    if (pos < (uint32_t)n) perm_tmp[pos] = (uint32_t)i;
}

constexpr uint32_t kSmallCell = 32;   // cells up to this size are ordered by one thread

// Orders one cell segment [s, e) of perm_tmp by caller index into perm and writes the sorted copy
// P[k] = rec(perm[k]), for the calling thread's cell when it is small; cells larger than
// kSmallCell are handled by order_big_cells.  The sort runs in registers (a 4-element sorting
// network, for the cells of up to four particles that dominate fine grids) or in a thread-local
// array (insertion sort), so the only global traffic is one read of the segment, the record
// gathers and the writes.
__device__ __forceinline__ void cswap(uint32_t &a, uint32_t &b)
{
    const uint32_t lo = min(a, b), hi = max(a, b);
    a = lo;
    b = hi;
}

// Position of fixed-point coordinate q inside its cell as a fraction of the cell (FP32 bit
// pattern): the low word of q nc is the offset within the cell in units of 2^-32 cells.
__device__ __forceinline__ uint32_t cell_frac_bits(uint32_t q, uint32_t nc)
{
    return __float_as_uint((float)(q * nc) * 2.3283064365386963e-10f);
}

// Transverse bounding box of one cell's (or a set of cells') particles as cell fractions, FP32
// bit patterns: {min y, max y, min z, max z}; z stays {0, 0} in 2D.
struct Box {
    uint32_t ylo = kInfBits, yhi = 0u, zlo = kInfBits, zhi = 0u;
    __device__ __forceinline__ void add(uint32_t fy, uint32_t fz)
    {
        ylo = min(ylo, fy);
        yhi = max(yhi, fy);
        zlo = min(zlo, fz);
        zhi = max(zhi, fz);
    }
    __device__ __forceinline__ void merge(const Box &o)
    {
        ylo = min(ylo, o.ylo);
        yhi = max(yhi, o.yhi);
        zlo = min(zlo, o.zlo);
        zhi = max(zhi, o.zhi);
    }
};

// Accumulates records into a box (the cell counts along y and z give the fractions).
struct BoxAcc {
    Box *box;
    uint32_t ncy, ncz;
    __device__ __forceinline__ void operator()(const uint4 &r) const
    {
        if (box) box->add(cell_frac_bits(r.y, ncy), cell_frac_bits(r.z, ncz));
    }
};

__device__ __forceinline__ Box shfl_down_box(const Box &b, int o)
{
    Box r;
    r.ylo = __shfl_down_sync(0xffffffffu, b.ylo, o);
    r.yhi = __shfl_down_sync(0xffffffffu, b.yhi, o);
    r.zlo = __shfl_down_sync(0xffffffffu, b.zlo, o);
    r.zhi = __shfl_down_sync(0xffffffffu, b.zhi, o);
    return r;
}

// Merges the warp's per-cell boxes into their pencils.  Lane l holds cell c (pencil c / ncx, or
// none when c >= ncells); consecutive lanes hold consecutive cells, so the lanes of one pencil form
// one contiguous segment.  A segmented shuffle reduction leaves each segment's box in its first
// lane, which merges it with one atomic min / max per word.  Every lane of the warp must call it.
__device__ __forceinline__ void merge_pencils(int c, int ncells, int ncx, Box b, uint4 *__restrict__ pencil)
{
    const int lane = threadIdx.x & 31;
    const unsigned p = c < ncells ? (unsigned)(c / ncx) : 0xffffffffu;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned p2 = __shfl_down_sync(0xffffffffu, p, o);
        const Box b2 = shfl_down_box(b, o);
        if (lane + o < 32 && p2 == p) b.merge(b2);
    }
    const unsigned pprev = __shfl_up_sync(0xffffffffu, p, 1);
    if (p != 0xffffffffu && (lane == 0 || pprev != p) && b.ylo <= b.yhi) {
        unsigned *w = reinterpret_cast<unsigned *>(pencil + p);
        atomicMin(w + 0, b.ylo);
        atomicMax(w + 1, b.yhi);
        if (b.zlo <= b.zhi) {
            atomicMin(w + 2, b.zlo);
            atomicMax(w + 3, b.zhi);
        }
    }
}

template <class Rec>
__device__ __forceinline__ void order_small_cell(uint32_t s, uint32_t e, const uint32_t *__restrict__ perm_tmp,
                                                 uint32_t *__restrict__ perm, uint4 *__restrict__ P, Rec rec,
                                                 BoxAcc acc = BoxAcc{nullptr, 0u, 0u})
{
    const uint32_t m = e - s;
    if (m <= 4) {
        uint32_t v0 = __ldg(perm_tmp + s);
        uint32_t v1 = m > 1 ? __ldg(perm_tmp + s + 1) : 0xffffffffu;
        uint32_t v2 = m > 2 ? __ldg(perm_tmp + s + 2) : 0xffffffffu;
        uint32_t v3 = m > 3 ? __ldg(perm_tmp + s + 3) : 0xffffffffu;
        cswap(v0, v1);
        cswap(v2, v3);
        cswap(v0, v2);
        cswap(v1, v3);
        cswap(v1, v2);
        const uint4 r0 = rec(v0);
        uint4 r1 = r0, r2 = r0, r3 = r0;
        if (m > 1) r1 = rec(v1);
        if (m > 2) r2 = rec(v2);
        if (m > 3) r3 = rec(v3);
        if (acc.box) {
            acc(r0);
            acc(r1);
            acc(r2);
            acc(r3);
        }
        perm[s] = v0;
        P[s] = r0;
        if (m > 1) {
            perm[s + 1] = v1;
            P[s + 1] = r1;
        }
        if (m > 2) {
            perm[s + 2] = v2;
            P[s + 2] = r2;
        }
        if (m > 3) {
            perm[s + 3] = v3;
            P[s + 3] = r3;
        }
        return;
    }
    uint32_t a[kSmallCell];
    for (uint32_t k = 0; k < m; ++k) a[k] = __ldg(perm_tmp + s + k);
    for (uint32_t k = 1; k < m; ++k) {
        const uint32_t v = a[k];
        uint32_t j = k;
        while (j > 0 && a[j - 1] > v) {
            a[j] = a[j - 1];
            --j;
        }
        a[j] = v;
    }
    for (uint32_t k = 0; k < m; ++k) {
        perm[s + k] = a[k];
        const uint4 r = rec(a[k]);
        acc(r);
        P[s + k] = r;
    }
}

// The big cells among the warp's 32 cells, one after another, each ordered by all 32 lanes: every
// element goes to s + (number of the cell's indices smaller than it), counted by streaming the
// segment through the warp 32 values at a time (coalesced load, broadcast by shuffles).  The
// indices are distinct, so the ranks are a permutation of the segment.  Every lane of the warp
// must call this (big = the lane's cell is valid and larger than kSmallCell).
template <class Rec>
__device__ __forceinline__ void order_big_cells(bool big, uint32_t s, uint32_t e,
                                                const uint32_t *__restrict__ perm_tmp,
                                                uint32_t *__restrict__ perm, uint4 *__restrict__ P, Rec rec,
                                                BoxAcc acc = BoxAcc{nullptr, 0u, 0u})
{
    const int lane = threadIdx.x & 31;
    unsigned todo = __ballot_sync(0xffffffffu, big);
    while (todo) {
        const int l = __ffs(todo) - 1;
        todo &= todo - 1u;
        const uint32_t bs = __shfl_sync(0xffffffffu, s, l), be = __shfl_sync(0xffffffffu, e, l);
        Box cb;   // this big cell's box, gathered over the lanes and handed to lane l
        for (uint32_t k0 = bs; k0 < be; k0 += 32) {
            const uint32_t k = k0 + (uint32_t)lane;
            const bool has = k < be;
            const uint32_t v = has ? __ldg(perm_tmp + k) : 0xffffffffu;
            uint32_t rank = 0u;
            for (uint32_t t0 = bs; t0 < be; t0 += 32) {
                const uint32_t u = t0 + (uint32_t)lane < be ? __ldg(perm_tmp + t0 + lane) : 0xffffffffu;
#pragma unroll
                for (int q = 0; q < 32; ++q) rank += __shfl_sync(0xffffffffu, u, q) < v ? 1u : 0u;
            }
            if (has && bs + rank < be) {
                perm[bs + rank] = v;
                const uint4 r = rec(v);
                if (acc.box) cb.add(cell_frac_bits(r.y, acc.ncy), cell_frac_bits(r.z, acc.ncz));
                P[bs + rank] = r;
            }
        }
        if (acc.box) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cb.merge(shfl_down_box(cb, o));
            const Box c0{__shfl_sync(0xffffffffu, cb.ylo, 0), __shfl_sync(0xffffffffu, cb.yhi, 0),
                         __shfl_sync(0xffffffffu, cb.zlo, 0), __shfl_sync(0xffffffffu, cb.zhi, 0)};
            if (lane == l) acc.box->merge(c0);
        }
    }
}

struct PlainRec {
    const uint32_t *xq;
    const float *C;
    int n, dim;
    __device__ __forceinline__ uint4 operator()(uint32_t a) const
    {
        uint4 p;
        p.x = __ldg(xq + a);
        p.y = __ldg(xq + n + a);
        p.z = dim == 3 ? __ldg(xq + 2 * (size_t)n + a) : 0u;
        p.w = __float_as_uint(__ldg(C + a));
        return p;
    }
};

// One thread per cell: order the cell's segment by caller index and write the sorted copy.
__global__ __launch_bounds__(kThreads) void k_order(const uint32_t *__restrict__ start, int ncells,
                                                    const uint32_t *__restrict__ perm_tmp,
                                                    const uint32_t *__restrict__ xq,
                                                    const float *__restrict__ C, int n, int dim,
                                                    uint32_t *__restrict__ perm,
                                                    uint4 *__restrict__ P, int ncx, int ncy, int ncz,
                                                    uint4 *__restrict__ pencil)
{
    pdl_wait();
    pdl_trigger();
    const int c = blockIdx.x * kThreads + threadIdx.x;
    uint32_t s = 0u, e = 0u;
    if (c < ncells) {
        s = __ldg(start + c);
        e = __ldg(start + c + 1);
    }
    const bool valid = e > s && e <= (uint32_t)n;
    const PlainRec rec{xq, C, n, dim};
    Box box;
    const BoxAcc bacc{pencil ? &box : nullptr, (uint32_t)ncy, (uint32_t)ncz};
    if (valid && e - s <= kSmallCell) order_small_cell(s, e, perm_tmp, perm, P, rec, bacc);
    order_big_cells(valid && e - s > kSmallCell, s, e, perm_tmp, perm, P, rec, bacc);
    if (pencil) merge_pencils(c, ncells, ncx, box, pencil);
}

// One block per cell, for grids whose cells hold many particles on average (wide kernels, coarse
// subdivisions): every thread ranks kRankItems elements at a time against the whole segment,
// streamed through shared memory kRankChunk values at a time; the element goes to s + rank.
constexpr int kRankChunk = 2048;
constexpr int kRankItems = 4;

__global__ __launch_bounds__(kThreads) void k_order_block(const uint32_t *__restrict__ start, int ncells,
                                                          const uint32_t *__restrict__ perm_tmp,
                                                          const uint32_t *__restrict__ xq,
                                                          const float *__restrict__ C, int n, int dim,
                                                          uint32_t *__restrict__ perm, uint4 *__restrict__ P,
                                                          int ncx, int ncy, int ncz, uint4 *__restrict__ pencil)
{
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t chunk[kRankChunk];
    __shared__ Box wbox[kThreads / 32];
    const int c = blockIdx.x;
    if (c >= ncells) return;
    const uint32_t s = __ldg(start + c), e = __ldg(start + c + 1);
    if (e <= s || e > (uint32_t)n) return;                       // uniform over the block
    const PlainRec rec{xq, C, n, dim};
    Box box;
    for (uint32_t k0 = s; k0 < e; k0 += kThreads * kRankItems) {
        uint32_t v[kRankItems], rank[kRankItems];
#pragma unroll
        for (int r = 0; r < kRankItems; ++r) {
            const uint32_t k = k0 + threadIdx.x + r * kThreads;
            v[r] = k < e ? __ldg(perm_tmp + k) : 0xffffffffu;
            rank[r] = 0u;
        }
        for (uint32_t t0 = s; t0 < e; t0 += kRankChunk) {
            const uint32_t len = e - t0 < (uint32_t)kRankChunk ? e - t0 : (uint32_t)kRankChunk;
            __syncthreads();
            for (uint32_t t = threadIdx.x; t < len; t += kThreads) chunk[t] = __ldg(perm_tmp + t0 + t);
            __syncthreads();
            for (uint32_t t = 0; t < len; ++t) {
                const uint32_t u = chunk[t];
#pragma unroll
                for (int r = 0; r < kRankItems; ++r) rank[r] += u < v[r] ? 1u : 0u;
            }
        }
#pragma unroll
        for (int r = 0; r < kRankItems; ++r) {
            const uint32_t k = k0 + threadIdx.x + r * kThreads;
            if (k < e && s + rank[r] < e) {
                perm[s + rank[r]] = v[r];
                const uint4 q = rec(v[r]);
                if (pencil) box.add(cell_frac_bits(q.y, (uint32_t)ncy), cell_frac_bits(q.z, (uint32_t)ncz));
                P[s + rank[r]] = q;
            }
        }
    }
    if (pencil) {   // block reduction of the cell's box, one merge into its pencil
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) box.merge(shfl_down_box(box, o));
        if ((threadIdx.x & 31) == 0) wbox[threadIdx.x >> 5] = box;
        __syncthreads();
        if (threadIdx.x == 0) {
            Box b = wbox[0];
            for (int w = 1; w < kThreads / 32; ++w) b.merge(wbox[w]);
            unsigned *pw = reinterpret_cast<unsigned *>(pencil + c / ncx);
            if (b.ylo <= b.yhi) {
                atomicMin(pw + 0, b.ylo);
                atomicMax(pw + 1, b.yhi);
            }
            if (b.zlo <= b.zhi) {
                atomicMin(pw + 2, b.zlo);
                atomicMax(pw + 3, b.zhi);
            }
        }
    }
}

// Batched plumes: caller particle i belongs to plume p = plume_of[i], whose positions are the
// [dim][n_p] block starting at xq + dim * goff_p; its key is coff_p + the plume-local key.
__global__ __launch_bounds__(kThreads) void k_count_batch(const uint32_t *__restrict__ xq, int n, int dim,
                                                          const RateParams *__restrict__ descs,
                                                          const uint16_t *__restrict__ plume_of,
                                                          uint32_t *__restrict__ keys,
                                                          uint32_t *__restrict__ rank,
                                                          uint32_t *__restrict__ count,
                                                          uint32_t *__restrict__ tile_sums)
{
    const int i = blockIdx.x * kThreads + threadIdx.x;
    uint32_t tile = 0xffffffffu;
    if (i < n) {
        const RateParams &d = descs[__ldg(plume_of + i)];
        const int np = d.n, goff = d.goff;
        const uint32_t key =
            (uint32_t)d.coff + cell_key(xq + (size_t)dim * goff, np, i - goff, dim, d.ncx, d.ncy, d.ncz);
        keys[i] = key;
        rank[i] = atomicAdd(count + key, 1u);
        tile = key / (uint32_t)kTileCells;
    }
    if (tile_sums) add_tile_totals(tile, tile_sums);
}

struct BatchRec {
    const uint32_t *xq;
    const float *C;
    int dim;
    const RateParams *descs;
    const uint16_t *plume_of;
    __device__ __forceinline__ uint4 operator()(uint32_t a) const
    {
        const RateParams &d = descs[__ldg(plume_of + a)];
        const uint32_t *xp = xq + (size_t)dim * d.goff;
        const uint32_t l = a - (uint32_t)d.goff, np = (uint32_t)d.n;
        uint4 p;
        p.x = __ldg(xp + l);
        p.y = __ldg(xp + np + l);
        p.z = dim == 3 ? __ldg(xp + 2 * (size_t)np + l) : 0u;
        p.w = __float_as_uint(__ldg(C + a));
        return p;
    }
};

__global__ __launch_bounds__(kThreads) void k_order_batch(const uint32_t *__restrict__ start, int ncells,
                                                          const uint32_t *__restrict__ perm_tmp,
                                                          const uint32_t *__restrict__ xq,
                                                          const float *__restrict__ C, int n, int dim,
                                                          const RateParams *__restrict__ descs,
                                                          const uint16_t *__restrict__ plume_of,
                                                          uint32_t *__restrict__ perm,
                                                          uint4 *__restrict__ P)
{
    const int c = blockIdx.x * kThreads + threadIdx.x;
    uint32_t s = 0u, e = 0u;
    if (c < ncells) {
        s = __ldg(start + c);
        e = __ldg(start + c + 1);
    }
    const bool valid = e > s && e <= (uint32_t)n;
    const BatchRec rec{xq, C, dim, descs, plume_of};
    if (valid && e - s <= kSmallCell) order_small_cell(s, e, perm_tmp, perm, P, rec);
    order_big_cells(valid && e - s > kSmallCell, s, e, perm_tmp, perm, P, rec);
}

}  // namespace

int scan_blocks(int m) { return (m + kScanTile - 1) / kScanTile; }

int tile_blocks(int m) { return (m + kTileCells - 1) / kTileCells; }
size_t tile_sums_bytes(int m) { return (size_t)tile_blocks(m) * kTileStride * sizeof(uint32_t); }

int cell_build_launches(int n, int ncells, bool onepass)
{
    const int scans = onepass ? 1 : (scan_blocks(ncells) <= kScanFoldBlocks ? 2 : 3);
    return scans + (n > 0 ? 3 : 0);   // k_count, k_place, k_order (or k_order_block)
}

cudaError_t launch_build_cells_batch(int dim, const uint32_t *xq, const float *C, int n, int ncells,
                                     const RateParams *descs, const uint16_t *plume_of,
                                     const Work &w, cudaStream_t s)
{
    const int nt = tile_blocks(ncells);
    cudaError_t e = cudaMemsetAsync(w.count, 0, (size_t)ncells * sizeof(uint32_t), s);
    if (e == cudaSuccess && w.tile_sums) e = cudaMemsetAsync(w.tile_sums, 0, (size_t)nt * kTileStride * 4, s);
    if (e != cudaSuccess) return e;
    const int nb = (n + kThreads - 1) / kThreads;
    if (nb > 0)
        k_count_batch<<<nb, kThreads, 0, s>>>(xq, n, dim, descs, plume_of, w.keys, w.rank, w.count, w.tile_sums);
    if (w.tile_sums) {
        k_scan_tiles<<<nt, kThreads, 0, s>>>(w.count, ncells, w.cell_start, (const uint32_t *)w.tile_sums);
    } else {
        const int sb = scan_blocks(ncells);
        k_scan_blocks<<<sb, kThreads, 0, s>>>(w.count, ncells, w.block_sums);
        k_scan_top<<<1, kThreads, 0, s>>>(w.block_sums, sb);
        k_scan_apply<false><<<sb, kThreads, 0, s>>>(w.count, ncells, w.block_sums, w.cell_start);
    }
    if (nb > 0) {
        k_place<<<nb, kThreads, 0, s>>>(w.keys, w.rank, n, w.cell_start, w.perm_tmp, w.tile_sums, nt);
        k_order_batch<<<(ncells + kThreads - 1) / kThreads, kThreads, 0, s>>>(
            w.cell_start, ncells, w.perm_tmp, xq, C, n, dim, descs, plume_of, w.perm, w.P0);
    }
    return cudaGetLastError();
}

cudaError_t launch_build_cells(int dim, const uint32_t *xq, const float *C, int n, const int *nc,
                               int ncells, const Work &w, cudaStream_t s, bool count_zero)
{
    const int nt = tile_blocks(ncells);
    cudaError_t e = count_zero ? cudaSuccess : cudaMemsetAsync(w.count, 0, (size_t)ncells * sizeof(uint32_t), s);
    if (e == cudaSuccess && !count_zero && w.tile_sums)
        e = cudaMemsetAsync(w.tile_sums, 0, (size_t)nt * kTileStride * 4, s);
    if (e != cudaSuccess) return e;
    const int nb = (n + kThreads - 1) / kThreads;
    if (nb > 0 && e == cudaSuccess)
        e = launch_pdl(k_count, nb, kThreads, 0, s, xq, n, dim, nc[0], nc[1], nc[2], w.keys, w.rank, w.count,
                       w.pencil, ncells / nc[0], w.tile_sums);
    const int sb = scan_blocks(ncells);
    if (w.tile_sums) {
        if (e == cudaSuccess)
            e = launch_pdl(k_scan_tiles, nt, kThreads, 0, s, w.count, ncells, w.cell_start,
                           (const uint32_t *)w.tile_sums);
    } else if (sb <= kScanFoldBlocks) {
        if (e == cudaSuccess) e = launch_pdl(k_scan_blocks, sb, kThreads, 0, s, w.count, ncells, w.block_sums);
        if (e == cudaSuccess)
            e = launch_pdl(k_scan_apply<true>, sb, kThreads, 0, s, w.count, ncells, w.block_sums, w.cell_start);
    } else {
        if (e == cudaSuccess) e = launch_pdl(k_scan_blocks, sb, kThreads, 0, s, w.count, ncells, w.block_sums);
        if (e == cudaSuccess) e = launch_pdl(k_scan_top, 1, kThreads, 0, s, w.block_sums, sb);
        if (e == cudaSuccess)
            e = launch_pdl(k_scan_apply<false>, sb, kThreads, 0, s, w.count, ncells, w.block_sums, w.cell_start);
    }
    if (nb > 0 && e == cudaSuccess) {
        e = launch_pdl(k_place, nb, kThreads, 0, s, w.keys, w.rank, n, w.cell_start, w.perm_tmp, w.tile_sums, nt);
        if (e != cudaSuccess) return e;
        if ((long long)n >= 16ll * ncells)   // many particles per cell: one block per cell
            e = launch_pdl(k_order_block, ncells, kThreads, 0, s, w.cell_start, ncells, w.perm_tmp, xq, C, n,
                           dim, w.perm, w.P0, nc[0], nc[1], nc[2], w.pencil);
        else
            e = launch_pdl(k_order, (ncells + kThreads - 1) / kThreads, kThreads, 0, s, w.cell_start, ncells,
                           w.perm_tmp, xq, C, n, dim, w.perm, w.P0, nc[0], nc[1], nc[2], w.pencil);
    }
    return e;
}

}  // namespace ade
