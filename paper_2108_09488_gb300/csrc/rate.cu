// rate.cu -- the neighbour-interaction kernel: Eq. 4-5 (Sec. 2.2) for every particle, with the
// predictor and corrector of Eq. 8-9 (Sec. 2.4) fused into its epilogue.
//
// For a uniform velocity field (Sec. 3) every particle carries the same tensor D (Eq. 3), so the
// per-component harmonic mean of Eq. 5 is 4 D D / (D + D) = 2 D and the pair factor reduces to
//     Dcal_ab = Gamma e^T K e - tr K = a (vhat . e)^2 + b,   K = 2 D, e = x_ab / r,
// a = 2 Gamma (alpha_L - alpha_T)|v|, b = 2 (Gamma - dim)(alpha_T |v| + D_m) - 2 (alpha_L - alpha_T)|v|
// (D = d_T I + (d_L - d_T) vhat vhat^T): one dot product, one product with 1/r and one fused
// multiply-add per pair, t = (sqrt|a| vhat . x_ab) / r, Dcal = sign(a) (t^2 + sign(a) b).
// With grad_a W = W'(r) x_ab / r, the dispersive term of Eq. 4 for one ordered pair is
//     1/2 (m_b / rhobar) Dcal_ab (C_a - C_b) W'(r) / r,
// and W'(r)/r = kc f(q): Wendland C2 (support H = 2h): f = (1-q)^3, kc = -20 B / H^2;
// Wendland C4 (Eq. 7, support H = h): f = (1-q)^5 (1+5q), kc = -(56/3) B / H^2.
// The convective term of Eq. 4 is identically zero for uniform v and is not evaluated.
//
// The walks share the pair arithmetic and the epilogue (rate_walk.cuh):
//   * direct (variants 0, 2, 3, 4; this file): one thread per cell-sorted particle; candidates are
//     read from the sorted copy in global memory (L1-cached 16-byte words {x, y, z, C});
//     separations are int32 differences of fixed-point words converted to FP32 for every pair;
//     each stencil row (2w+1 cells with consecutive keys) is one contiguous index range, two at a
//     periodic seam.  Branch-free (0, 3) or branching on the support test (2, 4), over the full
//     stencil (0, 2) or the cells within reach of the particle (trimmed rows: 3, 4).
//   * paired (variants 5-8; rate_pair.cu): the direct walks with two adjacent sorted particles per
//     thread sharing one candidate stream, the FP32 arithmetic packed in FP32x2 instructions.
//   * tiled (variant 1; this file): one CTA per block of TX x TY (x TZ) cells.  The CTA stages
//     every particle of the block and its k-cell halo into shared memory once, as int32 fixed-point
//     offsets from the block centre (the minimum image from the centre), plus a local cell start
//     table.  Each thread then walks its targets' stencil rows over shared memory; the pair
//     separation is the exact int32 difference converted to FP32, as in the direct walk, so both
//     round relative to the separation itself rather than to the block size.  The pair term is
//     evaluated without a branch: outside the support (1 - q) is clamped to 0, so the term
//     vanishes.  A block whose halo does not fit the staging buffer falls back to the direct walk.
//   * batched (this file): the direct walk over a persistent queue of (plume, range) work items.
// All walks sum each stencil row's terms in FP32 and add the row sums with Neumaier's compensated
// summation, visiting rows and, inside a row, particles in sorted order, so results are
// deterministic; the branch-free walks (full, trimmed, paired, tiled) give the same bits, and so
// do the branched ones among themselves (they can differ from the branch-free walks only by a
// term whose separation rounds to the support radius).
#include "ade_internal.h"

namespace ade {

namespace {

#include "rate_common.cuh"

#include "rate_walk.cuh"

// ---------------------------------------------------------------------------------------------
// direct kernel
// ---------------------------------------------------------------------------------------------
template <int DIM, int KERNEL, int EPI, bool ISO, bool COUNT, bool BF, bool TRIM>
__global__ __launch_bounds__(kRateThreads) void k_rate(const uint4 *__restrict__ Pe,
                                                       const uint4 *__restrict__ Pc,
                                                       const uint32_t *__restrict__ cs,
                                                       const uint32_t *__restrict__ perm,
                                                       const RateParams prm, const EpiOut out)
{
    pdl_wait();   // no early trigger: see pdl_trigger
    const int i = blockIdx.x * kRateThreads + threadIdx.x;
    const bool valid = i < prm.n;
    const int ii = valid ? i : prm.n - 1;
    const uint4 pa = __ldg(Pe + ii);
    // cell of the cell build: evaluation position minus the drift since the build
    const int cx = (int)__umulhi(pa.x - prm.back[0], (uint32_t)prm.ncx);
    const int cy = (int)__umulhi(pa.y - prm.back[1], (uint32_t)prm.ncy);
    const int cz = DIM == 3 ? (int)__umulhi(pa.z - prm.back[2], (uint32_t)prm.ncz) : 0;
    Acc acc{0.f, 0.f, __int_as_float(0x7f800000), __int_as_float(0xff800000), 0u};
    unsigned cnt = 0u;
    // Corrector: the caller index and C^l are loaded ahead of the pair loop (not in the trimmed
    // walk, where the two live registers cost more occupancy than the hidden latency gains).
    constexpr bool PRE = EPI == EPI_CORRECT && !TRIM;
    uint32_t a_pre = 0u;
    float C_pre = 0.f;
    if (PRE) {
        a_pre = __ldg(perm + ii);
        if (a_pre - (uint32_t)prm.goff < (uint32_t)prm.n) C_pre = out.C[a_pre];
    }
    __shared__ TrimRow srow[TRIM ? kMaxRows : 1];
    if (TRIM) stage_trim_rows(srow, prm);
    bool coop = false;   // every lane of the warp in one pencil: rows tested once per warp
    if (TRIM) {
        const int cyw = __shfl_sync(0xffffffffu, cy, 0), czw = __shfl_sync(0xffffffffu, cz, 0);
        coop = __all_sync(0xffffffffu, cy == cyw && cz == czw);
    }
    const float rate = rate_direct<DIM, KERNEL, ISO, COUNT, BF, TRIM>(Pe, cs, pa, cx, cy, cz, prm, cnt, srow, coop);
    if (valid) {
        acc.cnt = cnt;
        epilogue<DIM, EPI, PRE>(i, rate, pa, perm, prm, out, acc, a_pre, C_pre);
    }
    warp_finish<EPI, COUNT, kRateThreads>(acc, out);
}

// ---------------------------------------------------------------------------------------------
// tiled kernel
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int wrap_cell(int c, int n)
{
    c %= n;
    return c < 0 ? c + n : c;
}

// Shared-memory layout of the tiled kernel (dynamic shared memory):
//   int4   sp[cap]                staged particles {x, y, z, C bits}, offsets from the centre
//   int    lcs[hrows][HX + 1]     local start of every halo cell, per halo row (+ row end)
//   int    trow[3][tr + 1]        per inner row: target prefix, global sorted start, local start
template <int DIM, int KERNEL, int EPI, bool COUNT>
__global__ __launch_bounds__(kTileThreads, 2) void k_rate_tiled(const uint4 *__restrict__ Pe,
                                                             const uint4 *__restrict__ Pc,
                                                             const uint32_t *__restrict__ cs,
                                                             const uint32_t *__restrict__ perm,
                                                             const RateParams prm, const EpiOut out)
{
    pdl_wait();   // no early trigger: see pdl_trigger
    extern __shared__ float4 smem[];
    __shared__ int s_total;
    __shared__ int wsum[kTileThreads / 32];
    const int k = prm.k;
    const int TX = prm.tx, TY = prm.ty, TZ = DIM == 3 ? prm.tz : 1;
    const int HX = TX + 2 * k, HY = TY + 2 * k, HZ = DIM == 3 ? TZ + 2 * k : 1;
    const int kz = DIM == 3 ? k : 0;
    const int ncx = prm.ncx, ncy = prm.ncy, ncz = prm.ncz;
    const int b = blockIdx.x;
    const int tx0 = (b % prm.ntx) * TX;
    const int ty0 = ((b / prm.ntx) % prm.nty) * TY;
    const int tz0 = DIM == 3 ? (b / (prm.ntx * prm.nty)) * TZ : 0;
    const int vx = min(TX, ncx - tx0), vy = min(TY, ncy - ty0), vz = DIM == 3 ? min(TZ, ncz - tz0) : 1;
    const int hrows = HY * HZ;
    const int NH = HX * hrows;
    const int tr = TY * TZ;

    int4 *sp = reinterpret_cast<int4 *>(smem);
    int *lcs = reinterpret_cast<int *>(sp + prm.cap);
    int *tpre = lcs + hrows * (HX + 1);
    int *tglb = tpre + tr + 1;
    int *tloc = tglb + tr + 1;

    // 1. counts of the halo cells, exclusive scan in (row, x) order -> local cell starts
    int carry = 0;
    for (int h0 = 0; h0 < NH; h0 += kTileThreads) {
        const int h = h0 + threadIdx.x;
        int cnt = 0, hx = 0, row = 0;
        if (h < NH) {
            hx = h % HX;
            row = h / HX;
            const int hy = row % HY, hz = row / HY;
            const int gx = wrap_cell(tx0 - k + hx, ncx);
            const int gy = wrap_cell(ty0 - k + hy, ncy);
            const int gz = DIM == 3 ? wrap_cell(tz0 - k + hz, ncz) : 0;
            const int g = (gz * ncy + gy) * ncx + gx;
            cnt = (int)(__ldg(cs + g + 1) - __ldg(cs + g));
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int v = lane < kTileThreads / 32 ? wsum[lane] : 0;
            int vi = v;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, vi, o);
                if (lane >= o) vi += y;
            }
            if (lane < kTileThreads / 32) wsum[lane] = vi - v;
            if (lane == kTileThreads / 32 - 1) s_total = vi;
        }
        __syncthreads();
        const int excl = carry + wsum[wid] + incl - cnt;
        if (h < NH) {
            lcs[row * (HX + 1) + hx] = excl;
            if (hx == HX - 1) lcs[row * (HX + 1) + HX] = excl + cnt;
        }
        carry += s_total;
        __syncthreads();
    }
    // 2. target rows: inner cells [tx0, tx0 + vx) of every inner row, contiguous in sorted order
    if (threadIdx.x == 0) {
        int run = 0;
        for (int r = 0; r < tr; ++r) {
            const int iy = r % TY, iz = r / TY;
            tpre[r] = run;
            tglb[r] = 0;
            tloc[r] = 0;
            if (iy < vy && iz < vz) {
                const int g = ((tz0 + iz) * ncy + (ty0 + iy)) * ncx + tx0;
                const int g0 = (int)__ldg(cs + g), g1 = (int)__ldg(cs + g + vx);
                tglb[r] = g0;
                tloc[r] = lcs[((iz + kz) * HY + (iy + k)) * (HX + 1) + k];
                run += g1 - g0;
            }
        }
        tpre[tr] = run;
    }
    __syncthreads();
    const int ntarget = tpre[tr];
    const bool staged = carry <= prm.cap;

    // 3. stage the halo: one thread per halo cell copies that cell's particles
    if (staged) {
        const uint32_t ox = (uint32_t)(((unsigned long long)(2 * tx0 + TX) << 31) / (unsigned)ncx);
        const uint32_t oy = (uint32_t)(((unsigned long long)(2 * ty0 + TY) << 31) / (unsigned)ncy);
        const uint32_t oz =
            DIM == 3 ? (uint32_t)(((unsigned long long)(2 * tz0 + TZ) << 31) / (unsigned)ncz) : 0u;
        for (int h = threadIdx.x; h < NH; h += kTileThreads) {
            const int hx = h % HX, row = h / HX;
            const int hy = row % HY, hz = row / HY;
            const int gx = wrap_cell(tx0 - k + hx, ncx);
            const int gy = wrap_cell(ty0 - k + hy, ncy);
            const int gz = DIM == 3 ? wrap_cell(tz0 - k + hz, ncz) : 0;
            const int g = (gz * ncy + gy) * ncx + gx;
            const int g0 = (int)__ldg(cs + g), g1 = (int)__ldg(cs + g + 1);
            const int l0 = lcs[row * (HX + 1) + hx];
            for (int p = g0; p < g1; ++p) {
                const uint4 q = __ldg(Pe + p);
                sp[l0 + (p - g0)] = make_int4((int)(q.x - ox), (int)(q.y - oy),
                                              DIM == 3 ? (int)(q.z - oz) : 0, (int)q.w);
            }
        }
    }
    __syncthreads();

    // 4. targets: thread t takes targets t, t + NT, ... in (row, sorted) order
    Acc acc{0.f, 0.f, __int_as_float(0x7f800000), __int_as_float(0xff800000), 0u};
    int r = 0;
    for (int t = threadIdx.x; t < ntarget; t += kTileThreads) {
        while (tpre[r + 1] <= t) ++r;
        const int off = t - tpre[r];
        const int gi = tglb[r] + off;
        const uint4 pe = __ldg(Pe + gi);
        const int cx = (int)__umulhi(pe.x - prm.back[0], (uint32_t)ncx);
        const int cy = (int)__umulhi(pe.y - prm.back[1], (uint32_t)ncy);
        const int cz = DIM == 3 ? (int)__umulhi(pe.z - prm.back[2], (uint32_t)ncz) : 0;
        float rate;
        unsigned cnt = 0u;
        if (staged) {
            const int4 a = sp[tloc[r] + off];
            const float Ca = __int_as_float(a.w);
            const int hx = cx - tx0 + k, hy = cy - ty0 + k, hz = DIM == 3 ? cz - tz0 + k : 0;
            const PairConst kc(prm);
            float sum = 0.f, comp = 0.f;
            for (int ri = 0; ri < prm.nrows; ++ri) {
                const StencilRow row = prm.rows[ri];
                const int *lrow = lcs + ((hz + row.dz) * HY + (hy + row.dy)) * (HX + 1);
                const int j0 = lrow[hx - row.w], j1 = lrow[hx + row.w + 1];
                float rs = 0.f;
#pragma unroll 2
                for (int j = j0; j < j1; ++j) {
                    const int4 q = sp[j];
                    const float dx = (float)(a.x - q.x), dy = (float)(a.y - q.y);
                    const float dz = DIM == 3 ? (float)(a.z - q.z) : 0.f;
                    float r2 = fmaf(dx, dx, dy * dy);
                    if (DIM == 3) r2 = fmaf(dz, dz, r2);
                    const float rinv = rsqrt_ftz(fmaxf(r2, 1.0f));
                    const float om = fmaf(-r2 * rinv, kc.invH, 1.f);
                    const float s = dcal<DIM>(dx, dy, dz, rinv, kc);
                    const float w = r2 > 0.f ? shape2x<KERNEL>(om + fabsf(om)) * s : 0.f;
                    rs = fmaf(w, Ca - __int_as_float(q.w), rs);
                    if (COUNT) cnt += in_support_fp64<DIM>(a.x - q.x, a.y - q.y, a.z - q.z, prm);
                }
                neumaier_add(sum, comp, rs);
            }
            rate = prm.upf * shape_unscale<KERNEL>() * (sum + comp);
        } else {
            rate = rate_direct<DIM, KERNEL, true, COUNT>(Pe, cs, pe, cx, cy, cz, prm, cnt);
        }
        acc.cnt += cnt;
        epilogue<DIM, EPI>(gi, rate, pe, perm, prm, out, acc);
    }
    warp_finish<EPI, COUNT, kTileThreads>(acc, out);
}

// ---------------------------------------------------------------------------------------------
// batched plumes: persistent kernel over a queue of (plume, range) work items
// ---------------------------------------------------------------------------------------------
// Every warp takes work items from an atomic counter until the list is exhausted (no warp waits
// on another).  An item is a range of one plume's cell-sorted particles; the plume's constants are
// copied to the warp's shared-memory slot when the plume changes and each particle is evaluated with the same code as the
// single-plume direct kernel (rate_direct + epilogue), so a plume gives bit-identical results
// whether it runs alone or in a batch.  Items are ordered by decreasing estimated cost.
// PAIRED: each thread takes two adjacent sorted particles of the item (rate_direct_pair; a pair
// that cannot share a candidate stream takes the one-target walk for each), with the same sums.
template <int DIM, int KERNEL, int EPI, bool COUNT, bool PAIRED>
__global__ __launch_bounds__(kRateThreads) void k_rate_batch(const uint4 *__restrict__ Pe,
                                                             const uint32_t *__restrict__ cs,
                                                             const uint32_t *__restrict__ perm,
                                                             const RateParams *__restrict__ descs,
                                                             const BatchTile *__restrict__ tiles,
                                                             int ntiles, unsigned *queue,
                                                             const EpiOut out)
{
    // Every warp takes work items on its own (no block barrier): its plume's constants live in
    // the warp's own shared-memory slot, refreshed when the plume changes.
    __shared__ RateParams sp[kRateThreads / 32];
    constexpr int kWords = (int)(sizeof(RateParams) / sizeof(int));
    static_assert(sizeof(RateParams) % sizeof(int) == 0, "RateParams is copied word by word");
    const int lane = threadIdx.x & 31;
    RateParams &mine = sp[threadIdx.x >> 5];
    int cur = -1;
    unsigned cnt = 0u;
    for (;;) {
        int item = 0;
        if (lane == 0) item = (int)atomicAdd(queue, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= ntiles) break;
        const BatchTile t = tiles[item];
        if (t.plume != cur) {
            const int *src = reinterpret_cast<const int *>(descs + t.plume);
            int *dst = reinterpret_cast<int *>(&mine);
            for (int w = lane; w < kWords; w += 32) dst[w] = __ldg(src + w);
            cur = t.plume;
            __syncwarp();
        }
        const RateParams &prm = mine;
        EpiOut o = out;
        if (EPI == EPI_CORRECT) o.xq = out.xq + (size_t)prm.goff * (DIM - 1);
        if (PAIRED && !COUNT) {
            for (int k = 2 * lane; k < t.count; k += 64) {
                const int g0 = prm.goff + t.start + k;
                const bool v1 = k + 1 < t.count;
                const uint4 pa0 = __ldg(Pe + g0);
                const uint4 pa1 = __ldg(Pe + (v1 ? g0 + 1 : g0));
                const int cx0 = (int)__umulhi(pa0.x - prm.back[0], (uint32_t)prm.ncx);
                const int cy0 = (int)__umulhi(pa0.y - prm.back[1], (uint32_t)prm.ncy);
                const int cz0 = DIM == 3 ? (int)__umulhi(pa0.z - prm.back[2], (uint32_t)prm.ncz) : 0;
                const int cx1 = (int)__umulhi(pa1.x - prm.back[0], (uint32_t)prm.ncx);
                const int cy1 = (int)__umulhi(pa1.y - prm.back[1], (uint32_t)prm.ncy);
                const int cz1 = DIM == 3 ? (int)__umulhi(pa1.z - prm.back[2], (uint32_t)prm.ncz) : 0;
                float r0, r1 = 0.f;
                unsigned c = 0u;
                if (v1 && can_pair(cx0, cy0, cz0, cx1, cy1, cz1, prm.ncx)) {
                    rate_direct_pair<DIM, KERNEL, true, false>(Pe, cs + prm.coff, pa0, pa1, cx0, cx1, cy0, cz0, prm,
                                                               r0, r1);
                } else {
                    r0 = rate_direct<DIM, KERNEL, true, false>(Pe, cs + prm.coff, pa0, cx0, cy0, cz0, prm, c);
                    if (v1) r1 = rate_direct<DIM, KERNEL, true, false>(Pe, cs + prm.coff, pa1, cx1, cy1, cz1, prm, c);
                }
                Acc acc{0.f, 0.f, 0.f, 0.f, 0u};
                epilogue<DIM, EPI>(g0, r0, pa0, perm, prm, o, acc);
                if (v1) epilogue<DIM, EPI>(g0 + 1, r1, pa1, perm, prm, o, acc);
            }
        } else {
            for (int k = lane; k < t.count; k += 32) {
                const int gi = prm.goff + t.start + k;
                const uint4 pa = __ldg(Pe + gi);
                const int cx = (int)__umulhi(pa.x - prm.back[0], (uint32_t)prm.ncx);
                const int cy = (int)__umulhi(pa.y - prm.back[1], (uint32_t)prm.ncy);
                const int cz = DIM == 3 ? (int)__umulhi(pa.z - prm.back[2], (uint32_t)prm.ncz) : 0;
                unsigned c = 0u;
                const float rate = rate_direct<DIM, KERNEL, true, COUNT>(Pe, cs + prm.coff, pa, cx, cy, cz, prm, c);
                cnt += c;
                Acc acc{0.f, 0.f, 0.f, 0.f, 0u};
                epilogue<DIM, EPI>(gi, rate, pa, perm, prm, o, acc);
            }
        }
        __syncwarp();   // the warp's slot may be rewritten by its next item
    }
    if (COUNT) {
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out.pairs, (unsigned long long)cnt);
    }
}

template <int DIM, int KERNEL, bool COUNT, bool PAIRED>
void launch_batch_epi(int epi, int grid, const uint4 *Pe, const uint32_t *cs, const uint32_t *perm,
                      const RateParams *descs, const BatchTile *tiles, int ntiles, unsigned *queue,
                      const EpiOut &out, cudaStream_t s)
{
    switch (epi) {
    case EPI_RATE:
        k_rate_batch<DIM, KERNEL, EPI_RATE, COUNT, PAIRED><<<grid, kRateThreads, 0, s>>>(Pe, cs, perm, descs, tiles, ntiles, queue, out);
        break;
    case EPI_PREDICT:
        k_rate_batch<DIM, KERNEL, EPI_PREDICT, COUNT, PAIRED><<<grid, kRateThreads, 0, s>>>(Pe, cs, perm, descs, tiles, ntiles, queue, out);
        break;
    default:
        k_rate_batch<DIM, KERNEL, EPI_CORRECT, COUNT, PAIRED><<<grid, kRateThreads, 0, s>>>(Pe, cs, perm, descs, tiles, ntiles, queue, out);
        break;
    }
}

template <int DIM, int KERNEL>
void launch_batch_k(bool count, bool paired, int epi, int grid, const uint4 *Pe, const uint32_t *cs,
                    const uint32_t *perm, const RateParams *descs, const BatchTile *tiles, int ntiles,
                    unsigned *queue, const EpiOut &out, cudaStream_t s)
{
    if (count)
        launch_batch_epi<DIM, KERNEL, true, false>(epi, grid, Pe, cs, perm, descs, tiles, ntiles, queue, out, s);
    else if (paired)
        launch_batch_epi<DIM, KERNEL, false, true>(epi, grid, Pe, cs, perm, descs, tiles, ntiles, queue, out, s);
    else
        launch_batch_epi<DIM, KERNEL, false, false>(epi, grid, Pe, cs, perm, descs, tiles, ntiles, queue, out, s);
}

// ---------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------
template <int DIM, int KERNEL, int EPI, bool COUNT>
cudaError_t launch_variant(bool iso, const uint4 *Pe, const uint4 *Pc, const uint32_t *cs,
                           const uint32_t *perm, const RateParams &prm, const EpiOut &out, cudaStream_t s)
{
    if (prm.variant == 1 && iso) {
        const int blocks = prm.ntx * prm.nty * (DIM == 3 ? prm.ntz : 1);
        const size_t smem = tiled_smem_bytes(DIM, prm);
        auto fn = k_rate_tiled<DIM, KERNEL, EPI, COUNT>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        return launch_pdl(fn, blocks, kTileThreads, smem, s, Pe, Pc, cs, perm, prm, out);
    }
    if (prm.variant >= 5 && prm.variant <= 8 && !COUNT)   // paired walks (rate_pair.cu)
        return launch_rate_pair(DIM, KERNEL, EPI, iso, Pe, Pc, cs, perm, prm, out, s);
    const int blocks = rate_blocks(prm.n);
    // 2, 4 (and 7, 8 when counting pairs): branched direct walk
    const bool bf = prm.variant != 2 && prm.variant != 4 && prm.variant != 7 && prm.variant != 8;
    // 3, 4: trimmed rows (square or cubic boxes; the pair count is the same either way)
    const bool trim = (prm.variant == 3 || prm.variant == 4) && iso && !COUNT;
    if (iso) {
        if (trim) {
            if (bf)
                return launch_pdl(k_rate<DIM, KERNEL, EPI, true, false, true, true>, blocks, kRateThreads, 0, s, Pe, Pc, cs, perm, prm, out);
            else
                return launch_pdl(k_rate<DIM, KERNEL, EPI, true, false, false, true>, blocks, kRateThreads, 0, s, Pe, Pc, cs, perm, prm, out);
        } else if (bf) {
            return launch_pdl(k_rate<DIM, KERNEL, EPI, true, COUNT, true, false>, blocks, kRateThreads, 0, s, Pe, Pc, cs, perm, prm, out);
        } else {
            return launch_pdl(k_rate<DIM, KERNEL, EPI, true, COUNT, false, false>, blocks, kRateThreads, 0, s, Pe, Pc, cs, perm, prm, out);
        }
    } else {
        if (bf)
            return launch_pdl(k_rate<DIM, KERNEL, EPI, false, COUNT, true, false>, blocks, kRateThreads, 0, s, Pe, Pc, cs, perm, prm, out);
        else
            return launch_pdl(k_rate<DIM, KERNEL, EPI, false, COUNT, false, false>, blocks, kRateThreads, 0, s, Pe, Pc, cs, perm, prm, out);
    }
    return cudaGetLastError();
}

template <int DIM, int KERNEL, bool COUNT>
cudaError_t launch_epi(int epi, bool iso, const uint4 *Pe, const uint4 *Pc, const uint32_t *cs,
                       const uint32_t *perm, const RateParams &prm, const EpiOut &out, cudaStream_t s)
{
    switch (epi) {
    case EPI_RATE: return launch_variant<DIM, KERNEL, EPI_RATE, COUNT>(iso, Pe, Pc, cs, perm, prm, out, s);
    case EPI_PREDICT: return launch_variant<DIM, KERNEL, EPI_PREDICT, COUNT>(iso, Pe, Pc, cs, perm, prm, out, s);
    default: return launch_variant<DIM, KERNEL, EPI_CORRECT, COUNT>(iso, Pe, Pc, cs, perm, prm, out, s);
    }
}

template <int DIM, int KERNEL>
cudaError_t launch_dk(bool iso, bool count, int epi, const uint4 *Pe, const uint4 *Pc,
                      const uint32_t *cs, const uint32_t *perm, const RateParams &prm,
                      const EpiOut &out, cudaStream_t s)
{
    return count ? launch_epi<DIM, KERNEL, true>(epi, iso, Pe, Pc, cs, perm, prm, out, s)
                 : launch_epi<DIM, KERNEL, false>(epi, iso, Pe, Pc, cs, perm, prm, out, s);
}

}  // namespace

int rate_blocks(int n) { return (n + kRateThreads - 1) / kRateThreads; }

int rate_launch_blocks(int dim, const RateParams &prm, bool iso)
{
    if (prm.variant == 1 && iso) return prm.ntx * prm.nty * (dim == 3 ? prm.ntz : 1);
    if (prm.variant >= 5 && prm.variant <= 8) return rate_blocks((prm.n + 1) / 2);
    return rate_blocks(prm.n);
}

int rate_launch_warps(int dim, const RateParams &prm, bool iso)
{
    if (prm.variant == 1 && iso) return rate_launch_blocks(dim, prm, iso) * (kTileThreads / 32);
    return rate_launch_blocks(dim, prm, iso) * (kRateThreads / 32);
}

size_t tiled_smem_bytes(int dim, const RateParams &prm)
{
    const int k = prm.k;
    const int HX = prm.tx + 2 * k, HY = prm.ty + 2 * k, HZ = dim == 3 ? prm.tz + 2 * k : 1;
    const int tr = prm.ty * (dim == 3 ? prm.tz : 1);
    return (size_t)prm.cap * 16 + (size_t)HY * HZ * (HX + 1) * 4 + (size_t)3 * (tr + 1) * 4;
}

cudaError_t launch_rate_batch(int dim, int kernel, int epi, const uint4 *Pe, const uint32_t *cell_start,
                              const uint32_t *perm, const RateParams *descs, const BatchTile *tiles,
                              int ntiles, unsigned *queue, int grid, const EpiOut &out, cudaStream_t s,
                              bool paired)
{
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned), s);
    if (e != cudaSuccess || ntiles == 0) return e;
    const bool count = out.pairs != nullptr;
    if (dim == 2) {
        if (kernel == ADE_WENDLAND_C2)
            launch_batch_k<2, ADE_WENDLAND_C2>(count, paired, epi, grid, Pe, cell_start, perm, descs, tiles, ntiles, queue, out, s);
        else
            launch_batch_k<2, ADE_WENDLAND_C4>(count, paired, epi, grid, Pe, cell_start, perm, descs, tiles, ntiles, queue, out, s);
    } else {
        if (kernel == ADE_WENDLAND_C2)
            launch_batch_k<3, ADE_WENDLAND_C2>(count, paired, epi, grid, Pe, cell_start, perm, descs, tiles, ntiles, queue, out, s);
        else
            launch_batch_k<3, ADE_WENDLAND_C4>(count, paired, epi, grid, Pe, cell_start, perm, descs, tiles, ntiles, queue, out, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_rate(int dim, int kernel, bool iso, int epi, const uint4 *Pe, const uint4 *Pc,
                        const uint32_t *cell_start, const uint32_t *perm, const RateParams &prm,
                        const EpiOut &out, cudaStream_t s)
{
    if (prm.n == 0) return cudaSuccess;
    const bool count = out.pairs != nullptr;
    if (dim == 2)
        return kernel == ADE_WENDLAND_C2
                   ? launch_dk<2, ADE_WENDLAND_C2>(iso, count, epi, Pe, Pc, cell_start, perm, prm, out, s)
                   : launch_dk<2, ADE_WENDLAND_C4>(iso, count, epi, Pe, Pc, cell_start, perm, prm, out, s);
    return kernel == ADE_WENDLAND_C2
               ? launch_dk<3, ADE_WENDLAND_C2>(iso, count, epi, Pe, Pc, cell_start, perm, prm, out, s)
               : launch_dk<3, ADE_WENDLAND_C4>(iso, count, epi, Pe, Pc, cell_start, perm, prm, out, s);
}

}  // namespace ade
