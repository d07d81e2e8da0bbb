// rate.cu -- the neighbour-interaction kernel: Eq. 4-5 (Sec. 2.2) for every particle, with the
// predictor and corrector of Eq. 8-9 (Sec. 2.4) fused into its epilogue.
//
// For a uniform velocity field (Sec. 3) every particle carries the same tensor D (Eq. 3), so the
// per-component harmonic mean of Eq. 5 is 4 D D / (D + D) = 2 D and the pair factor reduces to
//     Dcal_ab = Gamma x_ab^T K x_ab / r^2 - tr K,   K = 2 D,
// evaluated as x^T (Gamma K - Gamma K_last I) x / r^2 + (Gamma K_last - tr K), K_last = K_yy in
// 2D and K_zz in 3D, which drops one diagonal term from the per-pair work.
// With grad_a W = W'(r) x_ab / r, the dispersive term of Eq. 4 for one ordered pair is
//     1/2 (m_b / rhobar) Dcal_ab (C_a - C_b) W'(r) / r,
// and W'(r)/r = kc f(q): Wendland C2 (support H = 2h): f = (1-q)^3, kc = -20 B / H^2;
// Wendland C4 (Eq. 7, support H = h): f = (1-q)^5 (1+5q), kc = -(56/3) B / H^2.
// The convective term of Eq. 4 is identically zero for uniform v and is not evaluated.
//
// Two variants share the pair arithmetic and the epilogue:
//   * direct: one thread per cell-sorted particle; candidates are read from the sorted copy in
//     global memory (L1-cached 16-byte words {x, y, z, C}); separations are int32 differences of
//     fixed-point words converted to FP32 for every pair; each stencil row (2w+1 cells with
//     consecutive keys) is one contiguous index range, two at a periodic seam.
//   * tiled: one CTA per block of TX x TY (x TZ) cells.  The CTA stages every particle of the
//     block and its k-cell halo into shared memory once, as int32 fixed-point offsets from the
//     block centre (the minimum image from the centre), plus a local cell start table.  Each
//     thread then walks its targets' stencil rows over shared memory; the pair separation is the
//     exact int32 difference converted to FP32, as in the direct walk, so both variants round
//     relative to the separation itself rather than to the block size.  The pair term is
//     evaluated without a branch: outside the support (1 - q) is clamped to 0, so the term
//     vanishes.  A block whose halo does not fit the staging buffer falls back to the direct walk.
// Both variants sum each stencil row's terms in FP32 and add the row sums with Neumaier's
// compensated summation, visiting rows and, inside a row, particles in sorted order, so results
// are deterministic and independent of the tiling.
#include "ade_internal.h"

namespace ade {

namespace {

#include "rate_common.cuh"

// In-support test of the pair counter, taken in FP64 with the operation order of a plain FP64
// evaluation (d_i = int difference x unit, r^2 = (d_x^2 + d_y^2) + d_z^2, no fused multiply-add),
// so the integer count does not depend on FP32 rounding at |x_ab| = H.
template <int DIM>
__device__ __forceinline__ unsigned in_support_fp64(int ix, int iy, int iz, const RateParams &prm)
{
    const double dx = (double)ix * prm.u[0], dy = (double)iy * prm.u[1];
    double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    if (DIM == 3) {
        const double dz = (double)iz * prm.u[2];
        r2 = __dadd_rn(r2, __dmul_rn(dz, dz));
    }
    return (r2 > 0.0 && r2 < prm.H2d) ? 1u : 0u;
}

// Per-pair constants, copied into registers once per particle (the parameter block may live in
// shared or constant memory).
struct PairConst {
    float H2, invH, sy, sz, c0;
    float K0, K1, K3, K4, K5;
    template <class P>
    __device__ __forceinline__ explicit PairConst(const P &prm)
        : H2(prm.H2), invH(prm.invH), sy(prm.sy), sz(prm.sz), c0(prm.c0), K0(prm.Kc[0]),
          K1(prm.Kc[1]), K3(prm.Kc[3]), K4(prm.Kc[4]), K5(prm.Kc[5])
    {
    }
};

// Dcal factor of the pair (without the kernel shape): x^T Kc x / r^2 + c0.
template <int DIM>
__device__ __forceinline__ float dcal(float dx, float dy, float dz, float rinv2, const PairConst &k)
{
    float Q;
    if (DIM == 2) {
        Q = dx * fmaf(k.K0, dx, k.K3 * dy);
    } else {
        float qx = fmaf(k.K0, dx, fmaf(k.K3, dy, k.K4 * dz));
        float qy = fmaf(k.K1, dy, k.K5 * dz);
        Q = fmaf(dx, qx, dy * qy);
    }
    return fmaf(Q, rinv2, k.c0);
}

// ---------------------------------------------------------------------------------------------
// direct walk over global memory
// ---------------------------------------------------------------------------------------------
// One candidate range of the direct walk.  The evaluation is branch-free: outside the support
// (1 - q) is clamped to 0, so the term is exactly 0; at zero separation (the particle itself, or a
// coincident particle) rsqrt(0) = inf makes q and s NaN, and IEEE max-num (fmaxf returns the
// non-NaN operand) turns them into (1 - q) = 0 and s = -FLT_MAX, so the weight is exactly 0 as
// well.  In-support terms use the same operations as a branched evaluation, so adding the zero
// terms leaves the sum unchanged.  The pair counter keeps an explicit FP64 test.
// BF = false keeps the branch on r^2 < H^2 instead: a warp whose lanes all miss skips the term,
// which pays off when warps are spatially coherent and the stencil is large (3D).
// ZS = false drops the clamp of s: zero separation occurs only within the particle's own cell, so
// rows other than the particle's own cell row (dy = dz = 0) never meet it, s is finite there and
// the clamp changes nothing.
template <int DIM, int KERNEL, bool ISO, bool COUNT, bool BF, bool ZS = true>
__device__ __forceinline__ void pair_range_direct(const uint4 *__restrict__ P, int j0, int j1,
                                                  const uint4 &pa, float Ca, const PairConst &k,
                                                  const RateParams &prm, float &rs, unsigned &cnt)
{
#pragma unroll 8
    for (int j = j0; j < j1; ++j) {
        const uint4 pb = __ldg(P + j);
        if (COUNT) cnt += in_support_fp64<DIM>((int)(pa.x - pb.x), (int)(pa.y - pb.y), (int)(pa.z - pb.z), prm);
        float dx = (float)(int)(pa.x - pb.x);
        float dy = (float)(int)(pa.y - pb.y);
        float dz = 0.f;
        if (DIM == 3) dz = (float)(int)(pa.z - pb.z);
        if (!ISO) {
            dy *= k.sy;
            if (DIM == 3) dz *= k.sz;
        }
        float r2 = fmaf(dx, dx, dy * dy);
        if (DIM == 3) r2 = fmaf(dz, dz, r2);
        if (BF) {
            const float rinv = rsqrtf(r2);
            const float omq = fmaxf(fmaf(-(r2 * rinv), k.invH, 1.f), 0.f);
            const float sr = dcal<DIM>(dx, dy, dz, rinv * rinv, k);
            const float s = ZS ? fmaxf(sr, -3.402823466e38f) : sr;
            rs = fmaf(shape<KERNEL>(omq) * s, Ca - __uint_as_float(pb.w), rs);
        } else if (r2 < k.H2 && r2 > 0.f) {
            const float rinv = rsqrtf(r2);
            const float omq = fmaf(-(r2 * rinv), k.invH, 1.f);
            const float s = dcal<DIM>(dx, dy, dz, rinv * rinv, k);
            rs = fmaf(shape<KERNEL>(omq) * s, Ca - __uint_as_float(pb.w), rs);
        }
    }
}

// Eq. 4 at one particle by the direct walk; (cx, cy, cz) is its cell.  TRIM: visit only the
// stencil cells within reach of the particle itself (see below).
template <int DIM, int KERNEL, bool ISO, bool COUNT, bool BF = true, bool TRIM = false>
__device__ float rate_direct(const uint4 *__restrict__ Pe, const uint32_t *__restrict__ cs,
                             const uint4 &pa, int cx, int cy, int cz, const RateParams &prm,
                             unsigned &cnt)
{
    const int ncx = prm.ncx, ncy = prm.ncy, ncz = prm.ncz, nrows = prm.nrows;
    const PairConst kc(prm);
    const float Ca = __uint_as_float(pa.w);
    float acc = 0.f, comp = 0.f;
    // Per-particle trimming of the stencil (TRIM).  The stencil row (dy, dz, w) holds every
    // neighbour of any point of the cell; for this particle only the cells within H of its own
    // position are
    // needed.  Its fractional position in its build cell is the low word of x nc (umulhi gives the
    // cell, the low 32 bits the offset within it exactly), so the row's distance e (in x-axis
    // units) and the x cell range [floor(f_x - xe), floor(f_x + xe)], xe = sqrt(H^2 - e^2) / width,
    // follow in FP32.  The radius is widened by 2^-12 H (far above the FP32 rounding of these
    // bounds), so a skipped candidate lies beyond H by more than the evaluation's rounding and its
    // term is exactly 0: the sums are bitwise those of the full stencil.
    const float two32 = 4294967296.f;
    const float fx = (float)((pa.x - prm.back[0]) * (uint32_t)ncx) * (1.f / two32);
    const float fy = (float)((pa.y - prm.back[1]) * (uint32_t)ncy) * (1.f / two32);
    const float fz = DIM == 3 ? (float)((pa.z - prm.back[2]) * (uint32_t)ncz) * (1.f / two32) : 0.f;
    const float inv_wx = (float)ncx * (1.f / two32);              // cells per x unit
    const float chy = two32 / (float)ncy * kc.sy, chz = DIM == 3 ? two32 / (float)ncz * kc.sz : 0.f;
    const float Hm2 = kc.H2 * (1.f + 1.f / 2048.f);                // (H (1 + 2^-12))^2, rounded up
    for (int ri = 0; ri < nrows; ++ri) {
        const StencilRow row = prm.rows[ri];
        float e2 = 0.f;
        if (TRIM) {
            const float ey = fmaxf(fmaxf((float)row.dy - fy, fy - (float)(row.dy + 1)), 0.f) * chy;
            e2 = ey * ey;
            if (DIM == 3) {
                const float ez = fmaxf(fmaxf((float)row.dz - fz, fz - (float)(row.dz + 1)), 0.f) * chz;
                e2 = fmaf(ez, ez, e2);
            }
        }
        int dlo = -(int)row.w, dhi = row.w;
        if (TRIM) {
            if (!(e2 < Hm2)) continue;                              // the whole row is out of reach
            const float t = Hm2 - e2;
            const float xe = t * rsqrtf(t) * inv_wx + 1.f / 4096.f;  // half-extent in cells
            dlo = max(__float2int_rd(fx - xe), dlo);
            dhi = min(__float2int_rd(fx + xe), dhi);
        }
        int yy = cy + row.dy;
        yy += (yy < 0) ? ncy : 0;
        yy -= (yy >= ncy) ? ncy : 0;
        int zz = 0;
        if (DIM == 3) {
            zz = cz + row.dz;
            zz += (zz < 0) ? ncz : 0;
            zz -= (zz >= ncz) ? ncz : 0;
        }
        const int base = (zz * ncy + yy) * ncx;
        const int lo = cx + dlo, hi = cx + dhi + 1;
        int s0, e0, s1 = 0, e1 = 0;
        if (lo < 0) {
            s0 = __ldg(cs + base + lo + ncx);
            e0 = __ldg(cs + base + ncx);
            s1 = __ldg(cs + base);
            e1 = __ldg(cs + base + hi);
        } else if (hi > ncx) {
            s0 = __ldg(cs + base + lo);
            e0 = __ldg(cs + base + ncx);
            s1 = __ldg(cs + base);
            e1 = __ldg(cs + base + hi - ncx);
        } else {
            s0 = __ldg(cs + base + lo);
            e0 = __ldg(cs + base + hi);
        }
        float rs = 0.f;
        if (row.dy == 0 && (DIM == 2 || row.dz == 0)) {      // the particle's own cell row
            pair_range_direct<DIM, KERNEL, ISO, COUNT, BF, true>(Pe, s0, e0, pa, Ca, kc, prm, rs, cnt);
            pair_range_direct<DIM, KERNEL, ISO, COUNT, BF, true>(Pe, s1, e1, pa, Ca, kc, prm, rs, cnt);
        } else {
            pair_range_direct<DIM, KERNEL, ISO, COUNT, BF, false>(Pe, s0, e0, pa, Ca, kc, prm, rs, cnt);
            pair_range_direct<DIM, KERNEL, ISO, COUNT, BF, false>(Pe, s1, e1, pa, Ca, kc, prm, rs, cnt);
        }
        neumaier_add(acc, comp, rs);
    }
    return prm.pf * (acc + comp);
}

// ---------------------------------------------------------------------------------------------
// paired direct walk: two targets per thread, packed FP32x2 arithmetic
// ---------------------------------------------------------------------------------------------
// Two cell-sorted particles a0, a1 of the same cell row (cx1 - cx0 <= 1) walk one candidate stream:
// per stencil row the union of their cell ranges.  Every candidate is loaded once and both terms
// are evaluated with the packed FP32x2 instructions of this architecture (one instruction, two
// independent IEEE results), each half with exactly the operations of pair_range_direct<BF>.  A
// candidate outside one target's own range lies beyond H (1 + 2^-12) of it -- the stencil rows and
// the trimmed ranges are built for that radius -- so its branch-free term is exactly 0 and each
// target's row sum is bitwise that of the one-target walk (same candidates, same order).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

template <int KERNEL>
__device__ __forceinline__ float2 shape2(float2 omq)
{
    if (KERNEL == ADE_WENDLAND_C2) return __fmul2_rn(__fmul2_rn(omq, omq), omq);
    const float2 o2 = __fmul2_rn(omq, omq);
    const float2 t = __ffma2_rn(f2(-5.f, -5.f), omq, f2(6.f, 6.f));
    return __fmul2_rn(__fmul2_rn(__fmul2_rn(o2, o2), omq), t);
}

// Packed per-pair constants (both halves equal).
struct PairConst2 {
    float2 K0, K1, K3, K4, K5, c0, ninvH, sy, sz;
    __device__ __forceinline__ explicit PairConst2(const PairConst &k)
        : K0(f2(k.K0, k.K0)), K1(f2(k.K1, k.K1)), K3(f2(k.K3, k.K3)), K4(f2(k.K4, k.K4)),
          K5(f2(k.K5, k.K5)), c0(f2(k.c0, k.c0)), ninvH(f2(-k.invH, -k.invH)), sy(f2(k.sy, k.sy)),
          sz(f2(k.sz, k.sz))
    {
    }
};

template <int DIM, int KERNEL, bool ISO, bool ZS>
__device__ __forceinline__ void pair_range_direct2(const uint4 *__restrict__ P, int j0, int j1,
                                                   const uint4 &pa0, const uint4 &pa1, float2 Ca,
                                                   const PairConst2 &k, float2 &rs)
{
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
        const uint4 pb = __ldg(P + j);
        float2 dx = f2((float)(int)(pa0.x - pb.x), (float)(int)(pa1.x - pb.x));
        float2 dy = f2((float)(int)(pa0.y - pb.y), (float)(int)(pa1.y - pb.y));
        float2 dz = f2(0.f, 0.f);
        if (DIM == 3) dz = f2((float)(int)(pa0.z - pb.z), (float)(int)(pa1.z - pb.z));
        if (!ISO) {
            dy = __fmul2_rn(dy, k.sy);
            if (DIM == 3) dz = __fmul2_rn(dz, k.sz);
        }
        float2 r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
        if (DIM == 3) r2 = __ffma2_rn(dz, dz, r2);
        const float2 rinv = f2(rsqrtf(r2.x), rsqrtf(r2.y));
        const float2 om = __ffma2_rn(__fmul2_rn(r2, rinv), k.ninvH, f2(1.f, 1.f));
        const float2 omq = f2(fmaxf(om.x, 0.f), fmaxf(om.y, 0.f));
        float2 Q;
        if (DIM == 2) {
            Q = __fmul2_rn(dx, __ffma2_rn(k.K0, dx, __fmul2_rn(k.K3, dy)));
        } else {
            const float2 qx = __ffma2_rn(k.K0, dx, __ffma2_rn(k.K3, dy, __fmul2_rn(k.K4, dz)));
            const float2 qy = __ffma2_rn(k.K1, dy, __fmul2_rn(k.K5, dz));
            Q = __ffma2_rn(dx, qx, __fmul2_rn(dy, qy));
        }
        const float2 sr = __ffma2_rn(Q, __fmul2_rn(rinv, rinv), k.c0);
        const float2 sc = ZS ? f2(fmaxf(sr.x, -3.402823466e38f), fmaxf(sr.y, -3.402823466e38f)) : sr;
        const float nCb = -__uint_as_float(pb.w);
        rs = __ffma2_rn(__fmul2_rn(shape2<KERNEL>(omq), sc), __fadd2_rn(Ca, f2(nCb, nCb)), rs);
    }
}

// Eq. 4 at two particles of the same cell row by the paired walk; (cx0, cx1, cy, cz) their cells.
template <int DIM, int KERNEL, bool ISO, bool TRIM>
__device__ void rate_direct_pair(const uint4 *__restrict__ Pe, const uint32_t *__restrict__ cs,
                                 const uint4 &pa0, const uint4 &pa1, int cx0, int cx1, int cy, int cz,
                                 const RateParams &prm, float &r0, float &r1)
{
    const int ncx = prm.ncx, ncy = prm.ncy, ncz = prm.ncz, nrows = prm.nrows;
    const PairConst kc(prm);
    const PairConst2 k2(kc);
    const float2 Ca = f2(__uint_as_float(pa0.w), __uint_as_float(pa1.w));
    float acc0 = 0.f, comp0 = 0.f, acc1 = 0.f, comp1 = 0.f;
    // the trimming of rate_direct, per target
    const float two32 = 4294967296.f;
    const float fx0 = (float)((pa0.x - prm.back[0]) * (uint32_t)ncx) * (1.f / two32);
    const float fx1 = (float)((pa1.x - prm.back[0]) * (uint32_t)ncx) * (1.f / two32);
    const float fy0 = (float)((pa0.y - prm.back[1]) * (uint32_t)ncy) * (1.f / two32);
    const float fy1 = (float)((pa1.y - prm.back[1]) * (uint32_t)ncy) * (1.f / two32);
    const float fz0 = DIM == 3 ? (float)((pa0.z - prm.back[2]) * (uint32_t)ncz) * (1.f / two32) : 0.f;
    const float fz1 = DIM == 3 ? (float)((pa1.z - prm.back[2]) * (uint32_t)ncz) * (1.f / two32) : 0.f;
    const float inv_wx = (float)ncx * (1.f / two32);
    const float chy = two32 / (float)ncy * kc.sy, chz = DIM == 3 ? two32 / (float)ncz * kc.sz : 0.f;
    const float Hm2 = kc.H2 * (1.f + 1.f / 2048.f);
    for (int ri = 0; ri < nrows; ++ri) {
        const StencilRow row = prm.rows[ri];
        int lo0 = cx0 - (int)row.w, hi0 = cx0 + row.w, lo1 = cx1 - (int)row.w, hi1 = cx1 + row.w;
        bool in0 = true, in1 = true;       // the target reaches the row (rate_direct does not skip it)
        bool ne0 = true, ne1 = true;       // ... and its cell range is not empty
        if (TRIM) {
            float e0 = fmaxf(fmaxf((float)row.dy - fy0, fy0 - (float)(row.dy + 1)), 0.f) * chy;
            float e1 = fmaxf(fmaxf((float)row.dy - fy1, fy1 - (float)(row.dy + 1)), 0.f) * chy;
            e0 *= e0;
            e1 *= e1;
            if (DIM == 3) {
                const float z0 = fmaxf(fmaxf((float)row.dz - fz0, fz0 - (float)(row.dz + 1)), 0.f) * chz;
                const float z1 = fmaxf(fmaxf((float)row.dz - fz1, fz1 - (float)(row.dz + 1)), 0.f) * chz;
                e0 = fmaf(z0, z0, e0);
                e1 = fmaf(z1, z1, e1);
            }
            in0 = e0 < Hm2;
            in1 = e1 < Hm2;
            const float t0 = in0 ? Hm2 - e0 : 1.f, t1 = in1 ? Hm2 - e1 : 1.f;
            const float xe0 = t0 * rsqrtf(t0) * inv_wx + 1.f / 4096.f;
            const float xe1 = t1 * rsqrtf(t1) * inv_wx + 1.f / 4096.f;
            lo0 = cx0 + max(__float2int_rd(fx0 - xe0), -(int)row.w);
            hi0 = cx0 + min(__float2int_rd(fx0 + xe0), (int)row.w);
            lo1 = cx1 + max(__float2int_rd(fx1 - xe1), -(int)row.w);
            hi1 = cx1 + min(__float2int_rd(fx1 + xe1), (int)row.w);
            ne0 = in0 && lo0 <= hi0;
            ne1 = in1 && lo1 <= hi1;
        }
        int lo, hi;
        if (ne0 && ne1) {
            lo = min(lo0, lo1);
            hi = max(hi0, hi1) + 1;
        } else if (ne0) {
            lo = lo0;
            hi = hi0 + 1;
        } else if (ne1) {
            lo = lo1;
            hi = hi1 + 1;
        } else {
            // no candidate for either target; a reached row still adds its (zero) row sum
            if (in0) neumaier_add(acc0, comp0, 0.f);
            if (in1) neumaier_add(acc1, comp1, 0.f);
            continue;
        }
        int yy = cy + row.dy;
        yy += (yy < 0) ? ncy : 0;
        yy -= (yy >= ncy) ? ncy : 0;
        int zz = 0;
        if (DIM == 3) {
            zz = cz + row.dz;
            zz += (zz < 0) ? ncz : 0;
            zz -= (zz >= ncz) ? ncz : 0;
        }
        const int base = (zz * ncy + yy) * ncx;
        int s0, e0, s1 = 0, e1 = 0;
        if (lo < 0) {
            s0 = __ldg(cs + base + lo + ncx);
            e0 = __ldg(cs + base + ncx);
            s1 = __ldg(cs + base);
            e1 = __ldg(cs + base + hi);
        } else if (hi > ncx) {
            s0 = __ldg(cs + base + lo);
            e0 = __ldg(cs + base + ncx);
            s1 = __ldg(cs + base);
            e1 = __ldg(cs + base + hi - ncx);
        } else {
            s0 = __ldg(cs + base + lo);
            e0 = __ldg(cs + base + hi);
        }
        float2 rs = f2(0.f, 0.f);
        if (row.dy == 0 && (DIM == 2 || row.dz == 0)) {      // the targets' own cell row
            pair_range_direct2<DIM, KERNEL, ISO, true>(Pe, s0, e0, pa0, pa1, Ca, k2, rs);
            pair_range_direct2<DIM, KERNEL, ISO, true>(Pe, s1, e1, pa0, pa1, Ca, k2, rs);
        } else {
            pair_range_direct2<DIM, KERNEL, ISO, false>(Pe, s0, e0, pa0, pa1, Ca, k2, rs);
            pair_range_direct2<DIM, KERNEL, ISO, false>(Pe, s1, e1, pa0, pa1, Ca, k2, rs);
        }
        // a target that does not reach the row (trimmed walk) skips it, as rate_direct does
        if (in0) neumaier_add(acc0, comp0, rs.x);
        if (in1) neumaier_add(acc1, comp1, rs.y);
    }
    r0 = prm.pf * (acc0 + comp0);
    r1 = prm.pf * (acc1 + comp1);
}

// ---------------------------------------------------------------------------------------------
// epilogue and block reductions
// ---------------------------------------------------------------------------------------------
// Writes of one particle at sorted position gi; pe = evaluation state {x, y, z, C}.
// PRE (corrector): the caller index a_pre = perm[gi] and C^l = C[a_pre] were loaded before the
// pair loop, so their latency hides behind it.
template <int DIM, int EPI, bool PRE = false>
__device__ __forceinline__ void epilogue(int gi, float rate, const uint4 &pe,
                                         const uint32_t *__restrict__ perm, const RateParams &prm,
                                         const EpiOut &out, Acc &acc, uint32_t a_pre = 0u,
                                         float C_pre = 0.f)
{
    if (EPI == EPI_RATE) {
        if (out.rate) {
            const uint32_t a = __ldg(perm + gi);
            if (a - (uint32_t)prm.goff < (uint32_t)prm.n) out.rate[a] = rate;
        }
    } else if (EPI == EPI_PREDICT) {
        // C^{l+1/2} = C^l + dt/2 r^l, x^{l+1/2} = x^l + dt/2 v.  Eq. 14 (out.Q set): the flux
        // Q = dC/dt relaxes to r over tau, C^{l+1/2} = C^l + dt/2 Q^l and
        // Q^{l+1/2} = Q^l + dt/2 (r^l - Q^l) / tau, kept in sorted order for the corrector.
        float dC = rate;
        if (out.Q) {
            const uint32_t a = __ldg(perm + gi);
            const float q = a - (uint32_t)prm.goff < (uint32_t)prm.n ? out.Q[a] : 0.f;
            out.Qh[gi] = fmaf(prm.dt, (rate - q) * out.tau_inv, q);
            dC = q;
        }
        uint4 q;
        q.x = pe.x + prm.inc[0];
        q.y = pe.y + prm.inc[1];
        q.z = pe.z + prm.inc[2];
        q.w = __float_as_uint(fmaf(prm.dt, dC, __uint_as_float(pe.w)));
        out.Pout[gi] = q;
    } else {
        // C^{l+1} = C^l + dt r^{l+1/2}, x^{l+1} = x^l + dt v, in the caller's order.  x^l is the
        // evaluation position minus the half-step drift (exact in fixed point); C^l is still in
        // the caller's array, read just before this thread overwrites it.  Eq. 14:
        // C^{l+1} = C^l + dt Q^{l+1/2}, Q^{l+1} = Q^l + dt (r^{l+1/2} - Q^{l+1/2}) / tau.
        const uint32_t a = PRE ? a_pre : __ldg(perm + gi);
        float Cn = 0.f;
        if (a - (uint32_t)prm.goff < (uint32_t)prm.n) {
            float dC = rate;
            if (out.Q) {
                const float qh = out.Qh[gi];
                const float q = out.Q[a];
                out.Q[a] = fmaf(prm.dt, (rate - qh) * out.tau_inv, q);
                dC = qh;
            }
            Cn = fmaf(prm.dt, dC, PRE ? C_pre : out.C[a]);
            out.C[a] = Cn;
            out.xq[a] = pe.x - prm.back[0] + prm.inc[0];
            out.xq[(size_t)prm.n + a] = pe.y - prm.back[1] + prm.inc[1];
            if (DIM == 3) out.xq[2 * (size_t)prm.n + a] = pe.z - prm.back[2] + prm.inc[2];
        }
        if (!isfinite(Cn)) atomicOr(out.status, 1);
        two_sum_add(acc.hi, acc.lo, Cn, 0.f);
        acc.mn = fminf(acc.mn, Cn);
        acc.mx = fmaxf(acc.mx, Cn);
    }
}

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
    const float rate = rate_direct<DIM, KERNEL, ISO, COUNT, BF, TRIM>(Pe, cs, pa, cx, cy, cz, prm, cnt);
    if (valid) {
        acc.cnt = cnt;
        epilogue<DIM, EPI, PRE>(i, rate, pa, perm, prm, out, acc, a_pre, C_pre);
    }
    warp_finish<EPI, COUNT, kRateThreads>(acc, out);
}

// Whether sorted particles a0, a1 (cells cx0 <= cx1 in row cy, cz) can share one candidate stream:
// the same cell row, at most one cell apart, and a grid wide enough that the union of their
// ranges (<= 2 kMaxSubdiv + 2 cells) never wraps onto itself.
__device__ __forceinline__ bool can_pair(int cx0, int cy0, int cz0, int cx1, int cy1, int cz1, int ncx)
{
    return cy0 == cy1 && cz0 == cz1 && cx1 - cx0 <= 1 && ncx >= 2 * kMaxSubdiv + 2;
}

// Paired kernel: thread t evaluates sorted particles 2t and 2t + 1; a pair that cannot share a
// candidate stream (can_pair) takes the one-target walk for each particle.  The full-row
// walk is held to 10 resident CTAs per SM (<= 48 registers), which measured faster on the 1024^2
// ladder; the trimmed walk measured faster without the limit.
template <int DIM, int KERNEL, int EPI, bool ISO, bool TRIM>
__global__ __launch_bounds__(kRateThreads, TRIM ? 0 : 10) void k_rate_pair(const uint4 *__restrict__ Pe,
                                                            const uint4 *__restrict__ Pc,
                                                            const uint32_t *__restrict__ cs,
                                                            const uint32_t *__restrict__ perm,
                                                            const RateParams prm, const EpiOut out)
{
    pdl_wait();   // no early trigger: see pdl_trigger
    const int t = blockIdx.x * kRateThreads + threadIdx.x;
    const int i0 = 2 * t, i1 = 2 * t + 1;
    const bool v0 = i0 < prm.n, v1 = i1 < prm.n;
    const int ii0 = v0 ? i0 : prm.n - 1, ii1 = v1 ? i1 : ii0;
    const uint4 pa0 = __ldg(Pe + ii0);
    const uint4 pa1 = __ldg(Pe + ii1);
    const int cx0 = (int)__umulhi(pa0.x - prm.back[0], (uint32_t)prm.ncx);
    const int cy0 = (int)__umulhi(pa0.y - prm.back[1], (uint32_t)prm.ncy);
    const int cz0 = DIM == 3 ? (int)__umulhi(pa0.z - prm.back[2], (uint32_t)prm.ncz) : 0;
    const int cx1 = (int)__umulhi(pa1.x - prm.back[0], (uint32_t)prm.ncx);
    const int cy1 = (int)__umulhi(pa1.y - prm.back[1], (uint32_t)prm.ncy);
    const int cz1 = DIM == 3 ? (int)__umulhi(pa1.z - prm.back[2], (uint32_t)prm.ncz) : 0;
    Acc acc{0.f, 0.f, __int_as_float(0x7f800000), __int_as_float(0xff800000), 0u};
    unsigned cnt = 0u;
    float r0, r1;
    const bool paired = v1 && can_pair(cx0, cy0, cz0, cx1, cy1, cz1, prm.ncx);
    if (paired) {
        rate_direct_pair<DIM, KERNEL, ISO, TRIM>(Pe, cs, pa0, pa1, cx0, cx1, cy0, cz0, prm, r0, r1);
    } else {
        r0 = rate_direct<DIM, KERNEL, ISO, false, true, TRIM>(Pe, cs, pa0, cx0, cy0, cz0, prm, cnt);
        r1 = v1 ? rate_direct<DIM, KERNEL, ISO, false, true, TRIM>(Pe, cs, pa1, cx1, cy1, cz1, prm, cnt) : 0.f;
    }
    if (v0) epilogue<DIM, EPI>(i0, r0, pa0, perm, prm, out, acc);
    if (v1) epilogue<DIM, EPI>(i1, r1, pa1, perm, prm, out, acc);
    warp_finish<EPI, false, kRateThreads>(acc, out);
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
                    const float rinv = rsqrtf(fmaxf(r2, 1.0f));
                    const float omq = fmaxf(fmaf(-r2 * rinv, kc.invH, 1.f), 0.f);
                    const float s = dcal<DIM>(dx, dy, dz, rinv * rinv, kc);
                    const float w = r2 > 0.f ? shape<KERNEL>(omq) * s : 0.f;
                    rs = fmaf(w, Ca - __int_as_float(q.w), rs);
                    if (COUNT) cnt += in_support_fp64<DIM>(a.x - q.x, a.y - q.y, a.z - q.z, prm);
                }
                neumaier_add(sum, comp, rs);
            }
            rate = prm.pf * (sum + comp);
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
// Every CTA takes work items from an atomic counter until the list is exhausted (no CTA waits on
// another).  An item is a range of one plume's cell-sorted particles; the plume's constants are
// copied to shared memory once per item and each particle is evaluated with the same code as the
// single-plume direct kernel (rate_direct + epilogue), so a plume gives bit-identical results
// whether it runs alone or in a batch.  Items are ordered by decreasing estimated cost.
template <int DIM, int KERNEL, int EPI, bool COUNT>
__global__ __launch_bounds__(kRateThreads) void k_rate_batch(const uint4 *__restrict__ Pe,
                                                             const uint32_t *__restrict__ cs,
                                                             const uint32_t *__restrict__ perm,
                                                             const RateParams *__restrict__ descs,
                                                             const BatchTile *__restrict__ tiles,
                                                             int ntiles, unsigned *queue,
                                                             const EpiOut out)
{
    __shared__ RateParams sp;
    __shared__ int s_item;
    constexpr int kWords = (int)(sizeof(RateParams) / sizeof(int));
    static_assert(sizeof(RateParams) % sizeof(int) == 0, "RateParams is copied word by word");
    int cur = -1;
    unsigned cnt = 0u;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= ntiles) break;
        const BatchTile t = tiles[item];
        if (t.plume != cur) {
            const int *src = reinterpret_cast<const int *>(descs + t.plume);
            int *dst = reinterpret_cast<int *>(&sp);
            for (int w = threadIdx.x; w < kWords; w += kRateThreads) dst[w] = __ldg(src + w);
            cur = t.plume;
        }
        __syncthreads();
        const RateParams &prm = sp;
        EpiOut o = out;
        if (EPI == EPI_CORRECT) o.xq = out.xq + (size_t)prm.goff * (DIM - 1);
        for (int k = threadIdx.x; k < t.count; k += kRateThreads) {
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
        __syncthreads();   // sp and s_item are rewritten by the next item
    }
    if (COUNT) {
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out.pairs, (unsigned long long)cnt);
    }
}

template <int DIM, int KERNEL, bool COUNT>
void launch_batch_epi(int epi, int grid, const uint4 *Pe, const uint32_t *cs, const uint32_t *perm,
                      const RateParams *descs, const BatchTile *tiles, int ntiles, unsigned *queue,
                      const EpiOut &out, cudaStream_t s)
{
    switch (epi) {
    case EPI_RATE:
        k_rate_batch<DIM, KERNEL, EPI_RATE, COUNT><<<grid, kRateThreads, 0, s>>>(Pe, cs, perm, descs, tiles, ntiles, queue, out);
        break;
    case EPI_PREDICT:
        k_rate_batch<DIM, KERNEL, EPI_PREDICT, COUNT><<<grid, kRateThreads, 0, s>>>(Pe, cs, perm, descs, tiles, ntiles, queue, out);
        break;
    default:
        k_rate_batch<DIM, KERNEL, EPI_CORRECT, COUNT><<<grid, kRateThreads, 0, s>>>(Pe, cs, perm, descs, tiles, ntiles, queue, out);
        break;
    }
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
    if ((prm.variant == 5 || prm.variant == 6) && !COUNT) {
        // 5, 6: paired branch-free walk (6: trimmed rows, square or cubic boxes); the pair counter
        // takes the one-target walk
        const int pblocks = rate_blocks((prm.n + 1) / 2);
        if (iso && prm.variant == 6)
            return launch_pdl(k_rate_pair<DIM, KERNEL, EPI, true, true>, pblocks, kRateThreads, 0, s, Pe, Pc, cs, perm, prm, out);
        if (iso)
            return launch_pdl(k_rate_pair<DIM, KERNEL, EPI, true, false>, pblocks, kRateThreads, 0, s, Pe, Pc, cs, perm, prm, out);
        return launch_pdl(k_rate_pair<DIM, KERNEL, EPI, false, false>, pblocks, kRateThreads, 0, s, Pe, Pc, cs, perm, prm, out);
    }
    const int blocks = rate_blocks(prm.n);
    const bool bf = prm.variant != 2 && prm.variant != 4;   // 2, 4: branched direct walk
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
    if (prm.variant == 5 || prm.variant == 6) return rate_blocks((prm.n + 1) / 2);
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
                              int ntiles, unsigned *queue, int grid, const EpiOut &out, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned), s);
    if (e != cudaSuccess || ntiles == 0) return e;
    const bool count = out.pairs != nullptr;
    if (dim == 2) {
        if (kernel == ADE_WENDLAND_C2)
            count ? launch_batch_epi<2, ADE_WENDLAND_C2, true>(epi, grid, Pe, cell_start, perm, descs, tiles, ntiles, queue, out, s)
                  : launch_batch_epi<2, ADE_WENDLAND_C2, false>(epi, grid, Pe, cell_start, perm, descs, tiles, ntiles, queue, out, s);
        else
            count ? launch_batch_epi<2, ADE_WENDLAND_C4, true>(epi, grid, Pe, cell_start, perm, descs, tiles, ntiles, queue, out, s)
                  : launch_batch_epi<2, ADE_WENDLAND_C4, false>(epi, grid, Pe, cell_start, perm, descs, tiles, ntiles, queue, out, s);
    } else {
        if (kernel == ADE_WENDLAND_C2)
            count ? launch_batch_epi<3, ADE_WENDLAND_C2, true>(epi, grid, Pe, cell_start, perm, descs, tiles, ntiles, queue, out, s)
                  : launch_batch_epi<3, ADE_WENDLAND_C2, false>(epi, grid, Pe, cell_start, perm, descs, tiles, ntiles, queue, out, s);
        else
            count ? launch_batch_epi<3, ADE_WENDLAND_C4, true>(epi, grid, Pe, cell_start, perm, descs, tiles, ntiles, queue, out, s)
                  : launch_batch_epi<3, ADE_WENDLAND_C4, false>(epi, grid, Pe, cell_start, perm, descs, tiles, ntiles, queue, out, s);
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
