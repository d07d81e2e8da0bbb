// rate_walk.cuh -- the direct candidate walks of the interaction kernels (rate.cu, rate_pair.cu):
// Eq. 4-5 at one particle (rate_direct) or at two adjacent cell-sorted particles sharing one
// candidate stream (rate_direct_pair), and the fused predictor / corrector epilogue of Eq. 8-9.
// Included inside an unnamed namespace of ade, after rate_common.cuh.
#pragma once

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
    float H2, invH, sy, sz;
    float w0, w1, w2, b;
    int m1;
    template <class P>
    __device__ __forceinline__ explicit PairConst(const P &prm)
        : H2(prm.H2), invH(prm.invH), sy(prm.sy), sz(prm.sz), w0(prm.uw[0]), w1(prm.uw[1]), w2(prm.uw[2]),
          b(prm.ub), m1(prm.m1)
    {
    }
};

// Pair factor of Eq. 5 up to the sign folded into upf: with uniform D (Eq. 3) the harmonic mean is
// K = 2D and Gamma e^T K e - tr K = a (vhat . e)^2 + b; here t = (sqrt|a| vhat . x) / r and the
// factor is t^2 + sign(a) b.  rinv = 1 / r.
template <int DIM>
__device__ __forceinline__ float dcal(float dx, float dy, float dz, float rinv, const PairConst &k)
{
    float u = fmaf(k.w0, dx, k.w1 * dy);
    if (DIM == 3) u = fmaf(k.w2, dz, u);
    const float t = u * rinv;
    return fmaf(t, t, k.b);
}

// ---------------------------------------------------------------------------------------------
// trimmed rows
// ---------------------------------------------------------------------------------------------
// Per-particle trimming of the stencil (walks with TRIM).  A stencil row (dy, dz, w) holds every
// neighbour of any point of the cell; one particle needs only the cells within H of itself.  The
// cell build records, per pencil (the cells of one (cy, cz) row along x), the transverse box of its
// particles as fractions of a cell.  With the particle at fractions (f_y, f_z) of its own cell,
// the pencil's particles lie at [dy + lo_y, dy + hi_y] cells from that cell's origin along y, so
// the gap max(dy + lo_y - f_y, f_y - dy - hi_y, 0) (and along z) bounds the transverse distance e
// from below, whatever the periodic wrap of the pencil index.  Rows with e >= H are skipped and
// the x cell range shrinks to [floor(f_x - xe), floor(f_x + xe)], xe = sqrt(H^2 - e^2) / width.
// The radius is widened by 2^-12 H (far above the FP32 rounding of these bounds), so a skipped
// candidate lies beyond H by more than the evaluation's rounding and its term is exactly 0: the
// sums are bitwise those of the full stencil.

// One stencil row as the trimmed walks read it (staged in shared memory by the kernel): the offsets
// as floats, the pencil-index offset dz ncy + dy (no wrap), and w | dy << 8 | dz << 16.
struct TrimRow {
    float fdy, fdz;
    int off, wdd;
};

__device__ __forceinline__ void stage_trim_rows(TrimRow *srow, const RateParams &prm)
{
    for (int r = threadIdx.x; r < prm.nrows; r += blockDim.x) {
        const StencilRow row = prm.rows[r];
        TrimRow t;
        t.fdy = (float)row.dy;
        t.fdz = (float)row.dz;
        t.off = (int)row.dz * prm.ncy + (int)row.dy;
        t.wdd = ((int)row.w & 0xff) | (((int)row.dy & 0xff) << 8) | (((int)row.dz & 0xff) << 16);
        srow[r] = t;
    }
    __syncthreads();
}

// Per-particle quantities of the trimming: fractional cell position (x, y, z), the index of the
// particle's own pencil, and whether no stencil row of the particle's cell wraps along y or z.
struct TrimSelf {
    float fx, fy, fz;
    int p0;
    bool interior;
};

template <int DIM>
__device__ __forceinline__ TrimSelf trim_self(const uint4 &pa, int cy, int cz, const RateParams &prm)
{
    const float inv32 = 2.3283064365386963e-10f;   // 2^-32
    TrimSelf t;
    t.fx = (float)((pa.x - prm.back[0]) * (uint32_t)prm.ncx) * inv32;
    t.fy = (float)((pa.y - prm.back[1]) * (uint32_t)prm.ncy) * inv32;
    t.fz = DIM == 3 ? (float)((pa.z - prm.back[2]) * (uint32_t)prm.ncz) * inv32 : 0.f;
    t.p0 = cz * prm.ncy + cy;
    t.interior = cy >= prm.k && cy < prm.ncy - prm.k && (DIM == 2 || (cz >= prm.k && cz < prm.ncz - prm.k));
    return t;
}

// Pencil index of row r for a particle in pencil (cy, cz).
template <int DIM>
__device__ __forceinline__ int row_pencil(const TrimRow &r, const TrimSelf &me, int cy, int cz, const RateParams &prm)
{
    if (me.interior) return me.p0 + r.off;
    int yy = cy + ((int)((unsigned)r.wdd << 16) >> 24);
    yy += (yy < 0) ? prm.ncy : 0;
    yy -= (yy >= prm.ncy) ? prm.ncy : 0;
    int zz = 0;
    if (DIM == 3) {
        zz = cz + ((int)((unsigned)r.wdd << 8) >> 24);
        zz += (zz < 0) ? prm.ncz : 0;
        zz -= (zz >= prm.ncz) ? prm.ncz : 0;
    }
    return zz * prm.ncy + yy;
}

// Geometry shared by the rows: (H (1 + 2^-12))^2 rounded up in x-units^2, cells per x unit, and
// half the y and z cell heights in x units (the gaps below are twice the gap in cells).
struct TrimGeom {
    float Hm2, inv_wx, hy, hz;
    __device__ __forceinline__ explicit TrimGeom(const RateParams &prm)
    {
        const float two32 = 4294967296.f;
        Hm2 = prm.H2 * (1.f + 1.f / 2048.f);
        inv_wx = (float)prm.ncx * (1.f / two32);
        hy = 0.5f * two32 / (float)prm.ncy * prm.sy;
        hz = 0.5f * two32 / (float)prm.ncz * prm.sz;
    }
};

// The x cell range [dlo, dhi] (relative to the particle's cell) of one row with pencil box bb for
// one particle; false when the row is out of its reach.  2 gap = |lo - r| + |r - hi| - (hi - lo)
// with r the particle's position relative to the row.
template <int DIM>
__device__ __forceinline__ bool trim_row(const float4 &bb, float wy, float wz, const TrimRow &r, int w,
                                         const TrimSelf &me, const TrimGeom &g, int &dlo, int &dhi)
{
    const float ry = me.fy - r.fdy;
    const float ey = ((fabsf(bb.x - ry) + fabsf(ry - bb.y)) - wy) * g.hy;
    float e2 = ey * ey;
    if (DIM == 3) {
        const float rz = me.fz - r.fdz;
        const float ez = ((fabsf(bb.z - rz) + fabsf(rz - bb.w)) - wz) * g.hz;
        e2 = fmaf(ez, ez, e2);
    }
    if (!(e2 < g.Hm2)) return false;
    const float t = g.Hm2 - e2;
    const float xe = fmaf(t * rsqrt_ftz(t), g.inv_wx, 1.f / 4096.f);   // half-extent in cells
    dlo = max(__float2int_rd(me.fx - xe), -w);
    dhi = min(__float2int_rd(me.fx + xe), w);
    return true;
}

__device__ __forceinline__ float4 load_box(const RateParams &prm, int pidx)
{
    return __ldg(reinterpret_cast<const float4 *>(prm.pencil) + pidx);
}

// Candidate index ranges of cells [lo, hi) of the pencil row starting at cell `base`: [s0, e0) and,
// at a periodic seam (lo < 0 or hi > ncx), [s1, e1) for the wrapped part; without a seam
// s1 = e1.  Branch-free (the lanes of a warp meet the seam at different rows), with the same four
// cell-table reads for every lane.
__device__ __forceinline__ void row_ranges(const uint32_t *__restrict__ cs, int base, int lo, int hi, int ncx,
                                           int &s0, int &e0, int &s1, int &e1)
{
    const bool wl = lo < 0, wh = hi > ncx;
    const int a0 = wl ? lo + ncx : lo;            // first piece [a0, b0)
    const int b0 = (wl || wh) ? ncx : hi;
    const int b1 = wl ? hi : (wh ? hi - ncx : 0); // second piece [0, b1)
    s0 = __ldg(cs + base + a0);
    e0 = __ldg(cs + base + b0);
    s1 = __ldg(cs + base);
    e1 = __ldg(cs + base + b1);
}

// ---------------------------------------------------------------------------------------------
// direct walk over global memory
// ---------------------------------------------------------------------------------------------
// One candidate range of the direct walk.  The evaluation is branch-free: outside the support
// 1 - q is clamped to 0 (as om + |om| = 2 max(om, 0); the shape of twice the argument is an exact
// power-of-two multiple, undone per particle), so the term is exactly 0; at zero separation (the
// particle itself, or a coincident particle) rsqrt(0) = inf makes q and s NaN, and IEEE max-num
// (fmaxf returns the non-NaN operand) turns them into 2 (1 - q) = 0 and s = -FLT_MAX, so the
// weight is exactly 0 as well.  In-support terms use the same operations as a branched
// evaluation, so adding the zero terms leaves the sum unchanged.  The pair counter keeps an
// explicit FP64 test.
// BF = false keeps the branch on r^2 < H^2 instead: a warp whose lanes all miss skips the term,
// which pays off when warps are spatially coherent and the stencil is large (3D).
// ZS = false drops both max-num clamps: zero separation occurs only within the particle's own
// cell, so rows other than the particle's own cell row (dy = dz = 0) never meet it, q and s are
// finite there and om + |om| clamps.
template <int DIM, int KERNEL, bool ISO, bool COUNT, bool BF, bool ZS = true>
__device__ __forceinline__ void pair_range_direct(const uint4 *__restrict__ P, int j0, int j1,
                                                  const uint4 &pa, float Ca, const PairConst &k,
                                                  const RateParams &prm, float &rs, unsigned &cnt)
{
#pragma unroll 8
    for (int j = j0; j < j1; ++j) {
        const uint4 pb = __ldg(P + j);
        if (COUNT) cnt += in_support_fp64<DIM>((int)(pa.x - pb.x), (int)(pa.y - pb.y), (int)(pa.z - pb.z), prm);
        const int m = DIM == 3 ? k.m1 : -1;   // as in pair_range_direct2
        float dx = sep(pa.x, pb.x, m);
        float dy = sep(pa.y, pb.y, m);
        float dz = 0.f;
        if (DIM == 3) dz = sep(pa.z, pb.z, m);
        if (!ISO) {
            dy *= k.sy;
            if (DIM == 3) dz *= k.sz;
        }
        float r2 = fmaf(dx, dx, dy * dy);
        if (DIM == 3) r2 = fmaf(dz, dz, r2);
        if (BF) {
            const float rinv = rsqrt_ftz(r2);
            const float om = fmaf(-(r2 * rinv), k.invH, 1.f);
            const float omq2 = ZS ? fmaxf(om + om, 0.f) : om + fabsf(om);
            const float sr = dcal<DIM>(dx, dy, dz, rinv, k);
            const float s = ZS ? fmaxf(sr, -3.402823466e38f) : sr;
            rs = fmaf(shape2x<KERNEL>(omq2) * s, Ca - __uint_as_float(pb.w), rs);
        } else if (r2 < k.H2 && r2 > 0.f) {
            const float rinv = rsqrt_ftz(r2);
            const float om = fmaf(-(r2 * rinv), k.invH, 1.f);
            const float s = dcal<DIM>(dx, dy, dz, rinv, k);
            rs = fmaf(shape2x<KERNEL>(om + om) * s, Ca - __uint_as_float(pb.w), rs);
        }
    }
}

// Twice the gap (squared, in x units^2) between the transverse interval [ylo, yhi] x [zlo, zhi]
// (cell fractions from the particles' cell; widths py, pz) and the box bb of row r:
// 2 gap = |b0 - a1| + |a0 - b1| - (b1 - b0) - (a1 - a0) per axis, 0 where they overlap.
template <int DIM>
__device__ __forceinline__ float row_gap2(const float4 &bb, const TrimRow &r, float ylo, float yhi, float py,
                                          float zlo, float zhi, float pz, const TrimGeom &g)
{
    const float ay0 = ylo - r.fdy, ay1 = yhi - r.fdy;
    const float ey = ((fabsf(bb.x - ay1) + fabsf(ay0 - bb.y)) - ((bb.y - bb.x) + py)) * g.hy;
    float e2 = ey * ey;
    if (DIM == 3) {
        const float az0 = zlo - r.fdz, az1 = zhi - r.fdz;
        const float ez = ((fabsf(bb.z - az1) + fabsf(az0 - bb.w)) - ((bb.w - bb.z) + pz)) * g.hz;
        e2 = fmaf(ez, ez, e2);
    }
    return e2;
}

// Rows tested once per warp (every lane in the same pencil, so all lanes share the stencil rows
// and their boxes): lane l takes row rb + l, tests it against the warp's transverse interval and
// returns through `reach` / xe / pidx / wx (bit 24 of wx marks the lanes' own pencil) the row's
// reachability, x half-extent in cells, pencil and row word.
template <int DIM>
__device__ __forceinline__ bool warp_row_test(int rb, const TrimRow *srow, int nrows, const TrimSelf &me, int cy,
                                              int cz, const RateParams &prm, const TrimGeom &g, float ylo, float yhi,
                                              float zlo, float zhi, float &xe, int &pidx, int &wx)
{
    const int ri = rb + (threadIdx.x & 31);
    xe = 0.f;
    pidx = wx = 0;
    if (ri >= nrows) return false;
    const TrimRow r = srow[ri];
    pidx = row_pencil<DIM>(r, me, cy, cz, prm);
    const float e2 = row_gap2<DIM>(load_box(prm, pidx), r, ylo, yhi, yhi - ylo, zlo, zhi, zhi - zlo, g);
    const float t = fmaxf(g.Hm2 - e2, 0.f);
    xe = fmaf(t * rsqrt_ftz(t), g.inv_wx, 1.f / 4096.f);
    wx = r.wdd | (r.off == 0 ? 1 << 24 : 0);
    return e2 < g.Hm2;
}

// Warp-wide transverse interval [ylo, yhi] x [zlo, zhi] (in place).
template <int DIM>
__device__ __forceinline__ void warp_interval(float &ylo, float &yhi, float &zlo, float &zhi)
{
    for (int o = 16; o > 0; o >>= 1) {
        ylo = fminf(ylo, __shfl_xor_sync(0xffffffffu, ylo, o));
        yhi = fmaxf(yhi, __shfl_xor_sync(0xffffffffu, yhi, o));
        if (DIM == 3) {
            zlo = fminf(zlo, __shfl_xor_sync(0xffffffffu, zlo, o));
            zhi = fmaxf(zhi, __shfl_xor_sync(0xffffffffu, zhi, o));
        }
    }
}

// Eq. 4 at one particle by the direct walk; (cx, cy, cz) is its cell.  TRIM: visit only the
// stencil cells within reach of the particle itself (rows from srow, staged by the kernel).
// COOP (every lane of the warp in the particle's pencil): the rows are tested once per warp
// against the warp's transverse interval, which contains the particle's, so a row or candidate
// that only the wider test admits lies beyond H (1 + 2^-12) of the particle and adds an exact zero:
// the sum is bitwise that of the per-particle test.
template <int DIM, int KERNEL, bool ISO, bool COUNT, bool BF = true, bool TRIM = false>
__device__ float rate_direct(const uint4 *__restrict__ Pe, const uint32_t *__restrict__ cs,
                             const uint4 &pa, int cx, int cy, int cz, const RateParams &prm,
                             unsigned &cnt, const TrimRow *srow = nullptr, bool coop = false)
{
    const int ncx = prm.ncx, ncy = prm.ncy, ncz = prm.ncz, nrows = prm.nrows;
    const PairConst kc(prm);
    const float Ca = __uint_as_float(pa.w);
    float acc = 0.f, comp = 0.f;
    if (TRIM && coop) {
        const TrimSelf me = trim_self<DIM>(pa, cy, cz, prm);
        const TrimGeom g(prm);
        float ylo = me.fy, yhi = me.fy, zlo = me.fz, zhi = me.fz;
        warp_interval<DIM>(ylo, yhi, zlo, zhi);
        for (int rb = 0; rb < nrows; rb += 32) {
            float xe;
            int pidx, wx;
            const bool reach = warp_row_test<DIM>(rb, srow, nrows, me, cy, cz, prm, g, ylo, yhi, zlo, zhi, xe, pidx, wx);
            for (unsigned mask = __ballot_sync(0xffffffffu, reach); mask != 0u; mask &= mask - 1u) {
                const int b = __ffs(mask) - 1;
                const float xeb = __shfl_sync(0xffffffffu, xe, b);
                const int pb = __shfl_sync(0xffffffffu, pidx, b), wb = __shfl_sync(0xffffffffu, wx, b);
                const int w = wb & 0xff;
                int s0, e0, s1, e1;
                row_ranges(cs, pb * ncx, cx + max(__float2int_rd(me.fx - xeb), -w),
                           cx + min(__float2int_rd(me.fx + xeb), w) + 1, ncx, s0, e0, s1, e1);
                float rs = 0.f;
                if ((wb >> 24) != 0) {                              // the particle's own cell row
                    pair_range_direct<DIM, KERNEL, ISO, COUNT, BF, true>(Pe, s0, e0, pa, Ca, kc, prm, rs, cnt);
                    pair_range_direct<DIM, KERNEL, ISO, COUNT, BF, true>(Pe, s1, e1, pa, Ca, kc, prm, rs, cnt);
                } else {
                    pair_range_direct<DIM, KERNEL, ISO, COUNT, BF, false>(Pe, s0, e0, pa, Ca, kc, prm, rs, cnt);
                    pair_range_direct<DIM, KERNEL, ISO, COUNT, BF, false>(Pe, s1, e1, pa, Ca, kc, prm, rs, cnt);
                }
                neumaier_add(acc, comp, rs);
            }
        }
        return prm.upf * shape_unscale<KERNEL>() * (acc + comp);
    }
    if (TRIM) {
        const TrimSelf me = trim_self<DIM>(pa, cy, cz, prm);
        const TrimGeom g(prm);
        for (int ri = 0; ri < nrows; ++ri) {
            const TrimRow r = srow[ri];
            const int pidx = row_pencil<DIM>(r, me, cy, cz, prm);
            const float4 bb = load_box(prm, pidx);
            if (!(bb.x <= bb.y)) continue;                          // empty pencil
            int dlo, dhi;
            if (!trim_row<DIM>(bb, bb.y - bb.x, bb.w - bb.z, r, r.wdd & 0xff, me, g, dlo, dhi))
                continue;                                           // the whole row is out of reach
            int s0, e0, s1, e1;
            row_ranges(cs, pidx * ncx, cx + dlo, cx + dhi + 1, ncx, s0, e0, s1, e1);
            float rs = 0.f;
            if (r.off == 0) {                                       // the particle's own cell row
                pair_range_direct<DIM, KERNEL, ISO, COUNT, BF, true>(Pe, s0, e0, pa, Ca, kc, prm, rs, cnt);
                pair_range_direct<DIM, KERNEL, ISO, COUNT, BF, true>(Pe, s1, e1, pa, Ca, kc, prm, rs, cnt);
            } else {
                pair_range_direct<DIM, KERNEL, ISO, COUNT, BF, false>(Pe, s0, e0, pa, Ca, kc, prm, rs, cnt);
                pair_range_direct<DIM, KERNEL, ISO, COUNT, BF, false>(Pe, s1, e1, pa, Ca, kc, prm, rs, cnt);
            }
            neumaier_add(acc, comp, rs);
        }
    } else {
        for (int ri = 0; ri < nrows; ++ri) {
            const StencilRow row = prm.rows[ri];
            int yy = cy + row.dy;
            yy += (yy < 0) ? ncy : 0;
            yy -= (yy >= ncy) ? ncy : 0;
            int zz = 0;
            if (DIM == 3) {
                zz = cz + row.dz;
                zz += (zz < 0) ? ncz : 0;
                zz -= (zz >= ncz) ? ncz : 0;
            }
            int s0, e0, s1, e1;
            row_ranges(cs, (zz * ncy + yy) * ncx, cx - (int)row.w, cx + row.w + 1, ncx, s0, e0, s1, e1);
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
    }
    return prm.upf * shape_unscale<KERNEL>() * (acc + comp);
}

// ---------------------------------------------------------------------------------------------
// paired direct walk: two targets per thread, packed FP32x2 arithmetic
// ---------------------------------------------------------------------------------------------
// Two cell-sorted particles a0, a1 of the same cell row (cx1 - cx0 <= 1) walk one candidate stream:
// per stencil row the union of their cell ranges.  Every candidate is loaded once and both terms
// are evaluated with the packed FP32x2 instructions of this architecture (one instruction, two
// independent IEEE results), each half with exactly the operations of pair_range_direct<BF>.  A
// candidate outside one target's own range lies beyond H (1 + 2^-12) of it -- the stencil rows and
// the trimmed ranges are built for that radius -- so its term is exactly 0 (branch-free) or
// skipped (branched), and each target's row sum is bitwise that of the one-target walk (same
// candidates, same order).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

template <int KERNEL>
__device__ __forceinline__ float2 shape2x2(float2 w)
{
    if (KERNEL == ADE_WENDLAND_C2) return __fmul2_rn(__fmul2_rn(w, w), w);
    const float2 o2 = __fmul2_rn(w, w);
    const float2 t = __ffma2_rn(f2(-2.5f, -2.5f), w, f2(6.f, 6.f));
    return __fmul2_rn(__fmul2_rn(__fmul2_rn(o2, o2), w), t);
}

// Packed per-pair constants (both halves equal).
struct PairConst2 {
    float2 w0, w1, w2, b, ninvH, sy, sz;
    float H2;
    int m1;     // -1 (see sep)
    __device__ __forceinline__ explicit PairConst2(const PairConst &k, int m1_)
        : w0(f2(k.w0, k.w0)), w1(f2(k.w1, k.w1)), w2(f2(k.w2, k.w2)), b(f2(k.b, k.b)),
          ninvH(f2(-k.invH, -k.invH)), sy(f2(k.sy, k.sy)), sz(f2(k.sz, k.sz)), H2(k.H2), m1(m1_)
    {
    }
};

template <int DIM>
__device__ __forceinline__ float2 dcal2(float2 dx, float2 dy, float2 dz, float2 rinv, const PairConst2 &k)
{
    float2 u = __ffma2_rn(k.w0, dx, __fmul2_rn(k.w1, dy));
    if (DIM == 3) u = __ffma2_rn(k.w2, dz, u);
    const float2 t = __fmul2_rn(u, rinv);
    return __ffma2_rn(t, t, k.b);
}

// BF = false: the branched form -- the term is evaluated when either target is in support
// (0 < r^2 < H^2), each half with the operations of pair_range_direct<BF = false>, and a half
// whose target is not in support adds an exact zero.
// The candidates are [s0, s0 + n0) followed by [s1, s1 + n1) (a row cut by the periodic seam of
// the cell grid); MERGED walks both in one loop, so that a warp whose lanes cut rows at different
// places keeps every lane busy, in the same candidate order as two loops.
template <int DIM, int KERNEL, bool ISO, bool ZS, bool BF = true, bool MERGED = false>
__device__ __forceinline__ void pair_range_direct2(const uint4 *__restrict__ P, int s0, int n0, int s1, int n1,
                                                   const uint4 &pa0, const uint4 &pa1, float2 Ca,
                                                   const PairConst2 &k, float2 &rs)
{
    const int nt = MERGED ? n0 + n1 : n0;
    const int jump = s1 - (s0 + n0);
#pragma unroll 4
    for (int t = 0; t < nt; ++t) {
        const int j = s0 + t + (MERGED && t >= n0 ? jump : 0);
        const uint4 pb = __ldg(P + j);
        // 3D walks are bound by the ALU pipe, so their separations take the multiply-add form;
        // in 2D (neither pipe saturated) a plain subtraction is cheaper
        const int m = DIM == 3 ? k.m1 : -1;
        float2 dx = f2(sep(pa0.x, pb.x, m), sep(pa1.x, pb.x, m));
        float2 dy = f2(sep(pa0.y, pb.y, m), sep(pa1.y, pb.y, m));
        float2 dz = f2(0.f, 0.f);
        if (DIM == 3) dz = f2(sep(pa0.z, pb.z, m), sep(pa1.z, pb.z, m));
        if (!ISO) {
            dy = __fmul2_rn(dy, k.sy);
            if (DIM == 3) dz = __fmul2_rn(dz, k.sz);
        }
        float2 r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
        if (DIM == 3) r2 = __ffma2_rn(dz, dz, r2);
        if (!BF) {
            const bool in0 = r2.x < k.H2 && r2.x > 0.f, in1 = r2.y < k.H2 && r2.y > 0.f;
            if (in0 || in1) {
                const float2 rinv = f2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
                const float2 om = __ffma2_rn(__fmul2_rn(r2, rinv), k.ninvH, f2(1.f, 1.f));
                const float2 w = __fmul2_rn(shape2x2<KERNEL>(__fadd2_rn(om, om)), dcal2<DIM>(dx, dy, dz, rinv, k));
                const float nCb = -__uint_as_float(pb.w);
                rs = __ffma2_rn(f2(in0 ? w.x : 0.f, in1 ? w.y : 0.f), __fadd2_rn(Ca, f2(nCb, nCb)), rs);
            }
            continue;
        }
        const float2 rinv = f2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
        const float2 om = __ffma2_rn(__fmul2_rn(r2, rinv), k.ninvH, f2(1.f, 1.f));
        const float2 omq2 = ZS ? f2(fmaxf(om.x + om.x, 0.f), fmaxf(om.y + om.y, 0.f))
                               : f2(om.x + fabsf(om.x), om.y + fabsf(om.y));
        const float2 sr = dcal2<DIM>(dx, dy, dz, rinv, k);
        const float2 sc = ZS ? f2(fmaxf(sr.x, -3.402823466e38f), fmaxf(sr.y, -3.402823466e38f)) : sr;
        const float nCb = -__uint_as_float(pb.w);
        rs = __ffma2_rn(__fmul2_rn(shape2x2<KERNEL>(omq2), sc), __fadd2_rn(Ca, f2(nCb, nCb)), rs);
    }
}

// One row of the paired walks: the candidates [s0, e0) and [s1, e1).  Where no lane of the warp
// meets the seam a single plain loop runs; otherwise every lane walks its two pieces in one loop.
template <int DIM, int KERNEL, bool ISO, bool ZS, bool BF>
__device__ __forceinline__ void pair_row2(const uint4 *__restrict__ P, int s0, int e0, int s1, int e1,
                                          const uint4 &pa0, const uint4 &pa1, float2 Ca, const PairConst2 &k,
                                          float2 &rs)
{
    const int n1 = e1 > s1 ? e1 - s1 : 0;
    if (__any_sync(__activemask(), n1 > 0))
        pair_range_direct2<DIM, KERNEL, ISO, ZS, BF, true>(P, s0, e0 - s0, s1, n1, pa0, pa1, Ca, k, rs);
    else
        pair_range_direct2<DIM, KERNEL, ISO, ZS, BF, false>(P, s0, e0 - s0, s1, 0, pa0, pa1, Ca, k, rs);
}

// Packed compensated addition: Neumaier's scheme per half with the two-sum error term (as
// neumaier_add), in FP32x2 instructions; a - b is taken as fma(b, -1, a), the same correctly
// rounded difference.
__device__ __forceinline__ void neumaier_add2(float2 &sum, float2 &comp, float2 x)
{
    const float2 m1 = f2(-1.f, -1.f);
    const float2 t = __fadd2_rn(sum, x);
    const float2 bp = __ffma2_rn(sum, m1, t);                                  // t - sum
    const float2 e = __fadd2_rn(__ffma2_rn(__ffma2_rn(bp, m1, t), m1, sum),    // sum - (t - bp)
                                __ffma2_rn(bp, m1, x));                        // x - bp
    comp = __fadd2_rn(comp, e);
    sum = t;
}

// One trimmed row of the paired walk: cells [cx0 + floor(xa - xe), cx0 + floor(xb + xe)] of pencil
// pidx, clipped to the row's half-width w = wx & 0xff; bit 24 of wx marks the targets' own pencil.
template <int DIM, int KERNEL, bool ISO, bool BF>
// The row's first and last candidates lie in whole cells at the ends of the range; one whose x
// word is farther than xe (rounded up to words: wpc words per cell) left of the left target xl,
// or right of the right target xr, is beyond H (1 + 2^-12) of both (the same bound as the cell
// range) and adds an exact zero, so it is dropped before the loop (when every lane of a warp drops
// one, the warp walks one candidate fewer).
__device__ __forceinline__ void pair_trim_row(const uint4 *__restrict__ Pe, const uint32_t *__restrict__ cs,
                                              int pidx, int wx, float xe, float xa, float xb, int cx0, int dcx,
                                              int ncx, const uint4 &pa0, const uint4 &pa1, float2 Ca,
                                              const PairConst2 &k2, float2 &acc, float2 &comp, uint32_t xl,
                                              uint32_t xr, float wpc)
{
    const int w = wx & 0xff;
    const int lo = cx0 + max(__float2int_rd(xa - xe), -w);
    const int hi = cx0 + min(__float2int_rd(xb + xe), w + dcx) + 1;
    int s0, e0, s1, e1;
    row_ranges(cs, pidx * ncx, lo, hi, ncx, s0, e0, s1, e1);
    const int xw = __float2int_ru(fminf(xe * wpc, 2.0e9f));
    if (s0 < e0 && (int)(__ldg(&Pe[s0].x) - xl) < -xw) ++s0;
    if (e1 > s1) {
        if ((int)(__ldg(&Pe[e1 - 1].x) - xr) > xw) --e1;
    } else if (e0 > s0 && (int)(__ldg(&Pe[e0 - 1].x) - xr) > xw) {
        --e0;
    }
    float2 rs = f2(0.f, 0.f);
    if (!BF || (wx >> 24) != 0)   // the targets' own cell row
        pair_row2<DIM, KERNEL, ISO, true, BF>(Pe, s0, e0, s1, e1, pa0, pa1, Ca, k2, rs);
    else
        pair_row2<DIM, KERNEL, ISO, false, BF>(Pe, s0, e0, s1, e1, pa0, pa1, Ca, k2, rs);
    neumaier_add2(acc, comp, rs);
}

// Eq. 4 at two particles of the same cell row by the paired walk; (cx0, cx1, cy, cz) their cells.
// TRIM: one trimmed range per row serves both particles -- the pair's transverse interval
// [min f, max f] against the pencil box bounds both particles' distances to the row from below,
// and [min f_x - xe, max f_x + xe] (cells from cx0) contains both particles' own ranges -- so each
// particle's row sum is bitwise that of rate_direct with TRIM (the extra candidates lie beyond
// H (1 + 2^-12) of it and add exact zeros, a row that is out of reach of one particle adds an exact
// zero to its sum, and an empty or unreachable pencil gives a gap of +inf).
// COOP (every lane of the warp holds a pair of the same pencil, so all lanes share the stencil
// rows and their boxes): the rows are tested once per warp, each lane one row, against the
// warp's transverse interval (which contains every pair's, so the same argument holds); the
// reachable rows, in stencil order, are then walked by all lanes with the pair's own x extent.
template <int DIM, int KERNEL, bool ISO, bool TRIM, bool BF = true>
__device__ void rate_direct_pair(const uint4 *__restrict__ Pe, const uint32_t *__restrict__ cs,
                                 const uint4 &pa0, const uint4 &pa1, int cx0, int cx1, int cy, int cz,
                                 const RateParams &prm, float &r0, float &r1, const TrimRow *srow = nullptr,
                                 bool coop = false)
{
    const int ncx = prm.ncx, ncy = prm.ncy, ncz = prm.ncz, nrows = prm.nrows;
    const PairConst kc(prm);
    const PairConst2 k2(kc, kc.m1);
    const float2 Ca = f2(__uint_as_float(pa0.w), __uint_as_float(pa1.w));
    float2 acc = f2(0.f, 0.f), comp = f2(0.f, 0.f);
    if (TRIM) {
        const TrimSelf m0 = trim_self<DIM>(pa0, cy, cz, prm), m1 = trim_self<DIM>(pa1, cy, cz, prm);
        const TrimGeom g(prm);
        float ylo = fminf(m0.fy, m1.fy), yhi = fmaxf(m0.fy, m1.fy);
        float zlo = fminf(m0.fz, m1.fz), zhi = fmaxf(m0.fz, m1.fz);
        const int dcx = cx1 - cx0;
        // the pair's x extent in cell coordinates from cell cx0 (two particles of one cell are
        // ordered by caller index, not by position)
        const float xa = fminf(m0.fx, m1.fx + (float)dcx), xb = fmaxf(m0.fx, m1.fx + (float)dcx);
        const bool first_left = m0.fx <= m1.fx + (float)dcx;   // which particle is xa
        const uint32_t xl = first_left ? pa0.x : pa1.x, xr = first_left ? pa1.x : pa0.x;
        const float wpc = 4294967296.f / (float)ncx;              // x words per cell
        if (coop) {
            constexpr unsigned kFull = 0xffffffffu;
            warp_interval<DIM>(ylo, yhi, zlo, zhi);
            for (int rb = 0; rb < nrows; rb += 32) {
                float xe;
                int pidx, wx;
                const bool reach = warp_row_test<DIM>(rb, srow, nrows, m0, cy, cz, prm, g, ylo, yhi, zlo, zhi, xe, pidx, wx);
                for (unsigned mask = __ballot_sync(kFull, reach); mask != 0u; mask &= mask - 1u) {
                    const int b = __ffs(mask) - 1;
                    pair_trim_row<DIM, KERNEL, ISO, BF>(Pe, cs, __shfl_sync(kFull, pidx, b), __shfl_sync(kFull, wx, b),
                                                        __shfl_sync(kFull, xe, b), xa, xb, cx0, dcx, ncx, pa0, pa1,
                                                        Ca, k2, acc, comp, xl, xr, wpc);
                }
            }
        } else {
            const float py = yhi - ylo, pz = zhi - zlo;
            for (int ri = 0; ri < nrows; ++ri) {
                const TrimRow r = srow[ri];
                const int pidx = row_pencil<DIM>(r, m0, cy, cz, prm);
                const float e2 = row_gap2<DIM>(load_box(prm, pidx), r, ylo, yhi, py, zlo, zhi, pz, g);
                if (!(e2 < g.Hm2)) continue;      // out of reach of both (or an empty pencil)
                const float t = g.Hm2 - e2;
                const float xe = fmaf(t * rsqrt_ftz(t), g.inv_wx, 1.f / 4096.f);
                pair_trim_row<DIM, KERNEL, ISO, BF>(Pe, cs, pidx, r.wdd | (r.off == 0 ? 1 << 24 : 0), xe, xa, xb,
                                                    cx0, dcx, ncx, pa0, pa1, Ca, k2, acc, comp, xl, xr, wpc);
            }
        }
    } else {
        for (int ri = 0; ri < nrows; ++ri) {
            const StencilRow row = prm.rows[ri];
            int yy = cy + row.dy;
            yy += (yy < 0) ? ncy : 0;
            yy -= (yy >= ncy) ? ncy : 0;
            int zz = 0;
            if (DIM == 3) {
                zz = cz + row.dz;
                zz += (zz < 0) ? ncz : 0;
                zz -= (zz >= ncz) ? ncz : 0;
            }
            int s0, e0, s1, e1;
            row_ranges(cs, (zz * ncy + yy) * ncx, cx0 - (int)row.w, cx1 + row.w + 1, ncx, s0, e0, s1, e1);
            float2 rs = f2(0.f, 0.f);
            if (!BF || (row.dy == 0 && (DIM == 2 || row.dz == 0)))   // the targets' own cell row
                pair_row2<DIM, KERNEL, ISO, true, BF>(Pe, s0, e0, s1, e1, pa0, pa1, Ca, k2, rs);
            else
                pair_row2<DIM, KERNEL, ISO, false, BF>(Pe, s0, e0, s1, e1, pa0, pa1, Ca, k2, rs);
            neumaier_add2(acc, comp, rs);
        }
    }
    const float pf = prm.upf * shape_unscale<KERNEL>();
    r0 = pf * (acc.x + comp.x);
    r1 = pf * (acc.y + comp.y);
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

// Whether sorted particles a0, a1 (cells cx0 <= cx1 in row cy, cz) can share one candidate stream:
// the same cell row, at most one cell apart, and a grid wide enough that the union of their
// ranges (<= 2 kMaxSubdiv + 2 cells) never wraps onto itself.
__device__ __forceinline__ bool can_pair(int cx0, int cy0, int cz0, int cx1, int cy1, int cz1, int ncx)
{
    return cy0 == cy1 && cz0 == cz1 && cx1 - cx0 <= 1 && ncx >= 2 * kMaxSubdiv + 2;
}

