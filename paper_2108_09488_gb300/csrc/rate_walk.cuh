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
    template <class P>
    __device__ __forceinline__ explicit PairConst(const P &prm)
        : H2(prm.H2), invH(prm.invH), sy(prm.sy), sz(prm.sz), w0(prm.uw[0]), w1(prm.uw[1]), w2(prm.uw[2]),
          b(prm.ub)
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

// Lower bound, in fixed-point units of the x axis, of the transverse distance from a target at
// build-relative coordinates (ya, za) to any particle of a pencil with box bb = {min y, max y,
// min z, max z} (also build-relative); squared.  Differences are taken as int32 (minimum image).
template <int DIM>
__device__ __forceinline__ float pencil_gap2(const uint4 &bb, uint32_t ya, uint32_t za, float sy, float sz)
{
    const float ey = (float)max(max((int)(bb.x - ya), (int)(ya - bb.y)), 0) * sy;
    float e2 = ey * ey;
    if (DIM == 3) {
        const float ez = (float)max(max((int)(bb.z - za), (int)(za - bb.w)), 0) * sz;
        e2 = fmaf(ez, ez, e2);
    }
    return e2;
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
            const float rinv = rsqrt_ftz(r2);
            const float omq = fmaxf(fmaf(-(r2 * rinv), k.invH, 1.f), 0.f);
            const float sr = dcal<DIM>(dx, dy, dz, rinv, k);
            const float s = ZS ? fmaxf(sr, -3.402823466e38f) : sr;
            rs = fmaf(shape<KERNEL>(omq) * s, Ca - __uint_as_float(pb.w), rs);
        } else if (r2 < k.H2 && r2 > 0.f) {
            const float rinv = rsqrt_ftz(r2);
            const float omq = fmaf(-(r2 * rinv), k.invH, 1.f);
            const float s = dcal<DIM>(dx, dy, dz, rinv, k);
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
    // position are needed.  The row's pencil box (the transverse extent of the particles in that
    // y-z row of cells at the cell build) bounds the transverse distance e from below, so rows with
    // e >= H are skipped, and the x cell range shrinks to [floor(f_x - xe), floor(f_x + xe)],
    // xe = sqrt(H^2 - e^2) / width, f_x the particle's fractional cell coordinate (the low word of
    // x nc: umulhi gives the cell, the low 32 bits the offset within it exactly).  The radius is
    // widened by 2^-12 H (far above the FP32 rounding of these bounds), so a skipped candidate lies
    // beyond H by more than the evaluation's rounding and its term is exactly 0: the sums are
    // bitwise those of the full stencil.
    const float two32 = 4294967296.f;
    const float fx = (float)((pa.x - prm.back[0]) * (uint32_t)ncx) * (1.f / two32);
    const uint32_t ya = pa.y - prm.back[1], za = pa.z - prm.back[2];
    const float inv_wx = (float)ncx * (1.f / two32);              // cells per x unit
    const float Hm2 = kc.H2 * (1.f + 1.f / 2048.f);                // (H (1 + 2^-12))^2, rounded up
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
        int dlo = -(int)row.w, dhi = row.w;
        if (TRIM) {
            const uint4 bb = __ldg(prm.pencil + (zz * ncy + yy));
            if (bb.x > bb.y) continue;                              // empty pencil
            const float e2 = pencil_gap2<DIM>(bb, ya, za, kc.sy, kc.sz);
            if (!(e2 < Hm2)) continue;                              // the whole row is out of reach
            const float t = Hm2 - e2;
            const float xe = t * rsqrt_ftz(t) * inv_wx + 1.f / 4096.f;  // half-extent in cells
            dlo = max(__float2int_rd(fx - xe), dlo);
            dhi = min(__float2int_rd(fx + xe), dhi);
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
    return prm.upf * (acc + comp);
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
__device__ __forceinline__ float2 shape2(float2 omq)
{
    if (KERNEL == ADE_WENDLAND_C2) return __fmul2_rn(__fmul2_rn(omq, omq), omq);
    const float2 o2 = __fmul2_rn(omq, omq);
    const float2 t = __ffma2_rn(f2(-5.f, -5.f), omq, f2(6.f, 6.f));
    return __fmul2_rn(__fmul2_rn(__fmul2_rn(o2, o2), omq), t);
}

// Packed per-pair constants (both halves equal).
struct PairConst2 {
    float2 w0, w1, w2, b, ninvH, sy, sz;
    float H2;
    __device__ __forceinline__ explicit PairConst2(const PairConst &k)
        : w0(f2(k.w0, k.w0)), w1(f2(k.w1, k.w1)), w2(f2(k.w2, k.w2)), b(f2(k.b, k.b)),
          ninvH(f2(-k.invH, -k.invH)), sy(f2(k.sy, k.sy)), sz(f2(k.sz, k.sz)), H2(k.H2)
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
template <int DIM, int KERNEL, bool ISO, bool ZS, bool BF = true>
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
        if (!BF) {
            const bool in0 = r2.x < k.H2 && r2.x > 0.f, in1 = r2.y < k.H2 && r2.y > 0.f;
            if (in0 || in1) {
                const float2 rinv = f2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
                const float2 omq = __ffma2_rn(__fmul2_rn(r2, rinv), k.ninvH, f2(1.f, 1.f));
                const float2 w = __fmul2_rn(shape2<KERNEL>(omq), dcal2<DIM>(dx, dy, dz, rinv, k));
                const float nCb = -__uint_as_float(pb.w);
                rs = __ffma2_rn(f2(in0 ? w.x : 0.f, in1 ? w.y : 0.f), __fadd2_rn(Ca, f2(nCb, nCb)), rs);
            }
            continue;
        }
        const float2 rinv = f2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
        const float2 om = __ffma2_rn(__fmul2_rn(r2, rinv), k.ninvH, f2(1.f, 1.f));
        const float2 omq = f2(fmaxf(om.x, 0.f), fmaxf(om.y, 0.f));
        const float2 sr = dcal2<DIM>(dx, dy, dz, rinv, k);
        const float2 sc = ZS ? f2(fmaxf(sr.x, -3.402823466e38f), fmaxf(sr.y, -3.402823466e38f)) : sr;
        const float nCb = -__uint_as_float(pb.w);
        rs = __ffma2_rn(__fmul2_rn(shape2<KERNEL>(omq), sc), __fadd2_rn(Ca, f2(nCb, nCb)), rs);
    }
}

// Eq. 4 at two particles of the same cell row by the paired walk; (cx0, cx1, cy, cz) their cells.
template <int DIM, int KERNEL, bool ISO, bool TRIM, bool BF = true>
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
    const uint32_t ya0 = pa0.y - prm.back[1], za0 = pa0.z - prm.back[2];
    const uint32_t ya1 = pa1.y - prm.back[1], za1 = pa1.z - prm.back[2];
    const float inv_wx = (float)ncx * (1.f / two32);
    const float Hm2 = kc.H2 * (1.f + 1.f / 2048.f);
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
        int lo0 = cx0 - (int)row.w, hi0 = cx0 + row.w, lo1 = cx1 - (int)row.w, hi1 = cx1 + row.w;
        bool in0 = true, in1 = true;       // the target reaches the row (rate_direct does not skip it)
        bool ne0 = true, ne1 = true;       // ... and its cell range is not empty
        if (TRIM) {
            const uint4 bb = __ldg(prm.pencil + (zz * ncy + yy));
            if (bb.x > bb.y) continue;      // empty pencil: rate_direct skips the row for both
            const float e0 = pencil_gap2<DIM>(bb, ya0, za0, kc.sy, kc.sz);
            const float e1 = pencil_gap2<DIM>(bb, ya1, za1, kc.sy, kc.sz);
            in0 = e0 < Hm2;
            in1 = e1 < Hm2;
            const float t0 = in0 ? Hm2 - e0 : 1.f, t1 = in1 ? Hm2 - e1 : 1.f;
            const float xe0 = t0 * rsqrt_ftz(t0) * inv_wx + 1.f / 4096.f;
            const float xe1 = t1 * rsqrt_ftz(t1) * inv_wx + 1.f / 4096.f;
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
        if (!BF || (row.dy == 0 && (DIM == 2 || row.dz == 0))) {   // the targets' own cell row
            pair_range_direct2<DIM, KERNEL, ISO, true, BF>(Pe, s0, e0, pa0, pa1, Ca, k2, rs);
            pair_range_direct2<DIM, KERNEL, ISO, true, BF>(Pe, s1, e1, pa0, pa1, Ca, k2, rs);
        } else {
            pair_range_direct2<DIM, KERNEL, ISO, false, BF>(Pe, s0, e0, pa0, pa1, Ca, k2, rs);
            pair_range_direct2<DIM, KERNEL, ISO, false, BF>(Pe, s1, e1, pa0, pa1, Ca, k2, rs);
        }
        // a target that does not reach the row (trimmed walk) skips it, as rate_direct does
        if (in0) neumaier_add(acc0, comp0, rs.x);
        if (in1) neumaier_add(acc1, comp1, rs.y);
    }
    r0 = prm.upf * (acc0 + comp0);
    r1 = prm.upf * (acc1 + comp1);
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

