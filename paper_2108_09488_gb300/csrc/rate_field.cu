// rate_field.cu -- Eq. 4-5 with a per-particle velocity field (heterogeneous flow), and the
// per-particle drift of the predictor-corrector (Eq. 8-9).
//
// Each particle carries its own constant velocity v_a (Eq. 1) and hence its own dispersion
// tensor D_a (Eq. 3).  For one ordered pair, in the notation of Eq. 4-5:
//   K_ij  = 4 D_ij,a D_ij,b / (D_ij,a + D_ij,b)     (0 where the denominator is 0),
//   Dcal  = Gamma x^T K x / r^2 - tr K,
//   disp  = 1/2 (m/rho) Dcal (C_a - C_b) W'(r)/r,
//   conv  = C_a (m/rho) (v_a - v_b) . x_ab W'(r)/r,      (grad_a W = W'(r) x_ab / r)
// with W'(r)/r = kc f(q) as in rate.cu.  Particles drift with their own velocities, so relative
// positions change during a step: the cell list is built for the radius H + dt vmax (the skin
// covers the relative drift up to the half step, |v_a - v_b| dt/2 <= dt vmax) while the support
// test uses H.  One thread per cell-sorted particle walks the stencil rows of its build-time
// cell as in the direct kernel; the row sums of both terms are added with Neumaier compensation
// in a fixed order, so results are deterministic.
// Records of v and D are formed once per field in the caller's order (v is constant in time) and
// permuted into the cell-sorted order after every cell build (k_field_permute), so the pair
// loop's loads stay contiguous: candidates of a row are consecutive sorted indices.
//
// Conditioning of Eq. 5.  Diagonal components of D (Eq. 3) are never negative, but off-diagonal
// ones take the sign of v_i v_j, so for neighbours whose velocities point into different quadrants
// D_ij,a + D_ij,b can cancel and K_ij = 4 D_ij,a D_ij,b / (D_ij,a + D_ij,b) is then arbitrarily
// large and sensitive to the rounding of D.  D is therefore computed in FP64 per particle and
// each off-diagonal component is kept as an unevaluated FP32 pair hi + lo (lo = the FP64 value
// minus hi); the pair's denominator is (hi_a + hi_b) + (lo_a + lo_b), whose first sum is exact when
// the two cancel (Sterbenz), so K_ij keeps FP32 relative accuracy.  The lo words ride in the
// otherwise unused fourth lanes of the float4 records, so the pair loop loads nothing extra.
#include "ade_internal.h"

namespace ade {

namespace {

#include "rate_common.cuh"

constexpr int kT = kRateThreads;

// Approximate reciprocal (MUFU, about 1 ulp; subnormal input and output flushed to zero).
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Harmonic-mean component of Eq. 5 for a diagonal entry, with a4 = 4 a precomputed per particle.
// a, b >= 0, so a + b = 0 only when 4ab = 0 too: clamping the denominator to the smallest normal
// number returns K = 0 there without a branch.
__device__ __forceinline__ float hmean_diag(float a, float a4, float b)
{
    return (a4 * b) * rcp_approx(fmaxf(a + b, 1.17549435e-38f));
}

// Twice an off-diagonal component, 2 K_ij, from hi + lo pairs (see the conditioning note above),
// with a8 = 8 a_hi precomputed per particle.  A zero denominator gives K_ij = 0 as in Eq. 5's
// convention; denominators below the smallest normal number count as zero.
__device__ __forceinline__ float hmean_off2(float ah, float a8, float al, float bh, float bl)
{
    const float den = (ah + bh) + (al + bl);
    const float k2 = (a8 * bh) * rcp_approx(den);
    return fabsf(den) >= 1.17549435e-38f ? k2 : 0.f;
}

// Fixed-point drift of one particle read from its Inc record: half step, or full step 2h + c.
__device__ __forceinline__ void half_drift(const uint4 &ic, uint32_t out[3])
{
    out[0] = ic.x;
    out[1] = ic.y;
    out[2] = ic.z;
}

__device__ __forceinline__ void full_drift(const uint4 &ic, uint32_t out[3])
{
    out[0] = 2u * ic.x + ((ic.w & 3u) - 1u);
    out[1] = 2u * ic.y + (((ic.w >> 2) & 3u) - 1u);
    out[2] = 2u * ic.z + (((ic.w >> 4) & 3u) - 1u);
}

// Velocities of the caller's field into the caller-order records (fourth lane cleared) and
// max_a |v_a| as FP32 bits (non-negative floats order like their bit patterns); a non-finite speed
// counts as +inf so that the host check rejects it.
template <int DIM>
__global__ __launch_bounds__(kT) void k_field_velocity(const float *__restrict__ v, int n, float4 *__restrict__ Vc,
                                                       unsigned *__restrict__ out_bits)
{
    const int i = blockIdx.x * kT + threadIdx.x;
    float s = 0.f;
    if (i < n) {
        const float a = v[i], b = v[(size_t)n + i], c = DIM == 3 ? v[2 * (size_t)n + i] : 0.f;
        Vc[i] = make_float4(a, b, c, 0.f);
        s = sqrtf(a * a + b * b + c * c);
        if (!(s <= 3.0e38f)) s = __int_as_float(0x7f800000);
    }
    for (int o = 16; o > 0; o >>= 1) s = fmaxf(s, __shfl_down_sync(0xffffffffu, s, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out_bits, __float_as_uint(s));
}

// Dispersion tensor (Eq. 3) of every particle in FP64 from its velocity, and its fixed-point
// drift per half and full step, stored as the records described in ade_internal.h (caller order).
template <int DIM>
__global__ __launch_bounds__(kT) void k_field_tensors(int n, FieldParams fp, float4 *__restrict__ Vc,
                                                      float4 *__restrict__ DAc, float4 *__restrict__ DBc,
                                                      uint4 *__restrict__ IncC)
{
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i >= n) return;
    const float4 vr = Vc[i];
    const double vv[3] = {vr.x, vr.y, DIM == 3 ? (double)vr.z : 0.0};
    uint32_t h[3], cbits = 0u;
    for (int k = 0; k < 3; ++k) {
        const long long hk = __double2ll_rn(vv[k] * (0.5 * fp.vscale[k]));
        const long long fk = __double2ll_rn(vv[k] * fp.vscale[k]);
        h[k] = (uint32_t)(unsigned long long)hk;
        cbits |= (uint32_t)(fk - 2 * hk + 1) << (2 * k);
    }
    IncC[i] = make_uint4(h[0], h[1], h[2], cbits);
    const double s = sqrt(vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2]);
    const double iso = fp.aT * s + fp.Dm;
    const double g = s > 0.0 ? (fp.aL - fp.aT) / s : 0.0;
    auto hi = [](double d) { return (float)d; };
    auto lo = [](double d) { return (float)(d - (double)(float)d); };
    const double dxx = iso + g * (vv[0] * vv[0]), dxy = g * (vv[0] * vv[1]), dyy = iso + g * (vv[1] * vv[1]);
    if (DIM == 2) {
        DAc[i] = make_float4(hi(dxx), hi(dxy), hi(dyy), lo(dxy));
    } else {
        const double dxz = g * (vv[0] * vv[2]), dyz = g * (vv[1] * vv[2]), dzz = iso + g * (vv[2] * vv[2]);
        Vc[i].w = lo(dxz);
        DAc[i] = make_float4(hi(dxx), hi(dxy), hi(dxz), lo(dxy));
        DBc[i] = make_float4(hi(dyy), hi(dyz), hi(dzz), lo(dyz));
    }
}

// Sorted records after a cell build.
template <int DIM>
__global__ __launch_bounds__(kT) void k_field_permute(const uint32_t *__restrict__ perm, int n,
                                                      const float4 *__restrict__ Vc, const float4 *__restrict__ DAc,
                                                      const float4 *__restrict__ DBc, const uint4 *__restrict__ IncC,
                                                      float4 *__restrict__ V, float4 *__restrict__ DA,
                                                      float4 *__restrict__ DB, uint4 *__restrict__ Inc)
{
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i >= n) return;
    const uint32_t a = __ldg(perm + i);
    V[i] = __ldg(Vc + a);
    DA[i] = __ldg(DAc + a);
    if (DIM == 3) DB[i] = __ldg(DBc + a);
    Inc[i] = __ldg(IncC + a);
}

template <int DIM, int KERNEL, int EPI, bool COUNT>
__global__ __launch_bounds__(kT) void k_rate_field(const uint4 *__restrict__ Pe, const uint32_t *__restrict__ cs,
                                                   const uint32_t *__restrict__ perm,
                                                   const float4 *__restrict__ V, const float4 *__restrict__ DA,
                                                   const float4 *__restrict__ DB, const uint4 *__restrict__ Inc,
                                                   const RateParams prm, const FieldParams fp, const EpiOut out)
{
    pdl_wait();   // no early trigger: see pdl_trigger
    const int i = blockIdx.x * kT + threadIdx.x;
    const bool valid = i < prm.n;
    const int ii = valid ? i : prm.n - 1;
    const uint4 pa = __ldg(Pe + ii);
    const float4 va = __ldg(V + ii);
    const float4 da = __ldg(DA + ii);
    const float4 db = DIM == 3 ? __ldg(DB + ii) : make_float4(0.f, 0.f, 0.f, 0.f);
    // fixed-point drift of this particle; the cell of the cell build is the evaluation position
    // minus the drift since the build (the half step, in the corrector)
    const uint4 ic = EPI == EPI_RATE ? make_uint4(0u, 0u, 0u, 0u) : __ldg(Inc + ii);
    uint32_t back[3] = {0u, 0u, 0u};
    if (EPI == EPI_CORRECT) half_drift(ic, back);
    const int ncx = prm.ncx, ncy = prm.ncy, ncz = prm.ncz;
    const int cx = (int)__umulhi(pa.x - back[0], (uint32_t)ncx);
    const int cy = (int)__umulhi(pa.y - back[1], (uint32_t)ncy);
    const int cz = DIM == 3 ? (int)__umulhi(pa.z - back[2], (uint32_t)ncz) : 0;
    const float Ca = __uint_as_float(pa.w);
    const float H2 = prm.H2, invH = prm.invH, sy = prm.sy, sz = prm.sz, gam = fp.gamma;
    // 4 D (diagonal) and 8 D (off-diagonal) of this particle for the harmonic means
    // (da.z is Dyy in 2D, Dxz in 3D)
    const float4 da4 = make_float4(4.f * da.x, 8.f * da.y, (DIM == 2 ? 4.f : 8.f) * da.z, 0.f);
    const float4 db4 = make_float4(4.f * db.x, 8.f * db.y, 4.f * db.z, 0.f);
    float sd = 0.f, cd = 0.f, sc = 0.f, cc = 0.f;
    unsigned cnt = 0u;
    for (int ri = 0; ri < prm.nrows; ++ri) {
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
        const int base = (zz * ncy + yy) * ncx;
        const int lo = cx - row.w, hi = cx + row.w + 1;
        int r0[2], r1[2];
        if (lo < 0) {
            r0[0] = __ldg(cs + base + lo + ncx);
            r1[0] = __ldg(cs + base + ncx);
            r0[1] = __ldg(cs + base);
            r1[1] = __ldg(cs + base + hi);
        } else if (hi > ncx) {
            r0[0] = __ldg(cs + base + lo);
            r1[0] = __ldg(cs + base + ncx);
            r0[1] = __ldg(cs + base);
            r1[1] = __ldg(cs + base + hi - ncx);
        } else {
            r0[0] = __ldg(cs + base + lo);
            r1[0] = __ldg(cs + base + hi);
            r0[1] = r1[1] = 0;
        }
        float rd = 0.f, rc = 0.f;
        for (int piece = 0; piece < 2; ++piece)
#pragma unroll 4
            for (int j = r0[piece]; j < r1[piece]; ++j) {
                const uint4 pb = __ldg(Pe + j);
                const int ix = (int)(pa.x - pb.x), iy = (int)(pa.y - pb.y), iz = (int)(pa.z - pb.z);
                if (COUNT) {
                    const double dxd = (double)ix * prm.u[0], dyd = (double)iy * prm.u[1];
                    double r2d = __dadd_rn(__dmul_rn(dxd, dxd), __dmul_rn(dyd, dyd));
                    if (DIM == 3) {
                        const double dzd = (double)iz * prm.u[2];
                        r2d = __dadd_rn(r2d, __dmul_rn(dzd, dzd));
                    }
                    cnt += (r2d > 0.0 && r2d < prm.H2d) ? 1u : 0u;
                }
                const float dx = (float)ix;
                const float dy = (float)iy * sy;
                const float dz = DIM == 3 ? (float)iz * sz : 0.f;
                float r2 = fmaf(dx, dx, dy * dy);
                if (DIM == 3) r2 = fmaf(dz, dz, r2);
                if (r2 < H2 && r2 > 0.f) {
                    const float rinv = rsqrtf(r2);
                    const float f = shape<KERNEL>(fmaf(-(r2 * rinv), invH, 1.f));
                    const float4 vb = __ldg(V + j);
                    const float4 d1 = __ldg(DA + j);
                    float Q, tr;
                    if (DIM == 2) {
                        const float kxx = hmean_diag(da.x, da4.x, d1.x);
                        const float kxy2 = hmean_off2(da.y, da4.y, da.w, d1.y, d1.w);
                        const float kyy = hmean_diag(da.z, da4.z, d1.z);
                        Q = fmaf(dx, fmaf(kxx, dx, kxy2 * dy), kyy * dy * dy);
                        tr = kxx + kyy;
                    } else {
                        const float4 d2 = __ldg(DB + j);
                        const float kxx = hmean_diag(da.x, da4.x, d1.x);
                        const float kxy2 = hmean_off2(da.y, da4.y, da.w, d1.y, d1.w);
                        const float kxz2 = hmean_off2(da.z, da4.z, va.w, d1.z, vb.w);
                        const float kyy = hmean_diag(db.x, db4.x, d2.x);
                        const float kyz2 = hmean_off2(db.y, db4.y, db.w, d2.y, d2.w);
                        const float kzz = hmean_diag(db.z, db4.z, d2.z);
                        const float qx = fmaf(kxx, dx, fmaf(kxy2, dy, kxz2 * dz));
                        const float qy = fmaf(kyy, dy, kyz2 * dz);
                        Q = fmaf(dx, qx, fmaf(dy, qy, kzz * dz * dz));
                        tr = kxx + kyy + kzz;
                    }
                    const float s = fmaf(gam * Q, rinv * rinv, -tr);
                    rd = fmaf(f * s, Ca - __uint_as_float(pb.w), rd);
                    float dvx = fmaf(va.x - vb.x, dx, (va.y - vb.y) * dy);
                    if (DIM == 3) dvx = fmaf(va.z - vb.z, dz, dvx);
                    rc = fmaf(f, dvx, rc);
                }
            }
        neumaier_add(sd, cd, rd);
        neumaier_add(sc, cc, rc);
    }
    const float rate = fmaf(prm.pf, sd + cd, fp.pconv * Ca * (sc + cc));

    Acc acc{0.f, 0.f, __int_as_float(0x7f800000), __int_as_float(0xff800000), valid ? cnt : 0u};
    if (valid) {
        if (EPI == EPI_RATE) {
            if (out.rate) {
                const uint32_t a = __ldg(perm + i);
                if (a < (uint32_t)prm.n) out.rate[a] = rate;
            }
        } else if (EPI == EPI_PREDICT) {
            // C^{l+1/2} = C^l + dt/2 r^l, x_a^{l+1/2} = x_a^l + dt/2 v_a
            uint32_t inc[3];
            half_drift(ic, inc);
            uint4 q;
            q.x = pa.x + inc[0];
            q.y = pa.y + inc[1];
            q.z = pa.z + inc[2];
            q.w = __float_as_uint(fmaf(prm.dt, rate, Ca));
            out.Pout[i] = q;
        } else {
            // C^{l+1} = C^l + dt r^{l+1/2}, x_a^{l+1} = x_a^l + dt v_a (caller order); x^l is the
            // evaluation position minus this particle's half-step drift (exact in fixed point)
            const uint32_t a = __ldg(perm + i);
            uint32_t inc[3];
            full_drift(ic, inc);
            float Cn = 0.f;
            if (a < (uint32_t)prm.n) {
                Cn = fmaf(prm.dt, rate, out.C[a]);
                out.C[a] = Cn;
                out.xq[a] = pa.x - back[0] + inc[0];
                out.xq[(size_t)prm.n + a] = pa.y - back[1] + inc[1];
                if (DIM == 3) out.xq[2 * (size_t)prm.n + a] = pa.z - back[2] + inc[2];
            }
            if (!isfinite(Cn)) atomicOr(out.status, 1);
            two_sum_add(acc.hi, acc.lo, Cn, 0.f);
            acc.mn = fminf(acc.mn, Cn);
            acc.mx = fmaxf(acc.mx, Cn);
        }
    }
    warp_finish<EPI, COUNT, kT>(acc, out);
}

template <int DIM, int KERNEL, bool COUNT>
void launch_field_epi(int epi, int blocks, const uint4 *Pe, const uint32_t *cs, const uint32_t *perm,
                      const FieldWork &fw, const RateParams &prm, const FieldParams &fp, const EpiOut &out,
                      cudaStream_t s)
{
    switch (epi) {
    case EPI_RATE:
        launch_pdl(k_rate_field<DIM, KERNEL, EPI_RATE, COUNT>, blocks, kT, 0, s, Pe, cs, perm, fw.V, fw.DA, fw.DB, fw.Inc, prm, fp, out);
        break;
    case EPI_PREDICT:
        launch_pdl(k_rate_field<DIM, KERNEL, EPI_PREDICT, COUNT>, blocks, kT, 0, s, Pe, cs, perm, fw.V, fw.DA, fw.DB, fw.Inc, prm, fp, out);
        break;
    default:
        launch_pdl(k_rate_field<DIM, KERNEL, EPI_CORRECT, COUNT>, blocks, kT, 0, s, Pe, cs, perm, fw.V, fw.DA, fw.DB, fw.Inc, prm, fp, out);
        break;
    }
}

template <int DIM, int KERNEL>
void launch_field_count(bool count, int epi, int blocks, const uint4 *Pe, const uint32_t *cs,
                        const uint32_t *perm, const FieldWork &fw, const RateParams &prm,
                        const FieldParams &fp, const EpiOut &out, cudaStream_t s)
{
    if (count)
        launch_field_epi<DIM, KERNEL, true>(epi, blocks, Pe, cs, perm, fw, prm, fp, out, s);
    else
        launch_field_epi<DIM, KERNEL, false>(epi, blocks, Pe, cs, perm, fw, prm, fp, out, s);
}

}  // namespace

cudaError_t launch_field_records(int dim, const float *v_dev, int n, const FieldParams &fp, const FieldWork &fw,
                                 cudaStream_t s)
{
    if (v_dev) {
        cudaError_t e = cudaMemsetAsync(fw.vmax_bits, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
    }
    if (n == 0) return cudaSuccess;
    const int blocks = (n + kT - 1) / kT;
    if (dim == 2) {
        if (v_dev) k_field_velocity<2><<<blocks, kT, 0, s>>>(v_dev, n, fw.Vc, fw.vmax_bits);
        k_field_tensors<2><<<blocks, kT, 0, s>>>(n, fp, fw.Vc, fw.DAc, fw.DBc, fw.IncC);
    } else {
        if (v_dev) k_field_velocity<3><<<blocks, kT, 0, s>>>(v_dev, n, fw.Vc, fw.vmax_bits);
        k_field_tensors<3><<<blocks, kT, 0, s>>>(n, fp, fw.Vc, fw.DAc, fw.DBc, fw.IncC);
    }
    return cudaGetLastError();
}

cudaError_t launch_field_permute(int dim, const uint32_t *perm, int n, const FieldWork &fw, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const int blocks = (n + kT - 1) / kT;
    if (dim == 2)
        launch_pdl(k_field_permute<2>, blocks, kT, 0, s, perm, n, fw.Vc, fw.DAc, fw.DBc, fw.IncC, fw.V, fw.DA, fw.DB, fw.Inc);
    else
        launch_pdl(k_field_permute<3>, blocks, kT, 0, s, perm, n, fw.Vc, fw.DAc, fw.DBc, fw.IncC, fw.V, fw.DA, fw.DB, fw.Inc);
    return cudaGetLastError();
}

cudaError_t launch_rate_field(int dim, int kernel, int epi, const uint4 *Pe, const uint32_t *cell_start,
                              const uint32_t *perm, const FieldWork &fw, const RateParams &prm,
                              const FieldParams &fp, const EpiOut &out, cudaStream_t s)
{
    if (prm.n == 0) return cudaSuccess;
    const int blocks = (prm.n + kT - 1) / kT;
    const bool count = out.pairs != nullptr;
    if (dim == 2) {
        if (kernel == ADE_WENDLAND_C2)
            launch_field_count<2, ADE_WENDLAND_C2>(count, epi, blocks, Pe, cell_start, perm, fw, prm, fp, out, s);
        else
            launch_field_count<2, ADE_WENDLAND_C4>(count, epi, blocks, Pe, cell_start, perm, fw, prm, fp, out, s);
    } else {
        if (kernel == ADE_WENDLAND_C2)
            launch_field_count<3, ADE_WENDLAND_C2>(count, epi, blocks, Pe, cell_start, perm, fw, prm, fp, out, s);
        else
            launch_field_count<3, ADE_WENDLAND_C4>(count, epi, blocks, Pe, cell_start, perm, fw, prm, fp, out, s);
    }
    return cudaGetLastError();
}

}  // namespace ade
