// sweep.cu -- one plume, many dispersivity sets: Eq. 4-5 for P parameter sets theta_p =
// (alpha_L, alpha_T, D_m)_p that share the particles, the uniform velocity and the time step, each
// with its own concentration field (a parameter sweep or the forward runs of an inversion).
//
// With a uniform v, K = 2D (Eq. 5 with equal tensors) and e = x_ab / r, the pair factor of Eq. 5 is
//     Dcal = Gamma e^T K e - tr K = a_p u + b_p,    u = (vhat . e)^2,
//     a_p = 2 Gamma (aL - aT) |v|,
//     b_p = 2 (Gamma - d) (aT |v| + Dm) - 2 (aL - aT) |v|,
// (substitute D of Eq. 3), so a pair's geometry -- separation, kernel shape f and u -- is computed
// once and each parameter set costs one fused multiply-add for Dcal, a multiply by f, the
// concentration difference and the accumulation.  The cell list, the positions and the drift are
// shared; only the concentrations are per set.  Parameter sets are evaluated in groups of up to 8
// per launch (registers); the sorted concentrations are interleaved [n][P4] (P4 = P rounded up to
// a multiple of 4) so that a group's values are one or two 16-byte loads per candidate.
// Summation as in rate.cu: FP32 row sums, Neumaier across rows, fixed order.
#include "ade_internal.h"

namespace ade {

namespace {

#include "rate_common.cuh"

constexpr int kT = kRateThreads;

template <int NT>
__device__ __forceinline__ void load_group(const float *__restrict__ p, float v[NT])
{
    if (NT == 1) {
        v[0] = __ldg(p);
    } else if (NT == 2) {
        const float2 q = __ldg(reinterpret_cast<const float2 *>(p));
        v[0] = q.x;
        v[1] = q.y;
    } else {
#pragma unroll
        for (int k = 0; k < NT; k += 4) {
            const float4 q = __ldg(reinterpret_cast<const float4 *>(p) + k / 4);
            v[k] = q.x;
            v[k + 1] = q.y;
            v[k + 2] = q.z;
            v[k + 3] = q.w;
        }
    }
}

// Sorted, interleaved concentrations: Cs[i * P4 + p] = C[p * n + perm[i]].
__global__ __launch_bounds__(kT) void k_sweep_gather(const uint32_t *__restrict__ perm, const float *__restrict__ C,
                                                     int n, int P, int P4, float *__restrict__ Cs)
{
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i >= n) return;
    const uint32_t a = __ldg(perm + i);
    for (int p = 0; p < P4; ++p) Cs[(size_t)i * P4 + p] = p < P ? __ldg(C + (size_t)p * n + a) : 0.f;
}

template <int DIM, int KERNEL, int EPI, int NT, bool COUNT>
__global__ __launch_bounds__(kT) void k_rate_sweep(const uint4 *__restrict__ Pe, const float *__restrict__ Ce,
                                                   const uint32_t *__restrict__ cs,
                                                   const uint32_t *__restrict__ perm, const RateParams prm,
                                                   const SweepParams sp, const SweepOut out)
{
    const int i = blockIdx.x * kT + threadIdx.x;
    const bool valid = i < prm.n;
    const int ii = valid ? i : prm.n - 1;
    const uint4 pa = __ldg(Pe + ii);
    const int P4 = sp.P4, g0 = sp.g0;
    float Ca[NT];
    load_group<NT>(Ce + (size_t)ii * P4 + g0, Ca);
    const int ncx = prm.ncx, ncy = prm.ncy, ncz = prm.ncz;
    const int cx = (int)__umulhi(pa.x - prm.back[0], (uint32_t)ncx);
    const int cy = (int)__umulhi(pa.y - prm.back[1], (uint32_t)ncy);
    const int cz = DIM == 3 ? (int)__umulhi(pa.z - prm.back[2], (uint32_t)ncz) : 0;
    const float H2 = prm.H2, invH = prm.invH, sy = prm.sy, sz = prm.sz;
    const float vx = sp.vh[0], vy = sp.vh[1], vz = sp.vh[2];
    float acc[NT], comp[NT];
#pragma unroll
    for (int k = 0; k < NT; ++k) acc[k] = comp[k] = 0.f;
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
        float rs[NT];
#pragma unroll
        for (int k = 0; k < NT; ++k) rs[k] = 0.f;
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
                    float c = fmaf(vx, dx, vy * dy);
                    if (DIM == 3) c = fmaf(vz, dz, c);
                    const float cr = c * rinv;
                    const float u = cr * cr;
                    float Cb[NT];
                    load_group<NT>(Ce + (size_t)j * P4 + g0, Cb);
#pragma unroll
                    for (int k = 0; k < NT; ++k) rs[k] = fmaf(f * fmaf(sp.a[k], u, sp.b[k]), Ca[k] - Cb[k], rs[k]);
                }
            }
#pragma unroll
        for (int k = 0; k < NT; ++k) neumaier_add(acc[k], comp[k], rs[k]);
    }
    if (COUNT) {
        unsigned c = valid ? cnt : 0u;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if ((threadIdx.x & 31) == 0 && c) atomicAdd(out.pairs, (unsigned long long)c);
    }
    if (!valid) return;
    float rate[NT];
#pragma unroll
    for (int k = 0; k < NT; ++k) rate[k] = prm.pf * (acc[k] + comp[k]);
    const size_t n = (size_t)prm.n;
    if (EPI == EPI_RATE) {
        if (out.rate) {
            const uint32_t a = __ldg(perm + i);
            if (a < (uint32_t)n)
#pragma unroll
                for (int k = 0; k < NT; ++k) out.rate[(size_t)(g0 + k) * n + a] = rate[k];
        }
    } else if (EPI == EPI_PREDICT) {
        // C_p^{l+1/2} = C_p^l + dt/2 r_p^l (sorted, interleaved); x^{l+1/2} = x^l + dt/2 v once
#pragma unroll
        for (int k = 0; k < NT; ++k) out.Cout[(size_t)i * P4 + g0 + k] = fmaf(prm.dt, rate[k], Ca[k]);
        if (g0 == 0) {
            uint4 q;
            q.x = pa.x + prm.inc[0];
            q.y = pa.y + prm.inc[1];
            q.z = pa.z + prm.inc[2];
            q.w = 0u;
            out.Pout[i] = q;
        }
    } else {
        // C_p^{l+1} = C_p^l + dt r_p^{l+1/2} and x^{l+1} = x^l + dt v, in the caller's order
        const uint32_t a = __ldg(perm + i);
        if (a < (uint32_t)n) {
            bool bad = false;
#pragma unroll
            for (int k = 0; k < NT; ++k) {
                float *Cp = out.C + (size_t)(g0 + k) * n + a;
                const float Cn = fmaf(prm.dt, rate[k], *Cp);
                *Cp = Cn;
                bad |= !isfinite(Cn);
            }
            if (bad) atomicOr(out.status, 1);
            if (g0 == 0) {
                out.xq[a] = pa.x - prm.back[0] + prm.inc[0];
                out.xq[n + a] = pa.y - prm.back[1] + prm.inc[1];
                if (DIM == 3) out.xq[2 * n + a] = pa.z - prm.back[2] + prm.inc[2];
            }
        }
    }
}

template <int DIM, int KERNEL, int NT>
void launch_sweep_nt(int epi, bool count, int blocks, const uint4 *Pe, const float *Ce, const uint32_t *cs,
                     const uint32_t *perm, const RateParams &prm, const SweepParams &sp, const SweepOut &out,
                     cudaStream_t s)
{
    if (count)
        k_rate_sweep<DIM, KERNEL, EPI_RATE, NT, true><<<blocks, kT, 0, s>>>(Pe, Ce, cs, perm, prm, sp, out);
    else if (epi == EPI_RATE)
        k_rate_sweep<DIM, KERNEL, EPI_RATE, NT, false><<<blocks, kT, 0, s>>>(Pe, Ce, cs, perm, prm, sp, out);
    else if (epi == EPI_PREDICT)
        k_rate_sweep<DIM, KERNEL, EPI_PREDICT, NT, false><<<blocks, kT, 0, s>>>(Pe, Ce, cs, perm, prm, sp, out);
    else
        k_rate_sweep<DIM, KERNEL, EPI_CORRECT, NT, false><<<blocks, kT, 0, s>>>(Pe, Ce, cs, perm, prm, sp, out);
}

template <int DIM, int KERNEL>
void launch_sweep_k(int epi, bool count, int blocks, const uint4 *Pe, const float *Ce, const uint32_t *cs,
                    const uint32_t *perm, const RateParams &prm, const SweepParams &sp, const SweepOut &out,
                    cudaStream_t s)
{
    switch (sp.nt) {
    case 1: launch_sweep_nt<DIM, KERNEL, 1>(epi, count, blocks, Pe, Ce, cs, perm, prm, sp, out, s); break;
    case 2: launch_sweep_nt<DIM, KERNEL, 2>(epi, count, blocks, Pe, Ce, cs, perm, prm, sp, out, s); break;
    case 4: launch_sweep_nt<DIM, KERNEL, 4>(epi, count, blocks, Pe, Ce, cs, perm, prm, sp, out, s); break;
    default: launch_sweep_nt<DIM, KERNEL, 8>(epi, count, blocks, Pe, Ce, cs, perm, prm, sp, out, s); break;
    }
}

}  // namespace

cudaError_t launch_sweep_gather(const uint32_t *perm, const float *C, int n, int P, int P4, float *Cs,
                                cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_sweep_gather<<<(n + kT - 1) / kT, kT, 0, s>>>(perm, C, n, P, P4, Cs);
    return cudaGetLastError();
}

cudaError_t launch_rate_sweep(int dim, int kernel, int epi, bool count, const uint4 *Pe, const float *Ce,
                              const uint32_t *cell_start, const uint32_t *perm, const RateParams &prm,
                              const SweepParams &sp, const SweepOut &out, cudaStream_t s)
{
    if (prm.n == 0) return cudaSuccess;
    if (sp.nt != 1 && sp.nt != 2 && sp.nt != 4 && sp.nt != 8) return cudaErrorInvalidValue;
    const int blocks = (prm.n + kT - 1) / kT;
    if (dim == 2) {
        if (kernel == ADE_WENDLAND_C2)
            launch_sweep_k<2, ADE_WENDLAND_C2>(epi, count, blocks, Pe, Ce, cell_start, perm, prm, sp, out, s);
        else
            launch_sweep_k<2, ADE_WENDLAND_C4>(epi, count, blocks, Pe, Ce, cell_start, perm, prm, sp, out, s);
    } else {
        if (kernel == ADE_WENDLAND_C2)
            launch_sweep_k<3, ADE_WENDLAND_C2>(epi, count, blocks, Pe, Ce, cell_start, perm, prm, sp, out, s);
        else
            launch_sweep_k<3, ADE_WENDLAND_C4>(epi, count, blocks, Pe, Ce, cell_start, perm, prm, sp, out, s);
    }
    return cudaGetLastError();
}

}  // namespace ade
