// rate.cu -- the neighbour-interaction kernel: Eq. 4-5 (Sec. 2.2) for every particle, with the
// predictor and corrector of Eq. 8-9 (Sec. 2.4) fused into its epilogue.
//
// For a uniform velocity field (Sec. 3) every particle carries the same tensor D (Eq. 3), so the
// per-component harmonic mean of Eq. 5 is 4 D D / (D + D) = 2 D and the pair factor reduces to
//     Dcal_ab = Gamma x_ab^T K x_ab / r^2 - tr K,   K = 2 D,
// evaluated as x^T (Gamma K - Gamma K_zz I) x / r^2 + (Gamma K_zz - tr K) (K_yy in 2D), which
// drops the diagonal term of the last axis from the per-pair work.
// With grad_a W = W'(r) x_ab / r, the dispersive term of Eq. 4 for one ordered pair is
//     1/2 (m_b / rhobar) Dcal_ab (C_a - C_b) W'(r) / r,
// and W'(r)/r = kc f(q): Wendland C2 (support H = 2h): f = (1-q)^3, kc = -20 B / H^2;
// Wendland C4 (Eq. 7, support H = h): f = (1-q)^5 (1+5q), kc = -(56/3) B / H^2.
// The convective term of Eq. 4 is identically zero for uniform v and is not evaluated.
//
// Layout and arithmetic:
//   * one thread per particle in cell-sorted order; the particle's cell comes from the cell-build
//     positions, its pair terms from the evaluation positions (they differ by the half-step drift);
//   * candidates are read as one 16-byte word {x, y, z, C} from the sorted copy; each stencil row
//     (2w+1 cells with consecutive keys) is one contiguous index range, two at a periodic seam;
//   * separations are int32 differences of fixed-point words converted to FP32, so the minimum
//     image and translation invariance are exact; pair arithmetic is FP32;
//   * each row's terms are summed in FP32 and the row sums are added with Neumaier's compensated
//     summation, in a fixed order (rows, then sorted index), so results are deterministic.
#include "ade_internal.h"

namespace ade {

namespace {

__device__ __forceinline__ void neumaier_add(float &sum, float &comp, float x)
{
    float t = sum + x;
    if (fabsf(sum) >= fabsf(x))
        comp += (sum - t) + x;
    else
        comp += (x - t) + sum;
    sum = t;
}

template <int DIM, int KERNEL, bool ISO, bool COUNT>
__device__ __forceinline__ void pair_range(const uint4 *__restrict__ P, int j0, int j1, const uint4 &pa,
                                           float Ca, const RateParams &prm, float &rs, unsigned &cnt)
{
    for (int j = j0; j < j1; ++j) {
        uint4 pb = __ldg(P + j);
        float dx = (float)(int)(pa.x - pb.x);
        float dy = (float)(int)(pa.y - pb.y);
        float dz = 0.f;
        if (DIM == 3) dz = (float)(int)(pa.z - pb.z);
        if (!ISO) {
            dy *= prm.sy;
            if (DIM == 3) dz *= prm.sz;
        }
        float r2 = fmaf(dx, dx, dy * dy);
        if (DIM == 3) r2 = fmaf(dz, dz, r2);
        if (r2 < prm.H2 && r2 > 0.f) {
            float rinv = rsqrtf(r2);
            float r = r2 * rinv;
            float f;
            if (KERNEL == ADE_WENDLAND_C2) {
                float omq = fmaf(-r, prm.invH, 1.f);
                f = omq * omq * omq;
            } else {
                float q = r * prm.invH;
                float omq = 1.f - q;
                float o2 = omq * omq;
                f = o2 * o2 * omq * fmaf(5.f, q, 1.f);
            }
            // Gamma x^T K x = Gamma K_last r^2 + x^T (Gamma K - Gamma K_last I) x: the r^2 part
            // is folded into the constant c0 = Gamma K_last - tr K.
            float Q;
            if (DIM == 2) {
                Q = dx * fmaf(prm.Kc[0], dx, prm.Kc[3] * dy);
            } else {
                float qx = fmaf(prm.Kc[0], dx, fmaf(prm.Kc[3], dy, prm.Kc[4] * dz));
                float qy = fmaf(prm.Kc[1], dy, prm.Kc[5] * dz);
                Q = fmaf(dx, qx, dy * qy);
            }
            float sfac = fmaf(Q, rinv * rinv, prm.c0);
            rs = fmaf(f * sfac, Ca - __uint_as_float(pb.w), rs);
            if (COUNT) ++cnt;
        }
    }
}

template <int DIM, int KERNEL, int EPI, bool ISO, bool COUNT>
__global__ __launch_bounds__(kRateThreads) void k_rate(const uint4 *__restrict__ Pe,
                                                       const uint4 *__restrict__ Pc,
                                                       const uint32_t *__restrict__ cs,
                                                       const uint32_t *__restrict__ perm,
                                                       const RateParams prm, const EpiOut out)
{
    const int i = blockIdx.x * kRateThreads + threadIdx.x;
    const bool valid = i < prm.n;
    const int ii = valid ? i : prm.n - 1;
    const uint4 pa = __ldg(Pe + ii);
    const uint4 pc = (Pe == Pc) ? pa : __ldg(Pc + ii);
    const int ncx = prm.ncx, ncy = prm.ncy, ncz = prm.ncz;
    const int cx = (int)__umulhi(pc.x, (uint32_t)ncx);
    const int cy = (int)__umulhi(pc.y, (uint32_t)ncy);
    const int cz = DIM == 3 ? (int)__umulhi(pc.z, (uint32_t)ncz) : 0;
    const float Ca = __uint_as_float(pa.w);

    float acc = 0.f, comp = 0.f;
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
        pair_range<DIM, KERNEL, ISO, COUNT>(Pe, s0, e0, pa, Ca, prm, rs, cnt);
        pair_range<DIM, KERNEL, ISO, COUNT>(Pe, s1, e1, pa, Ca, prm, rs, cnt);
        neumaier_add(acc, comp, rs);
    }
    const float rate = prm.pf * (acc + comp);

    if (COUNT) {
        unsigned c = valid ? cnt : 0u;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if ((threadIdx.x & 31) == 0 && c) atomicAdd(out.pairs, (unsigned long long)c);
    }

    if (EPI == EPI_RATE) {
        if (valid && out.rate) {
            const uint32_t a = __ldg(perm + i);
            if (a < (uint32_t)prm.n) out.rate[a] = rate;
        }
    } else if (EPI == EPI_PREDICT) {
        if (valid) {
            uint4 q;
            q.x = pa.x + prm.inc[0];
            q.y = pa.y + prm.inc[1];
            q.z = pa.z + prm.inc[2];
            q.w = __float_as_uint(fmaf(prm.dt, rate, Ca));
            out.Pout[i] = q;
        }
    } else {
        // corrector: C^{l+1} = C^l + dt r^{l+1/2}, x^{l+1} = x^l + dt v, back to caller order
        double s = 0.0, mn = __longlong_as_double(0x7ff0000000000000ll), mx = -mn;
        if (valid) {
            const float Cl = __uint_as_float(pc.w);
            const float Cn = fmaf(prm.dt, rate, Cl);
            const uint32_t a = __ldg(perm + i);
            if (a < (uint32_t)prm.n) {
                out.C[a] = Cn;
                out.xq[a] = pc.x + prm.inc[0];
                out.xq[(size_t)prm.n + a] = pc.y + prm.inc[1];
                if (DIM == 3) out.xq[2 * (size_t)prm.n + a] = pc.z + prm.inc[2];
            }
            if (!isfinite(Cn)) atomicOr(out.status, 1);
            s = (double)Cn;
            mn = s;
            mx = s;
        }
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_down_sync(0xffffffffu, s, o);
            mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
            mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
        }
        __shared__ double red[3][kRateThreads / 32];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) {
            red[0][wid] = s;
            red[1][wid] = mn;
            red[2][wid] = mx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = red[0][0], b = red[1][0], c = red[2][0];
            for (int w = 1; w < kRateThreads / 32; ++w) {
                a += red[0][w];
                b = fmin(b, red[1][w]);
                c = fmax(c, red[2][w]);
            }
            out.partials[3 * (size_t)blockIdx.x + 0] = a;
            out.partials[3 * (size_t)blockIdx.x + 1] = b;
            out.partials[3 * (size_t)blockIdx.x + 2] = c;
        }
    }
}

template <int DIM, int KERNEL, bool ISO, bool COUNT>
cudaError_t launch_epi(int epi, int blocks, const uint4 *Pe, const uint4 *Pc, const uint32_t *cs,
                       const uint32_t *perm, const RateParams &prm, const EpiOut &out, cudaStream_t s)
{
    switch (epi) {
    case EPI_RATE:
        k_rate<DIM, KERNEL, EPI_RATE, ISO, COUNT><<<blocks, kRateThreads, 0, s>>>(Pe, Pc, cs, perm, prm, out);
        break;
    case EPI_PREDICT:
        k_rate<DIM, KERNEL, EPI_PREDICT, ISO, COUNT><<<blocks, kRateThreads, 0, s>>>(Pe, Pc, cs, perm, prm, out);
        break;
    default:
        k_rate<DIM, KERNEL, EPI_CORRECT, ISO, COUNT><<<blocks, kRateThreads, 0, s>>>(Pe, Pc, cs, perm, prm, out);
        break;
    }
    return cudaGetLastError();
}

template <int DIM, int KERNEL>
cudaError_t launch_dk(bool iso, bool count, int epi, int blocks, const uint4 *Pe, const uint4 *Pc,
                      const uint32_t *cs, const uint32_t *perm, const RateParams &prm,
                      const EpiOut &out, cudaStream_t s)
{
    if (iso) {
        return count ? launch_epi<DIM, KERNEL, true, true>(epi, blocks, Pe, Pc, cs, perm, prm, out, s)
                     : launch_epi<DIM, KERNEL, true, false>(epi, blocks, Pe, Pc, cs, perm, prm, out, s);
    }
    return count ? launch_epi<DIM, KERNEL, false, true>(epi, blocks, Pe, Pc, cs, perm, prm, out, s)
                 : launch_epi<DIM, KERNEL, false, false>(epi, blocks, Pe, Pc, cs, perm, prm, out, s);
}

}  // namespace

int rate_blocks(int n) { return (n + kRateThreads - 1) / kRateThreads; }

cudaError_t launch_rate(int dim, int kernel, bool iso, int epi, const uint4 *Pe, const uint4 *Pc,
                        const uint32_t *cell_start, const uint32_t *perm, const RateParams &prm,
                        const EpiOut &out, cudaStream_t s)
{
    const int blocks = rate_blocks(prm.n);
    if (blocks == 0) return cudaSuccess;
    const bool count = out.pairs != nullptr;
    if (dim == 2)
        return kernel == ADE_WENDLAND_C2
                   ? launch_dk<2, ADE_WENDLAND_C2>(iso, count, epi, blocks, Pe, Pc, cell_start, perm, prm, out, s)
                   : launch_dk<2, ADE_WENDLAND_C4>(iso, count, epi, blocks, Pe, Pc, cell_start, perm, prm, out, s);
    return kernel == ADE_WENDLAND_C2
               ? launch_dk<3, ADE_WENDLAND_C2>(iso, count, epi, blocks, Pe, Pc, cell_start, perm, prm, out, s)
               : launch_dk<3, ADE_WENDLAND_C4>(iso, count, epi, blocks, Pe, Pc, cell_start, perm, prm, out, s);
}

}  // namespace ade
