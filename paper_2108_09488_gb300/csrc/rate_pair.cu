// rate_pair.cu -- the paired walks of the interaction kernel (variants 5-8): two adjacent
// cell-sorted particles per thread, sharing one candidate stream, with the FP32 part of both terms
// of Eq. 4-5 in packed FP32x2 instructions and the predictor / corrector of Eq. 8-9 (Sec. 2.4)
// fused into the epilogue, as in rate.cu.  Branch-free (5, 6) and branched (7, 8) forms, each
// with full (5, 7) or trimmed (6, 8) stencil rows.  Results are bitwise those of the one-target
// walks of rate.cu (see rate_walk.cuh).
#include "ade_internal.h"

namespace ade {

namespace {

#include "rate_common.cuh"
#include "rate_walk.cuh"

// Paired kernel: thread t evaluates sorted particles 2t and 2t + 1; a pair that cannot share a
// candidate stream (can_pair) takes the one-target walk for each particle.  The branch-free
// full-row walk is held to 10 resident CTAs per SM (<= 48 registers), which measured faster on the
// 1024^2 ladder; the trimmed and branched walks are left to the compiler.
template <int DIM, int KERNEL, int EPI, bool ISO, bool TRIM, bool BF>
__global__ __launch_bounds__(kRateThreads, (BF && !TRIM) ? 10 : 0) void k_rate_pair(const uint4 *__restrict__ Pe,
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
    __shared__ TrimRow srow[TRIM ? kMaxRows : 1];
    if (TRIM) stage_trim_rows(srow, prm);
    const bool paired = v1 && can_pair(cx0, cy0, cz0, cx1, cy1, cz1, prm.ncx);
    bool coop = false;   // every lane of the warp holds a pair of one pencil: rows tested once per warp
    if (TRIM) {
        const int cyw = __shfl_sync(0xffffffffu, cy0, 0), czw = __shfl_sync(0xffffffffu, cz0, 0);
        coop = __all_sync(0xffffffffu, paired && cy0 == cyw && cz0 == czw);
    }
    if (paired) {
        rate_direct_pair<DIM, KERNEL, ISO, TRIM, BF>(Pe, cs, pa0, pa1, cx0, cx1, cy0, cz0, prm, r0, r1, srow, coop);
    } else {
        r0 = rate_direct<DIM, KERNEL, ISO, false, BF, TRIM>(Pe, cs, pa0, cx0, cy0, cz0, prm, cnt, srow);
        r1 = v1 ? rate_direct<DIM, KERNEL, ISO, false, BF, TRIM>(Pe, cs, pa1, cx1, cy1, cz1, prm, cnt, srow) : 0.f;
    }
    if (v0) epilogue<DIM, EPI>(i0, r0, pa0, perm, prm, out, acc);
    if (v1) epilogue<DIM, EPI>(i1, r1, pa1, perm, prm, out, acc);
    warp_finish<EPI, false, kRateThreads>(acc, out);
}

template <int DIM, int KERNEL, int EPI>
cudaError_t launch_pair_epi(bool iso, int variant, const uint4 *Pe, const uint4 *Pc, const uint32_t *cs,
                            const uint32_t *perm, const RateParams &prm, const EpiOut &out, cudaStream_t s)
{
    const int blocks = rate_blocks((prm.n + 1) / 2);
    const bool bf = variant == 5 || variant == 6;
    const bool trim = (variant == 6 || variant == 8) && iso;   // trimmed rows: square or cubic boxes
    if (iso) {
        if (bf)
            return trim ? launch_pdl(k_rate_pair<DIM, KERNEL, EPI, true, true, true>, blocks, kRateThreads, 0, s, Pe, Pc, cs, perm, prm, out)
                        : launch_pdl(k_rate_pair<DIM, KERNEL, EPI, true, false, true>, blocks, kRateThreads, 0, s, Pe, Pc, cs, perm, prm, out);
        return trim ? launch_pdl(k_rate_pair<DIM, KERNEL, EPI, true, true, false>, blocks, kRateThreads, 0, s, Pe, Pc, cs, perm, prm, out)
                    : launch_pdl(k_rate_pair<DIM, KERNEL, EPI, true, false, false>, blocks, kRateThreads, 0, s, Pe, Pc, cs, perm, prm, out);
    }
    return bf ? launch_pdl(k_rate_pair<DIM, KERNEL, EPI, false, false, true>, blocks, kRateThreads, 0, s, Pe, Pc, cs, perm, prm, out)
              : launch_pdl(k_rate_pair<DIM, KERNEL, EPI, false, false, false>, blocks, kRateThreads, 0, s, Pe, Pc, cs, perm, prm, out);
}

template <int DIM, int KERNEL>
cudaError_t launch_pair_k(int epi, bool iso, int variant, const uint4 *Pe, const uint4 *Pc, const uint32_t *cs,
                          const uint32_t *perm, const RateParams &prm, const EpiOut &out, cudaStream_t s)
{
    switch (epi) {
    case EPI_RATE: return launch_pair_epi<DIM, KERNEL, EPI_RATE>(iso, variant, Pe, Pc, cs, perm, prm, out, s);
    case EPI_PREDICT: return launch_pair_epi<DIM, KERNEL, EPI_PREDICT>(iso, variant, Pe, Pc, cs, perm, prm, out, s);
    default: return launch_pair_epi<DIM, KERNEL, EPI_CORRECT>(iso, variant, Pe, Pc, cs, perm, prm, out, s);
    }
}

}  // namespace

cudaError_t launch_rate_pair(int dim, int kernel, int epi, bool iso, const uint4 *Pe, const uint4 *Pc,
                             const uint32_t *cs, const uint32_t *perm, const RateParams &prm, const EpiOut &out,
                             cudaStream_t s)
{
    if (prm.n == 0) return cudaSuccess;
    const int v = prm.variant;
    if (dim == 2)
        return kernel == ADE_WENDLAND_C2 ? launch_pair_k<2, ADE_WENDLAND_C2>(epi, iso, v, Pe, Pc, cs, perm, prm, out, s)
                                         : launch_pair_k<2, ADE_WENDLAND_C4>(epi, iso, v, Pe, Pc, cs, perm, prm, out, s);
    return kernel == ADE_WENDLAND_C2 ? launch_pair_k<3, ADE_WENDLAND_C2>(epi, iso, v, Pe, Pc, cs, perm, prm, out, s)
                                     : launch_pair_k<3, ADE_WENDLAND_C4>(epi, iso, v, Pe, Pc, cs, perm, prm, out, s);
}

}  // namespace ade
