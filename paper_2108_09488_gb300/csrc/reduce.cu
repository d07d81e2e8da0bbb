// reduce.cu -- FP64 reductions of the particle state and the closed-form error norms.
//
//   * k_fold_warp_partials: deterministic fixed-order fold of the per-warp partials written by
//     the corrector epilogue: sum C (the host multiplies by m for sum m C), min C, max C.
//   * k_state_partials + k_reduce_final: the same statistics of any concentration array.
//   * k_closed_form_err: the closed form of Sec. 3 (Eq. 12-13 in 2D; the same Gaussian in 3D) at
//     every particle, C_an = C0 w^d / sqrt(det S) sum_images exp(-1/2 xi^T S^-1 xi),
//     S = w^2 I + 2 t D, xi = x - (x0 + v t) + image shift, and the per-block partials of
//     sum (C - C_an)^2, max |C - C_an| and max |C_an| (error norms of Table 2 and Figs. 5, 7).
// Both run in FP64: they are off the per-pair path and read each particle once.
#include <cooperative_groups.h>

#include "ade_internal.h"

namespace ade {

namespace {

constexpr int kRedThreads = 256;

__device__ __forceinline__ double dinf() { return __longlong_as_double(0x7ff0000000000000ll); }

// partials: [nblocks][3]; ops: slot 0 sum, slot 1 min (or max when max_slot1), slot 2 max.
__global__ __launch_bounds__(kRedThreads) void k_reduce_final(const double *__restrict__ partials,
                                                              int nblocks, int max_slot1,
                                                              double *__restrict__ out)
{
    __shared__ double sh[3][kRedThreads];
    double a = 0.0, b = max_slot1 ? -dinf() : dinf(), c = -dinf();
    for (int k = threadIdx.x; k < nblocks; k += kRedThreads) {
        a += partials[3 * (size_t)k + 0];
        double pb = partials[3 * (size_t)k + 1];
        b = max_slot1 ? fmax(b, pb) : fmin(b, pb);
        c = fmax(c, partials[3 * (size_t)k + 2]);
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    sh[2][threadIdx.x] = c;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] = max_slot1 ? fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + o])
                                           : fmin(sh[1][threadIdx.x], sh[1][threadIdx.x + o]);
            sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sh[0][0];
        out[1] = sh[1][0];
        out[2] = sh[2][0];
    }
}

// Fold of the corrector's m per-warp partials {hi, lo, min, max} by one thread-block cluster of
// G <= 8 CTAs (G fixed by m alone).  CTA r folds the contiguous chunk [r chunk, (r + 1) chunk):
// thread t takes partials t, t + T, ... in order (up to eight loads in flight) with the error-free
// two-sum in FP32, then a fixed shuffle tree per warp; warp 0 of the CTA folds its warps' results
// by the same tree; CTA 0 reads the G CTA results through distributed shared memory and folds
// them in CTA order.  Only the final hi + lo is formed in FP64: dependent FP64 operations are slow
// on this part.  No fence or atomic; the order does not depend on timing.
constexpr int kFoldThreads = 1024;
constexpr int kFoldPerCta = 1024;   // partials per CTA before another CTA of the cluster is used
static_assert(kFoldMaxCtas <= 32, "CTA 0 folds one CTA result per lane of one warp");
static_assert(kFoldThreads == 32 * 32, "warp 0 folds one result per warp of the CTA");

__device__ __forceinline__ void fold_two_sum(float &hi, float &lo, float x, float xlo)
{
    const float s = hi + x;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (x - bb);
    hi = s;
    lo = lo + (err + xlo);
}

// Fixed shuffle tree over the 32 lanes of {hi, lo, min, max}; lane 0 holds the result.
__device__ __forceinline__ float4 fold_warp(float4 r)
{
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, r.x, o);
        const float l2 = __shfl_down_sync(0xffffffffu, r.y, o);
        r.z = fminf(r.z, __shfl_down_sync(0xffffffffu, r.z, o));
        r.w = fmaxf(r.w, __shfl_down_sync(0xffffffffu, r.w, o));
        fold_two_sum(r.x, r.y, h2, l2);
    }
    return r;
}

__global__ __launch_bounds__(kFoldThreads) void k_fold_warp_partials(const float4 *__restrict__ wp, int m,
                                                                     int chunk, double *__restrict__ stats)
{
    pdl_wait();
    pdl_trigger();
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ float4 wres[kFoldThreads / 32];
    __shared__ float4 cres;
    const float inf = __int_as_float(0x7f800000);
    const int rank = (int)cluster.block_rank();
    const int b0 = rank * chunk;
    const int b1 = min(m, b0 + chunk);
    float hi = 0.f, lo = 0.f, mn = inf, mx = -inf;
    constexpr int U = 8;
    for (int k0 = b0 + (int)threadIdx.x; k0 < b1; k0 += U * kFoldThreads) {
        float4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = k0 + u * kFoldThreads;
            v[u] = k < b1 ? __ldcg(wp + k) : make_float4(0.f, 0.f, inf, -inf);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            fold_two_sum(hi, lo, v[u].x, v[u].y);
            mn = fminf(mn, v[u].z);
            mx = fmaxf(mx, v[u].w);
        }
    }
    const float4 w = fold_warp(make_float4(hi, lo, mn, mx));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) wres[wid] = w;
    __syncthreads();
    if (wid == 0) {
        const float4 r = fold_warp(wres[lane]);   // kFoldThreads / 32 == 32 warps
        if (lane == 0) cres = r;
    }
    cluster.sync();
    if (rank == 0 && wid == 0) {
        const int G = (int)cluster.num_blocks();
        float4 r = make_float4(0.f, 0.f, inf, -inf);
        if (lane < G) r = *cluster.map_shared_rank(&cres, lane);
        r = fold_warp(r);
        if (lane == 0) {
            stats[0] = (double)r.x + (double)r.y;
            stats[1] = (double)r.z;
            stats[2] = (double)r.w;
        }
    }
    cluster.sync();   // CTA 0 has read every CTA's result before any CTA exits
}

struct CFParams {
    double box[3];
    double center[3];
    double Sinv[9];
    double amp;   // C0 w^d / sqrt(det S)
    int nimg;
};

template <int DIM>
__global__ __launch_bounds__(kRedThreads) void k_closed_form_err(const uint32_t *__restrict__ xq,
                                                                 const float *__restrict__ C, int n,
                                                                 const CFParams prm,
                                                                 double *__restrict__ partials)
{
    const int i = blockIdx.x * kRedThreads + threadIdx.x;
    double e2 = 0.0, emax = 0.0, amax = 0.0;
    if (i < n) {
        double xi0[3] = {0.0, 0.0, 0.0};
        for (int d = 0; d < DIM; ++d) {
            double u = (double)xq[(size_t)d * n + i] * (prm.box[d] * 2.3283064365386963e-10);
            double dd = u - prm.center[d];
            dd -= prm.box[d] * rint(dd / prm.box[d]);
            xi0[d] = dd;
        }
        double s = 0.0;
        const int lz = DIM == 3 ? prm.nimg : 0;
        for (int iz = -lz; iz <= lz; ++iz)
            for (int iy = -prm.nimg; iy <= prm.nimg; ++iy)
                for (int ix = -prm.nimg; ix <= prm.nimg; ++ix) {
                    double X[3] = {xi0[0] + ix * prm.box[0], xi0[1] + iy * prm.box[1],
                                   DIM == 3 ? xi0[2] + iz * prm.box[2] : 0.0};
                    double quad = 0.0;
                    for (int a = 0; a < DIM; ++a)
                        for (int b = 0; b < DIM; ++b) quad += X[a] * prm.Sinv[a * 3 + b] * X[b];
                    s += exp(-0.5 * quad);
                }
        double can = prm.amp * s;
        double e = (double)C[i] - can;
        e2 = e * e;
        emax = fabs(e);
        amax = fabs(can);
    }
    for (int o = 16; o > 0; o >>= 1) {
        e2 += __shfl_down_sync(0xffffffffu, e2, o);
        emax = fmax(emax, __shfl_down_sync(0xffffffffu, emax, o));
        amax = fmax(amax, __shfl_down_sync(0xffffffffu, amax, o));
    }
    __shared__ double red[3][kRedThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = e2;
        red[1][wid] = emax;
        red[2][wid] = amax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) {
            a += red[0][w];
            b = fmax(b, red[1][w]);
            c = fmax(c, red[2][w]);
        }
        partials[3 * (size_t)blockIdx.x + 0] = a;
        partials[3 * (size_t)blockIdx.x + 1] = b;
        partials[3 * (size_t)blockIdx.x + 2] = c;
    }
}

// Per-block {sum C, min C, max C} of the caller's concentrations.
__global__ __launch_bounds__(kRedThreads) void k_state_partials(const float *__restrict__ C, int n,
                                                                double *__restrict__ partials)
{
    const int i = blockIdx.x * kRedThreads + threadIdx.x;
    double s = 0.0, mn = dinf(), mx = -dinf();
    if (i < n) {
        s = (double)C[i];
        mn = s;
        mx = s;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    __shared__ double red[3][kRedThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = s;
        red[1][wid] = mn;
        red[2][wid] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = red[0][0], b = red[1][0], c = red[2][0];
        for (int w = 1; w < kRedThreads / 32; ++w) {
            a += red[0][w];
            b = fmin(b, red[1][w]);
            c = fmax(c, red[2][w]);
        }
        partials[3 * (size_t)blockIdx.x + 0] = a;
        partials[3 * (size_t)blockIdx.x + 1] = b;
        partials[3 * (size_t)blockIdx.x + 2] = c;
    }
}

// One block per plume: FP64 {sum C, min C, max C} over the plume's caller range, fixed order.
__global__ __launch_bounds__(kRedThreads) void k_batch_stats(const float *__restrict__ C,
                                                             const int *__restrict__ offsets,
                                                             double *__restrict__ stats)
{
    const int p = blockIdx.x;
    const int lo = offsets[p], hi = offsets[p + 1];
    double s = 0.0, mn = dinf(), mx = -dinf();
    for (int i = lo + threadIdx.x; i < hi; i += kRedThreads) {
        const double v = (double)C[i];
        s += v;
        mn = fmin(mn, v);
        mx = fmax(mx, v);
    }
    __shared__ double sh[3][kRedThreads];
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = mn;
    sh[2][threadIdx.x] = mx;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] = fmin(sh[1][threadIdx.x], sh[1][threadIdx.x + o]);
            sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        stats[3 * p + 0] = sh[0][0];
        stats[3 * p + 1] = sh[1][0];
        stats[3 * p + 2] = sh[2][0];
    }
}

}  // namespace

cudaError_t launch_batch_stats(const float *C, const int *offsets, int nplumes, double *stats,
                               cudaStream_t s)
{
    if (nplumes > 0) k_batch_stats<<<nplumes, kRedThreads, 0, s>>>(C, offsets, stats);
    return cudaGetLastError();
}

cudaError_t launch_state_stats(const float *C, int n, double *partials, double *stats, cudaStream_t s)
{
    int nb = (n + kRedThreads - 1) / kRedThreads;
    if (nb > 0) k_state_partials<<<nb, kRedThreads, 0, s>>>(C, n, partials);
    k_reduce_final<<<1, kRedThreads, 0, s>>>(partials, nb, 0, stats);
    return cudaGetLastError();
}

int closed_form_blocks(int n) { return (n + kRedThreads - 1) / kRedThreads; }

cudaError_t launch_fold_warp_partials(const float4 *wpart, int m, double *stats, cudaStream_t s)
{
    if (m <= 0) return cudaSuccess;
    int G = (m + kFoldPerCta - 1) / kFoldPerCta;
    if (G > kFoldMaxCtas) G = kFoldMaxCtas;
    const int chunk = (m + G - 1) / G;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)G, 1, 1);
    cfg.blockDim = dim3(kFoldThreads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // see pdl_wait
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, k_fold_warp_partials, wpart, m, chunk, stats);
}

cudaError_t launch_closed_form_error(int dim, const uint32_t *xq, const float *C, int n,
                                     const double *box, const double *center, const double *Sinv,
                                     double amp, double C0, double vol, int nimg,
                                     double *partials, int nblocks, double *out, cudaStream_t s)
{
    (void)C0;
    (void)vol;
    CFParams prm;
    for (int d = 0; d < 3; ++d) {
        prm.box[d] = box[d];
        prm.center[d] = center[d];
    }
    for (int k = 0; k < 9; ++k) prm.Sinv[k] = Sinv[k];
    prm.amp = amp;
    prm.nimg = nimg;
    if (nblocks > 0) {
        if (dim == 2)
            k_closed_form_err<2><<<nblocks, kRedThreads, 0, s>>>(xq, C, n, prm, partials);
        else
            k_closed_form_err<3><<<nblocks, kRedThreads, 0, s>>>(xq, C, n, prm, partials);
    }
    k_reduce_final<<<1, kRedThreads, 0, s>>>(partials, nblocks, 1, out);
    return cudaGetLastError();
}

}  // namespace ade
