// rate_common.cuh -- device helpers shared by the interaction kernels (rate.cu, rate_field.cu):
// compensated row summation, the kernel shape factor f(q) of W'(r)/r = kc f(q), and the
// block-wide epilogue reductions of the fused corrector (pair count, FP64 {sum, min, max} of C
// with a last-block fixed-order fold).  Included inside an unnamed namespace of ade.
#pragma once

__device__ __forceinline__ void neumaier_add(float &sum, float &comp, float x)
{
    float t = sum + x;
    if (fabsf(sum) >= fabsf(x))
        comp += (sum - t) + x;
    else
        comp += (x - t) + sum;
    sum = t;
}

__device__ __forceinline__ double dinf() { return __longlong_as_double(0x7ff0000000000000ll); }

// Kernel shape factor f(q) with W'(r)/r = kc f(q); omq = 1 - q (clamped at 0 by the caller for the
// branch-free form).
template <int KERNEL>
__device__ __forceinline__ float shape(float omq)
{
    if (KERNEL == ADE_WENDLAND_C2) return omq * omq * omq;
    float o2 = omq * omq;
    return o2 * o2 * omq * fmaf(-5.f, omq, 6.f);  // (1-q)^5 (1 + 5q), 1 + 5q = 6 - 5(1-q)
}

// Per-thread accumulators of the corrector's reductions: the sum of C as an unevaluated FP32 pair
// hi + lo kept with Knuth's error-free two-sum (converted to FP64 once per warp, so the FP64 pipe,
// which is scarce on this part, sees a few instructions per warp), FP32 min and max (exact: the
// values are FP32), in-support pair count.
struct Acc {
    float hi, lo;
    float mn, mx;
    unsigned cnt;
};

__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float x, float xlo)
{
    const float s = hi + x;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (x - bb);
    hi = s;
    lo = lo + (err + xlo);
}

// Fixed-order reduction of nb partial triples {sum, min, max} by one block of NT threads.  Thread
// t folds partials t, t + NT, t + 2 NT, ... in that order; the loads are issued 16 at a time so
// that they are in flight together.
template <int NT>
__device__ void reduce_partials_last_block(const double *partials, int nb, double *stats)
{
    __shared__ double sh[3][NT];
    constexpr int U = 16;
    double a = 0.0, b = dinf(), c = -dinf();
    for (int k0 = threadIdx.x; k0 < nb; k0 += U * NT) {
        double va[U], vb[U], vc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int k = k0 + u * NT;
            const bool ok = k < nb;
            va[u] = ok ? __ldcg(partials + 3 * (size_t)k + 0) : 0.0;
            vb[u] = ok ? __ldcg(partials + 3 * (size_t)k + 1) : dinf();
            vc[u] = ok ? __ldcg(partials + 3 * (size_t)k + 2) : -dinf();
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            a += va[u];
            b = fmin(b, vb[u]);
            c = fmax(c, vc[u]);
        }
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    sh[2][threadIdx.x] = c;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] = fmin(sh[1][threadIdx.x], sh[1][threadIdx.x + o]);
            sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        stats[0] = sh[0][0];
        stats[1] = sh[1][0];
        stats[2] = sh[2][0];
    }
}

// Block-wide part of the epilogue: pair count, and for the corrector the per-block partials and
// the last block's final reduction.  Every thread of the block must call it.
template <int EPI, bool COUNT, int NT>
__device__ __forceinline__ void block_finish(Acc acc, const EpiOut &out)
{
    if (COUNT) {
        unsigned c = acc.cnt;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if ((threadIdx.x & 31) == 0 && c) atomicAdd(out.pairs, (unsigned long long)c);
    }
    if (EPI != EPI_CORRECT) return;
    // min and max: FP32 warp shuffles (exact).  Sum: the (hi, lo) pairs are combined by a fixed
    // shuffle tree with the error-free two-sum, then converted to FP64 by lane 0.
    float mn = acc.mn, mx = acc.mx, hi = acc.hi, lo = acc.lo;
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_down_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
        const float h2 = __shfl_down_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_down_sync(0xffffffffu, lo, o);
        two_sum_add(hi, lo, h2, l2);
    }
    __shared__ double red[3][NT / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = (double)hi + (double)lo;
        red[1][wid] = (double)mn;
        red[2][wid] = (double)mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = red[0][0], b = red[1][0], c = red[2][0];
        for (int w = 1; w < NT / 32; ++w) {
            a += red[0][w];
            b = fmin(b, red[1][w]);
            c = fmax(c, red[2][w]);
        }
        out.partials[3 * (size_t)blockIdx.x + 0] = a;
        out.partials[3 * (size_t)blockIdx.x + 1] = b;
        out.partials[3 * (size_t)blockIdx.x + 2] = c;
        __threadfence();
        last = atomicAdd(out.done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        // the last block to finish reduces every block's partials in a fixed order
        __threadfence();
        reduce_partials_last_block<NT>(out.partials, gridDim.x, out.stats);
        if (threadIdx.x == 0) *out.done = 0u;
    }
}
