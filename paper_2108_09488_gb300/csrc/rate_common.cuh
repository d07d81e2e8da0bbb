// rate_common.cuh -- device helpers shared by the interaction kernels (rate.cu, rate_field.cu):
// compensated row summation, the kernel shape factor f(q) of W'(r)/r = kc f(q), and the
// warp-wide epilogue reductions of the fused corrector (pair count, per-warp {sum, min, max} of
// C).  Included inside an unnamed namespace of ade.
#pragma once

// 1/sqrt(x) from the special-function unit with subnormal inputs flushed to zero.  The walks take
// it of r^2 in fixed-point units, which is 0 (the particle itself) or at least 1, never subnormal.
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Compensated summation (Neumaier's scheme): sum += x, with the rounding error of that addition
// accumulated in comp.  The error is taken with Knuth's branch-free two-sum, which yields exactly
// (sum + x) - fl(sum + x), the same value as the magnitude-ordered form, in six FP32 additions.
// Minimum-image separation of two fixed-point words as an FP32 value: the int32 difference a - b
// as the multiply-add a + m b with m = -1 read at run time (so it stays an integer multiply-add,
// which this architecture issues to the FMA pipe rather than the ALU pipe), converted with
// round-to-nearest.
__device__ __forceinline__ float sep(uint32_t a, uint32_t b, int m)
{
    return (float)((int)a + m * (int)b);
}

__device__ __forceinline__ void neumaier_add(float &sum, float &comp, float x)
{
    const float t = sum + x;
    const float bp = t - sum;
    comp += (sum - (t - bp)) + (x - bp);
    sum = t;
}

// The walks clamp 1 - q at 0 as om + |om| = 2 max(om, 0) (one FP32 addition); the kernel shape
// of twice the argument is an exact power-of-two multiple of the shape, undone once per particle.
template <int KERNEL>
__device__ __forceinline__ float shape_unscale()
{
    return KERNEL == ADE_WENDLAND_C2 ? 0.125f : 0.03125f;   // 1 / 2^3, 1 / 2^5
}

// Kernel shape factor f(q) with W'(r)/r = kc f(q); omq = 1 - q (clamped at 0 by the caller for the
// branch-free form).  shape2x takes 2 (1 - q) and returns 2^3 f (C2) or 2^5 f (C4) exactly.
template <int KERNEL>
__device__ __forceinline__ float shape(float omq)
{
    if (KERNEL == ADE_WENDLAND_C2) return omq * omq * omq;
    float o2 = omq * omq;
    return o2 * o2 * omq * fmaf(-5.f, omq, 6.f);  // (1-q)^5 (1 + 5q), 1 + 5q = 6 - 5(1-q)
}

template <int KERNEL>
__device__ __forceinline__ float shape2x(float w)
{
    if (KERNEL == ADE_WENDLAND_C2) return w * w * w;
    float o2 = w * w;
    return o2 * o2 * w * fmaf(-2.5f, w, 6.f);      // (2(1-q))^5 (6 - 5(1-q))
}

// Per-thread accumulators of the corrector's reductions: the sum of C as an unevaluated FP32 pair
// hi + lo kept with Knuth's error-free two-sum (converted to FP64 only by the grid-wide fold, so
// the FP64 pipe, which is scarce on this part, is not used in the rate kernels), FP32 min and max
// (exact: the values are FP32), in-support pair count.
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

// Warp-wide part of the epilogue: pair count, and for the corrector one partial per warp
// {hi, lo, min, max} of its particles' new C, folded by a fixed shuffle tree (error-free two-sum
// for the sum, exact FP32 min and max).  No block barrier, fence or atomic: the grid-wide fold
// is a separate one-block launch that follows on the stream (launch_fold_warp_partials).  Every
// thread of the warp must call it.
template <int EPI, bool COUNT, int NT>
__device__ __forceinline__ void warp_finish(Acc acc, const EpiOut &out)
{
    if (COUNT) {
        unsigned c = acc.cnt;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if ((threadIdx.x & 31) == 0 && c) atomicAdd(out.pairs, (unsigned long long)c);
    }
    if (EPI != EPI_CORRECT) return;
    float mn = acc.mn, mx = acc.mx, hi = acc.hi, lo = acc.lo;
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_down_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
        const float h2 = __shfl_down_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_down_sync(0xffffffffu, lo, o);
        two_sum_add(hi, lo, h2, l2);
    }
    if ((threadIdx.x & 31) == 0)
        out.wpart[(size_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5)] = make_float4(hi, lo, mn, mx);
}
