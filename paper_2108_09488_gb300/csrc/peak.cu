// peak.cu -- measured issue rates of the two pipes the pair term runs on: FP32 fused multiply-add
// (FFMA) and the multi-function unit's reciprocal square root (MUFU.RSQ).  They turn the pair
// kernels' instruction counts into time: the ALU roof of the interaction kernels is
// (FP32 lanes x clock) / (FP32-pipe instructions per pair), and this probe checks the lane count
// and clock on the device at hand.
//
// Each thread runs 8 independent dependency chains (enough to cover the pipe latency at full
// occupancy) for `iters` rounds; the grid fills every SM several times over.  The results are
// written only when a value no input can produce appears, so the compiler keeps the work.
#include "ade_internal.h"

namespace ade {

namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;

__global__ __launch_bounds__(kPeakThreads) void k_ffma_probe(float seed, int iters, float *sink)
{
    float a[kChains];
    const float b = 0.999999f, c = 1e-7f * (float)(threadIdx.x & 7);
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed + (float)k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.0f) sink[blockIdx.x * kPeakThreads + threadIdx.x] = s;
}

__global__ __launch_bounds__(kPeakThreads) void k_rsqrt_probe(float seed, int iters, float *sink)
{
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed + (float)k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = rsqrtf(a[k]);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.0f) sink[blockIdx.x * kPeakThreads + threadIdx.x] = s;
}

}  // namespace

}  // namespace ade

extern "C" int ade_alu_peaks(double *ffma_per_s_host, double *rsqrt_per_s_host, void *stream)
{
    if (!ffma_per_s_host || !rsqrt_per_s_host) return ade::report_error(ADE_ERR_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return ade::report_error(ADE_ERR_CUDA, cudaGetErrorString(e));
    const int blocks = sms * 8;
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&sink, (size_t)blocks * ade::kPeakThreads * sizeof(float));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double rate[2] = {0.0, 0.0};
    for (int kind = 0; kind < 2 && e == cudaSuccess; ++kind) {
        const int iters = kind == 0 ? 2048 : 256;
        float best = 1e30f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // first round warms up the clocks
            e = cudaEventRecord(e0, s);
            if (kind == 0)
                ade::k_ffma_probe<<<blocks, ade::kPeakThreads, 0, s>>>(1.0f, iters, sink);
            else
                ade::k_rsqrt_probe<<<blocks, ade::kPeakThreads, 0, s>>>(1.5f, iters, sink);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && rep > 0) best = ms < best ? ms : best;
        }
        const double ops = (double)blocks * ade::kPeakThreads * iters * 16.0 * ade::kChains;
        rate[kind] = ops / (best * 1e-3);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) return ade::report_error(ADE_ERR_CUDA, cudaGetErrorString(e));
    *ffma_per_s_host = rate[0];
    *rsqrt_per_s_host = rate[1];
    return ADE_OK;
}
