// Throughput microbenchmarks of the arithmetic pipes that bound the property
// kernels: FP64 FMA (the FP64 paths), FP32 FMA and the special-function unit
// (exp2) of the FP32 paths.  Each thread runs eight independent dependency
// chains, enough warps per SM to cover the pipe latency; the result is kept
// alive by a store that a comparison with an impossible value guards.  They
// give the roofline denominators measured on the device the library runs on.
#include <cuda_runtime.h>

#include "pr_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kPeakBlock = 256;

__global__ void __launch_bounds__(kPeakBlock) dfma_kernel(double *sink, int iters, double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.2345e300) sink[0] = s;
}

__global__ void __launch_bounds__(kPeakBlock) ffma_kernel(float *sink, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.2345e30f) sink[0] = s;
}

__device__ __forceinline__ float ex2_approx(float v)
{
    float r;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

__global__ void __launch_bounds__(kPeakBlock) ex2_kernel(float *sink, int iters)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = -1e-3f * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = -ex2_approx(x[c]);   // stays in [-1, -0.5]
    }
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.2345e30f) sink[0] = s;
}

}  // namespace

extern "C" pr_status pr_measure_peak(int kind, double *ops_per_s)
{
    PR_CHECK_ARG(ops_per_s != nullptr, "pr_measure_peak: null output");
    PR_CHECK_ARG(kind == PR_PEAK_FP64_FMA || kind == PR_PEAK_FP32_FMA || kind == PR_PEAK_MUFU_EX2,
                 "pr_measure_peak: unknown kind %d", kind);
    int dev = 0, sms = 0;
    PR_CUDA_TRY(cudaGetDevice(&dev));
    PR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8;
    const int iters = (kind == PR_PEAK_FP64_FMA) ? 2048 : 32768;
    void *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PR_CUDA_TRY(cudaMalloc(&sink, 16));
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best_ms = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first launch warms up
        cudaEventRecord(e0);
        if (kind == PR_PEAK_FP64_FMA)
            dfma_kernel<<<blocks, kPeakBlock>>>((double *)sink, iters, 0.9999999, 1e-7);
        else if (kind == PR_PEAK_FP32_FMA)
            ffma_kernel<<<blocks, kPeakBlock>>>((float *)sink, iters, 0.9999f, 1e-4f);
        else
            ex2_kernel<<<blocks, kPeakBlock>>>((float *)sink, iters);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best_ms) best_ms = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) {
        prgb::set_error("pr_measure_peak: %s", cudaGetErrorString(e));
        return PR_ECUDA;
    }
    const double ops_per_elem = (kind == PR_PEAK_MUFU_EX2) ? 1.0 : 2.0;   // an FMA is two flops
    *ops_per_s = ops_per_elem * (double)blocks * kPeakBlock * kChains * iters / (best_ms * 1e-3);
    return PR_OK;
}
