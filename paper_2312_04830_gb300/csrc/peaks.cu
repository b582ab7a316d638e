// Throughput microbenchmarks of the arithmetic pipes that bound the property
// kernels: FP64 FMA (the FP64 paths), FP32 FMA and the special-function unit
// (exp2) of the FP32 paths.  Each thread runs eight independent dependency
// chains, enough warps per SM to cover the pipe latency; the result is kept
// alive by a store that a comparison with an impossible value guards.  They
// give the roofline denominators measured on the device the library runs on.
#include <cuda_runtime.h>

#include "pr_internal.h"
#include "pr_math64.cuh"

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

// FP64 library calls (exp, log, division, square root, cube root) with CUDA's
// own implementations: calls per second when nothing else runs, i.e. how many
// FP64-pipe slots one call takes (the DFMA rate over this rate).  Each chain
// maps [-1.5, -0.4] into itself with the call and at most one FP64 add or FMA
// besides, so no clamp is needed; arguments are of order one, as in the
// property kernels.
template <int OP>
__device__ __forceinline__ double f64_call(double x)
{
    if (OP == 0) return exp(x) - 1.5;          // [-1.277, -0.830]
    if (OP == 1) return fma(0.5, log(-x), -0.9);   // [-1.358, -0.697]
    if (OP == 2) return 1.0 / (x - 0.5);       // [-1.111, -0.5]
    if (OP == 3) return -sqrt(-x);             // [-1.225, -0.632]
    return -cbrt(-x);                          // [-1.145, -0.737]
}

template <int OP>
__global__ void __launch_bounds__(kPeakBlock) f64_call_kernel(double *sink, int iters)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = -0.6 - 1e-4 * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = f64_call<OP>(x[c]);
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.2345e300) sink[0] = s;
}

// The library's FP64 exp, expm1, log, log1p (fn 0..3) and CUDA's (fn 4..7) on
// an array, for their accuracy tests.
__global__ void eval_math_kernel(int fn, int64_t n, const double *x, double *y)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        double r;
        switch (fn) {
        case 0: r = m64::exp(v); break;
        case 1: r = m64::expm1(v); break;
        case 2: r = m64::log(v); break;
        case 3: r = m64::log1p(v); break;
        case 4: r = ::exp(v); break;
        case 5: r = ::expm1(v); break;
        case 6: r = ::log(v); break;
        default: r = ::log1p(v); break;
        }
        y[i] = r;
    }
}

}  // namespace

extern "C" pr_status pr_eval_math(int fn, int64_t n, const double *x, double *y, void *stream)
{
    PR_CHECK_ARG(fn >= 0 && fn <= 7, "pr_eval_math: unknown function %d", fn);
    PR_CHECK_ARG(n >= 0, "pr_eval_math: n < 0");
    if (n == 0) return PR_OK;
    PR_CHECK_ARG(x && y && prgb::aligned(x, 8) && prgb::aligned(y, 8), "pr_eval_math: bad array");
    const int64_t b = (n + 255) / 256;
    eval_math_kernel<<<(int)(b < 4096 ? b : 4096), 256, 0, (cudaStream_t)stream>>>(fn, n, x, y);
    PR_CUDA_TRY(cudaGetLastError());
    return PR_OK;
}

extern "C" pr_status pr_measure_peak(int kind, double *ops_per_s)
{
    PR_CHECK_ARG(ops_per_s != nullptr, "pr_measure_peak: null output");
    PR_CHECK_ARG(kind >= PR_PEAK_FP64_FMA && kind <= PR_PEAK_FP64_CBRT, "pr_measure_peak: unknown kind %d", kind);
    int dev = 0, sms = 0;
    PR_CUDA_TRY(cudaGetDevice(&dev));
    PR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8;
    const bool call = kind >= PR_PEAK_FP64_EXP;
    const int iters = call ? 128 : (kind == PR_PEAK_FP64_FMA) ? 2048 : 32768;
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
        else if (kind == PR_PEAK_MUFU_EX2)
            ex2_kernel<<<blocks, kPeakBlock>>>((float *)sink, iters);
        else if (kind == PR_PEAK_FP64_EXP)
            f64_call_kernel<0><<<blocks, kPeakBlock>>>((double *)sink, iters);
        else if (kind == PR_PEAK_FP64_LOG)
            f64_call_kernel<1><<<blocks, kPeakBlock>>>((double *)sink, iters);
        else if (kind == PR_PEAK_FP64_DIV)
            f64_call_kernel<2><<<blocks, kPeakBlock>>>((double *)sink, iters);
        else if (kind == PR_PEAK_FP64_SQRT)
            f64_call_kernel<3><<<blocks, kPeakBlock>>>((double *)sink, iters);
        else
            f64_call_kernel<4><<<blocks, kPeakBlock>>>((double *)sink, iters);
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
    const double ops_per_elem = (kind == PR_PEAK_FP64_FMA || kind == PR_PEAK_FP32_FMA) ? 2.0 : 1.0;   // an FMA is two flops
    *ops_per_s = ops_per_elem * (double)blocks * kPeakBlock * kChains * iters / (best_ms * 1e-3);
    return PR_OK;
}
