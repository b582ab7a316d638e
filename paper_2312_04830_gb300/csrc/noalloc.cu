// pr_fallback_props_noalloc: the surrogate's Peng-Robinson fallback step
// (compact the flagged cells, then evaluate them in FP64) for callers that
// cannot allocate device memory.
//
// Why: some host programs that embed this library may not call cudaMalloc at
// all -- for example a solver that hands every device buffer over from its own
// memory pool, or code that runs where allocating would break a memory budget
// fixed ahead of time.  The regular path keeps its compaction list in memory
// that surrogate_create allocates; this entry point instead uses a fixed
// scratch array compiled into the library, so the call itself allocates
// nothing.
//
// The scratch array (one counter and PR_NOALLOC_MAX_CELLS cell indices,
// about 4 MB) lives in device memory of every GPU that loads the library,
// until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "pr_device.cuh"
#include "pr_internal.h"

using prk::SpeciesRec;

namespace {

constexpr int kNoallocMaxDevices = 64;
constexpr size_t kCounterBytes = 256;   // the counter, padded so that the list stays 256-byte aligned

// File-scope scratch: [counter (uint32) | pad to 256 B | int32 list[PR_NOALLOC_MAX_CELLS]].
static __device__ __align__(256) unsigned char g_noalloc_scratch[kCounterBytes + 4ull * PR_NOALLOC_MAX_CELLS];

// Device address of g_noalloc_scratch per device (in host code the symbol's
// name is only a host-side stand-in, never a device address).
void *g_scratch_ptr[kNoallocMaxDevices] = {};
std::mutex g_scratch_mu;

__global__ void noalloc_compact_kernel(int64_t n, const uint8_t *__restrict__ mask, unsigned int *count,
                                       int32_t *list)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (mask[i]) list[atomicAdd(count, 1u)] = (int32_t)i;
}

// FP64 properties of the listed cells; float inputs and outputs.
template <int NS, bool KIJ>
__global__ void __launch_bounds__(128) noalloc_props_kernel(const int32_t *list, const unsigned int *count,
                                                            const float *T, const float *p, const float *Y,
                                                            int64_t ldY, float *out, int64_t ldo,
                                                            const SpeciesRec<double> *sp, const double *pair,
                                                            const double *kij, int N, int flags)
{
    __shared__ SpeciesRec<double> s_sp[NS];
    __shared__ double s_pair[NS * NS];
    __shared__ double s_kij[KIJ ? NS * NS : 1];
    {
        const double *src = reinterpret_cast<const double *>(sp);
        double *dst = reinterpret_cast<double *>(s_sp);
        for (int j = threadIdx.x; j < (int)(NS * sizeof(SpeciesRec<double>) / 8); j += blockDim.x) dst[j] = src[j];
        for (int j = threadIdx.x; j < NS * NS; j += blockDim.x) {
            s_pair[j] = pair[j];
            if (KIJ) s_kij[j] = kij[j];
        }
    }
    __syncthreads();
    const unsigned int m = *count;
    for (unsigned int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
        const int64_t i = list[t];
        const double Tv = (double)T[i], pv = (double)p[i];
        prk::Comp<double, NS> c;
        double ysum = 0, s = 0;
        bool ok = (Tv > 0) && (pv > 0) && isfinite(Tv) && isfinite(pv);
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            const double y = (k < N) ? (double)Y[(int64_t)k * ldY + i] : 0.0;
            ok = ok && (y >= 0) && isfinite(y);
            ysum += y;
            c.x[k] = y * s_sp[k].inv_W;
            s += c.x[k];
        }
        ok = ok && fabs(ysum - 1.0) <= 1e-6 && s > 0;
        const double is = 1.0 / s;
        double bm = 0;
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            c.x[k] *= is;
            bm = fma(c.x[k], s_sp[k].b, bm);
        }
        c.Wbar = is;
        c.bm = bm;
        float o[6];
        for (int q = 0; q < 6; ++q) o[q] = __int_as_float(0x7fc00000);
        if (ok) {
            prk::Thermo<double> th;
            prk::thermo<double, double, NS, KIJ>(c, Tv, pv, s_sp, s_kij, th);
            if (th.status != prk::kNoRoot) {
                double mu, lam;
                prk::transport<double, NS>(c, Tv, th, s_sp, s_pair, flags, mu, lam);
                o[0] = (float)(pv * c.Wbar / (th.Z * prk::kR * Tv));
                o[1] = (float)th.Z;
                o[2] = (float)th.h;
                o[3] = (float)th.cp;
                o[4] = (float)mu;
                o[5] = (float)lam;
            }
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) out[(int64_t)q * ldo + i] = o[q];
    }
}

// Device address of the scratch array on the current device, looked up once
// per device (with that device current).
pr_status scratch_on_current_device(void **ptr)
{
    int dev = -1;
    PR_CUDA_TRY(cudaGetDevice(&dev));
    PR_CHECK_ARG(dev >= 0 && dev < kNoallocMaxDevices, "pr_fallback_props_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            prgb::set_error("pr_fallback_props_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return PR_ECUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *ptr = g_scratch_ptr[dev];
    return PR_OK;
}

template <int NS, bool KIJ>
void launch_noalloc(const pr_ctx *ctx, const int32_t *list, const unsigned int *count, const float *T,
                    const float *p, const float *Y, int64_t ldY, float *out, int64_t ldo, cudaStream_t st)
{
    noalloc_props_kernel<NS, KIJ><<<ctx->num_sms * 4, 128, 0, st>>>(
        list, count, T, p, Y, ldY, out, ldo, (const SpeciesRec<double> *)ctx->d_sp64, ctx->d_pair64, ctx->d_kij64,
        ctx->n_species, ctx->flags);
}

}  // namespace

extern "C" pr_status pr_fallback_props_noalloc(pr_ctx *ctx, int64_t n, const float *T, const float *p,
                                               const float *Y, int64_t ldY, const uint8_t *mask, float *out,
                                               int64_t ldo, void *stream)
{
    PR_CHECK_ARG(ctx != nullptr, "pr_fallback_props_noalloc: null context");
    PR_CHECK_ARG(n >= 0, "pr_fallback_props_noalloc: n < 0");
    PR_CHECK_ARG(n <= PR_NOALLOC_MAX_CELLS,
                 "pr_fallback_props_noalloc: n = %lld exceeds the fixed scratch capacity of %d cells",
                 (long long)n, PR_NOALLOC_MAX_CELLS);
    if (n == 0) return PR_OK;
    PR_CHECK_ARG(T && p && Y && mask && out, "pr_fallback_props_noalloc: null array");
    PR_CHECK_ARG(ldY >= n && ldo >= n, "pr_fallback_props_noalloc: ldY/ldo < n");
    PR_CHECK_ARG(prgb::aligned(T, 4) && prgb::aligned(p, 4) && prgb::aligned(Y, 4) && prgb::aligned(out, 4),
                 "pr_fallback_props_noalloc: misaligned array");
    void *scratch = nullptr;
    pr_status s = scratch_on_current_device(&scratch);
    if (s) return s;
    unsigned int *count = reinterpret_cast<unsigned int *>(scratch);
    int32_t *list = reinterpret_cast<int32_t *>(reinterpret_cast<unsigned char *>(scratch) + kCounterBytes);
    cudaStream_t st = (cudaStream_t)stream;
    // the scratch keeps the previous call's contents: the counter must restart at zero
    PR_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(unsigned int), st));
    const int64_t blocks = (n + 255) / 256;
    noalloc_compact_kernel<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(n, mask, count, list);
    if (ctx->ns_pad == 9) {
        if (ctx->has_kij) launch_noalloc<9, true>(ctx, list, count, T, p, Y, ldY, out, ldo, st);
        else launch_noalloc<9, false>(ctx, list, count, T, p, Y, ldY, out, ldo, st);
    } else {
        if (ctx->has_kij) launch_noalloc<32, true>(ctx, list, count, T, p, Y, ldY, out, ldo, st);
        else launch_noalloc<32, false>(ctx, list, count, T, p, Y, ldY, out, ldo, st);
    }
    PR_CUDA_TRY(cudaGetLastError());
    return PR_OK;
}
