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

#include "pr_device.cuh"
#include "pr_internal.h"

using prk::SpeciesRec;

namespace {

constexpr size_t kCounterBytes = 256;   // the counter, padded so that the list stays 256-byte aligned

// File-scope scratch: [counter (uint32) | pad to 256 B | int32 list[PR_NOALLOC_MAX_CELLS]].
static __device__ __align__(256) unsigned char g_noalloc_scratch[kCounterBytes + 4ull * PR_NOALLOC_MAX_CELLS];

__global__ void noalloc_compact_kernel(int64_t n, const uint8_t *__restrict__ mask, unsigned int *count,
                                       int32_t *list)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (mask[i]) list[atomicAdd(count, 1u)] = (int32_t)i;
}

// FP64 properties of the listed cells; float inputs and outputs (the same
// per-cell step as the surrogate's fallback kernel).
template <int NS, bool KIJ>
__global__ void __launch_bounds__(128) noalloc_props_kernel(const int32_t *list, const unsigned int *count,
                                                            const float *T, const float *p, const float *Y,
                                                            int64_t ldY, float *out, int64_t ldo,
                                                            const SpeciesRec<double> *sp, const double *pair,
                                                            const double *kij, int N, int flags, double tmid_u)
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
    for (unsigned int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x)
        prk::fallback_cell_fp64<NS, KIJ>(list[t], T, p, Y, ldY, out, ldo, s_sp, s_pair, s_kij, N, flags, tmid_u);
}

template <int NS, bool KIJ>
void launch_noalloc(const pr_ctx *ctx, const int32_t *list, const unsigned int *count, const float *T,
                    const float *p, const float *Y, int64_t ldY, float *out, int64_t ldo, cudaStream_t st)
{
    noalloc_props_kernel<NS, KIJ><<<ctx->num_sms * 4, 128, 0, st>>>(
        list, count, T, p, Y, ldY, out, ldo, (const SpeciesRec<double> *)ctx->d_sp64, ctx->d_pair64, ctx->d_kij64,
        ctx->n_species, ctx->flags, ctx->tmid_u);
}

}  // namespace

namespace prgb {
// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, never a device address, so
// the address is looked up here, once per context, by pr_create (with the
// context's device current) and kept in the context.
pr_status noalloc_scratch_address(void **ptr)
{
    *ptr = nullptr;
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();   // not left for a later launch check to report
        set_error("cudaGetSymbolAddress of the allocation-free scratch failed: %s", cudaGetErrorString(e));
        return PR_ECUDA;
    }
    *ptr = p;
    return PR_OK;
}
}  // namespace prgb

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
    // the context's tables live on its device, and the scratch address was
    // taken there: another current device would read memory it cannot reach
    int dev = -1;
    PR_CUDA_TRY(cudaGetDevice(&dev));
    PR_CHECK_ARG(dev == ctx->device,
                 "pr_fallback_props_noalloc: the current device (%d) is not the context's device (%d)", dev,
                 ctx->device);
    void *scratch = ctx->noalloc_scratch;
    if (!scratch) {
        prgb::set_error("pr_fallback_props_noalloc: the scratch address could not be looked up when the context "
                        "was created");
        return PR_ECUDA;
    }
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
