// Tensor-core GEMM for the surrogate MLP: D[M x N] = A[M x K] * B[N x K]^T
// with BF16 operands (both K-major, loaded by TMA with 128-byte swizzling),
// an FP32 accumulator in tensor memory (tcgen05.mma, cta_group::1, M = 128)
// and fused epilogues for every GEMM of the MLP's forward and backward pass.
//
// CTA = 6 warps: warp 0 issues TMA loads into an S-stage shared-memory ring,
// one thread of warp 1 issues the MMAs (K = 16 each, 4 per 64-wide k-block)
// and commits each stage back to the producer, warps 2-5 drain the
// accumulator (each warp owns the TMEM lane quarter warp % 4, i.e. 32 rows)
// and run the epilogue.  One output tile (and one K split) per CTA; two CTAs
// fit on an SM so that one CTA's epilogue overlaps the other's main loop.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "umma.cuh"

namespace mlp {

constexpr int BM = 128;
constexpr int BK = 64;

enum Epi : int {
    kEpiHidden = 0,    // h = GeLU(acc + b) -> out; (train) h^T -> outT, GeLU'(acc + b) -> gd
    kEpiOutPhys = 1,   // y = acc + b (n < 6) -> de-standardise -> physical properties out6[6][ld6]
    kEpiOutLoss = 2,   // y = acc + b; d = y - target (0 where the target is not finite); loss += d^2;
                       // dz = scale d -> out, outT, colsum
    kEpiDx = 3,        // dz = acc * gd -> out, outT, colsum
    kEpiDw = 4,        // partial[split][m][n] = acc (FP32)
};

struct GemmArgs {
    int M, N, K;              // logical sizes; A is [M][K], B is [N][K]
    int kb_per_split;         // 64-wide k-blocks per K split (gridDim.z splits)
    const float *bias;        // [N]
    __nv_bfloat16 *out;       // [M][ldo] batch-major
    int64_t ldo;
    __nv_bfloat16 *outT;      // [N][ldoT] feature-major (may be null)
    int64_t ldoT;
    __nv_bfloat16 *gd;        // [M][ldg] GeLU'(z): written by kEpiHidden (train), read by kEpiDx
    int64_t ldg;
    float *partial;           // kEpiDw: [split][Mpad][N]
    int Mpad;
    float *colsum;            // [gridDim.x][N] per-CTA column sums of dz (bias gradients)
    float *out6;              // kEpiOutPhys: [6][ld6]
    int64_t ld6;
    const float *out_mean, *out_std;   // [6] de-standardisation
    const float *target;      // kEpiOutLoss: standardised targets [6][ldt]
    int64_t ldt;
    float loss_scale;         // d loss / d y = loss_scale * (y - target)
    float *loss_part;         // [gridDim.x] per-CTA sum of squared errors
    int *err;                 // set to 1 when a bounded wait runs out
};

template <int BN>
struct Cfg {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int S = (BN >= 256) ? 2 : ((98304 / STAGE) < 6 ? (98304 / STAGE) : 6);
    static constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;
    static constexpr int BAR_BYTES = 8 * (2 * S + 1) + 16;
    static constexpr int RED_BYTES = 4 * BN * 4 + 64;
    static constexpr int SMEM = 1024 + S * STAGE + BAR_BYTES + RED_BYTES;
};

__device__ __forceinline__ float gelu_f(float z)
{
    return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}

__device__ __forceinline__ float gelu_grad_f(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * __expf(-0.5f * z * z);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void store_row16_bf16(__nv_bfloat16 *dst, const float (&v)[16])
{
    uint4 lo = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
    uint4 hi = make_uint4(pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]), pack_bf16(v[12], v[13]),
                          pack_bf16(v[14], v[15]));
    reinterpret_cast<uint4 *>(dst)[0] = lo;
    reinterpret_cast<uint4 *>(dst)[1] = hi;
}

__device__ __forceinline__ void load_row16_bf16(const __nv_bfloat16 *src, float (&v)[16])
{
    const uint4 a = reinterpret_cast<const uint4 *>(src)[0];
    const uint4 b = reinterpret_cast<const uint4 *>(src)[1];
    const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        __nv_bfloat162 p = *reinterpret_cast<const __nv_bfloat162 *>(&w[k]);
        float2 f = __bfloat1622float2(p);
        v[2 * k] = f.x;
        v[2 * k + 1] = f.y;
    }
}

// Sum 16 per-lane values over the 32 lanes of a warp; afterwards even lane L
// holds the sum of column (L >> 1).  15 shuffles instead of 80.
__device__ __forceinline__ float warp_colsum16(float (&v)[16], int lane)
{
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const bool up = lane & 16;
        const float send = up ? v[k] : v[k + 8];
        const float keep = up ? v[k + 8] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool up = lane & 8;
        const float send = up ? v[k] : v[k + 4];
        const float keep = up ? v[k + 4] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const bool up = lane & 4;
        const float send = up ? v[k] : v[k + 2];
        const float keep = up ? v[k + 2] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        const bool up = lane & 2;
        const float send = up ? v[0] : v[1];
        const float keep = up ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

__device__ __forceinline__ void named_barrier_epi()
{
    asm volatile("bar.sync 1, 128;" ::: "memory");
}

template <int BN, int EPI>
__global__ void __launch_bounds__(192, 1) gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                      const __grid_constant__ CUtensorMap tmB, const GemmArgs a)
{
    using C = Cfg<BN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + C::S * C::STAGE);
    uint64_t *empty = full + C::S;
    uint64_t *accf = empty + C::S;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accf + 1);
    float *red = reinterpret_cast<float *>(smem + C::S * C::STAGE + C::BAR_BYTES);   // [4][BN] + 16

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int kb_total = (a.K + BK - 1) / BK;
    const int kb0 = blockIdx.z * a.kb_per_split;
    const int nkb = min(a.kb_per_split, kb_total - kb0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::S; ++s) {
            umma::mbar_init(&full[s], 1);
            umma::mbar_init(&empty[s], 1);
        }
        umma::mbar_init(accf, 1);
        umma::fence_mbar_init();
        umma::tma_prefetch_desc(&tmA);
        umma::tma_prefetch_desc(&tmB);
    }
    if (warp == 1) {
        umma::tmem_alloc(tmem_slot, C::TMEM_COLS);
        umma::tmem_relinquish();
    }
    umma::tc_fence_before();
    __syncthreads();
    umma::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool fail = false;

    if (warp == 0) {
        if (lane == 0) {
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % C::S;
                const uint32_t ph = (uint32_t)(kb / C::S) & 1u;
                if (kb >= C::S && !umma::mbar_wait(&empty[s], ph ^ 1u)) { fail = true; break; }
                uint8_t *st = smem + s * C::STAGE;
                umma::mbar_arrive_expect_tx(&full[s], C::STAGE);
                umma::tma_load_2d(st, &tmA, &full[s], (kb0 + kb) * BK, m0);
                umma::tma_load_2d(st + C::A_BYTES, &tmB, &full[s], (kb0 + kb) * BK, n0);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = umma::idesc_bf16_f32(BM, BN);
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % C::S;
                const uint32_t ph = (uint32_t)(kb / C::S) & 1u;
                if (!umma::mbar_wait(&full[s], ph)) { fail = true; break; }
                umma::tc_fence_after();
                const uint32_t sa = umma::smem_u32(smem + s * C::STAGE);
                const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
                for (int k = 0; k < BK / 16; ++k) {
                    umma::mma_bf16(tmem, umma::sdesc_kmajor_sw128(sa + k * 32), umma::sdesc_kmajor_sw128(sb + k * 32),
                                   idesc, (kb > 0 || k > 0) ? 1u : 0u);
                }
                umma::mma_commit(&empty[s]);
            }
            umma::mma_commit(accf);
        }
    } else {
        // ------------------------------------------------------ epilogue
        const int q = warp & 3;                     // TMEM lane quarter of this warp
        const int row = q * 32 + lane;
        const int m = m0 + row;
        const bool mval = m < a.M;
        if (!umma::mbar_wait(accf, 0)) fail = true;
        umma::tc_fence_after();
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16);
        float lsum = 0.f;
#pragma unroll 1
        for (int c = 0; c < BN / 16; ++c) {
            uint32_t r[16];
            umma::tmem_ld16(taddr + c * 16, r);
            umma::tmem_ld_wait();
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
            const int nb = n0 + c * 16;
            if (EPI == kEpiHidden) {
                float g[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float z = v[j] + __ldg(a.bias + nb + j);
                    v[j] = gelu_f(z);
                    g[j] = gelu_grad_f(z);
                }
                if (mval) {
                    store_row16_bf16(a.out + (int64_t)m * a.ldo + nb, v);
                    if (a.gd) store_row16_bf16(a.gd + (int64_t)m * a.ldg + nb, g);
                    if (a.outT) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) a.outT[(int64_t)(nb + j) * a.ldoT + m] = __float2bfloat16_rn(v[j]);
                    }
                }
            } else if (EPI == kEpiOutPhys) {
                if (mval && c == 0) {
#pragma unroll
                    for (int j = 0; j < 6; ++j) {
                        const float s = v[j] + __ldg(a.bias + j);
                        const float qv = s * __ldg(a.out_std + j) + __ldg(a.out_mean + j);
                        a.out6[(int64_t)j * a.ld6 + m] = (j == 1 || j == 2) ? qv : __expf(qv);
                    }
                }
            } else if (EPI == kEpiOutLoss) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float d = 0.f;
                    if (mval && c == 0 && j < 6) {
                        const float t = __ldg(a.target + (int64_t)j * a.ldt + m);
                        d = isfinite(t) ? v[j] + __ldg(a.bias + j) - t : 0.f;   // non-finite targets are masked
                    }
                    lsum += d * d;
                    v[j] = a.loss_scale * d;
                }
                if (mval) {
                    store_row16_bf16(a.out + (int64_t)m * a.ldo + nb, v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) a.outT[(int64_t)(nb + j) * a.ldoT + m] = __float2bfloat16_rn(v[j]);
                }
            } else if (EPI == kEpiDx) {
                float g[16];
                if (mval) load_row16_bf16(a.gd + (int64_t)m * a.ldg + nb, g);
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = mval ? v[j] * g[j] : 0.f;
                if (mval) {
                    store_row16_bf16(a.out + (int64_t)m * a.ldo + nb, v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) a.outT[(int64_t)(nb + j) * a.ldoT + m] = __float2bfloat16_rn(v[j]);
                }
            } else {  // kEpiDw
                if (m < a.Mpad) {
                    float4 *dst = reinterpret_cast<float4 *>(
                        a.partial + ((int64_t)blockIdx.z * a.Mpad + m) * a.N + nb);
#pragma unroll
                    for (int j = 0; j < 4; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                }
            }
            if (EPI == kEpiOutLoss || EPI == kEpiDx) {
                const float s = warp_colsum16(v, lane);
                if ((lane & 1) == 0) red[q * BN + c * 16 + (lane >> 1)] = s;
            }
        }
        if (EPI == kEpiOutLoss || EPI == kEpiDx) {
            if (EPI == kEpiOutLoss) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
                if (lane == 0) red[4 * BN + q] = lsum;
            }
            named_barrier_epi();
            const int t = threadIdx.x - 64;
            for (int col = t; col < BN; col += 128)
                a.colsum[(int64_t)blockIdx.x * a.N + n0 + col] =
                    red[col] + red[BN + col] + red[2 * BN + col] + red[3 * BN + col];
            if (EPI == kEpiOutLoss && t == 0)
                a.loss_part[blockIdx.x] = red[4 * BN] + red[4 * BN + 1] + red[4 * BN + 2] + red[4 * BN + 3];
        }
    }
    __syncwarp();   // reconverge each warp (role lanes vs idle lanes) before the CTA barrier
    if (fail) atomicExch(a.err, 1);
    umma::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        umma::tc_fence_after();
        umma::tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

}  // namespace mlp
