// Tensor-core GEMM for the surrogate MLP: D[M x N] = A[M x K] * B[N x K]^T
// with BF16 operands (both K-major, loaded by TMA with 128-byte swizzling),
// FP32 accumulators in tensor memory (tcgen05.mma, cta_group::1, M = 128)
// and fused epilogues for every GEMM of the MLP's forward and backward pass.
//
// Persistent kernel, one CTA per SM, 10 warps: warp 0 issues TMA loads into
// an S-stage shared-memory ring, one thread of warp 1 issues the MMAs (K = 16
// each, 4 per 64-wide k-block), warps 2-9 drain the accumulator and run the
// epilogue (warp w owns TMEM lane quarter w % 4, i.e. 32 rows, and one half of
// the tile's columns).  The accumulator is double-buffered in TMEM (2 x BN
// columns), so the epilogue of one tile overlaps the main loop of the next.
// Tiles are visited with the N index fastest, so the CTAs working on the
// N-tiles of one M-tile run together and share the A tile through L2; each
// CTA loads its own full weight (B) tile.
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
    kEpiHidden = 0,    // h = GeLU(acc + b) -> out; (train) GeLU'(acc + b) -> gd
    kEpiOutPhys = 1,   // y = acc + b (n < nout) -> de-standardise -> physical values out6[nout][ld6]
    kEpiOutLoss = 2,   // y = acc + b; d = y - target (0 where the target is not finite); loss += d^2 (or |d|);
                       // dz = scale d -> out, colsum
    kEpiDx = 3,        // dz = acc * gd -> out, colsum
    kEpiDw = 4,        // partial[split][m][n] = acc (FP32)
    kEpiDwMN = 5,      // as kEpiDw, with A and B read MN-major: A from [K][M], B from [K][N]
                       // (tmA / tmB with 64 x 64 boxes), e.g. dW = dz^T h from the batch-major dz
                       // and h; BN >= 64
};

struct GemmArgs {
    int M, N, K;              // logical sizes; A is [M][K], B is [N][K]
    int kb_per_split;         // 64-wide k-blocks per K split
    int m_tiles, n_tiles, splits;   // tile grid (splits along K)
    const float *bias;        // [N]
    __nv_bfloat16 *out;       // [M][ldo] batch-major
    int64_t ldo;
    __nv_bfloat16 *gd;        // [M][ldg] GeLU'(z): written by kEpiHidden (train), read by kEpiDx
    int64_t ldg;
    float *partial;           // kEpiDw: [split][Mpad][N]
    int Mpad;
    float *colsum;            // [m_tiles][N] per-M-tile column sums of dz (bias gradients)
    float *out6;              // kEpiOutPhys: [nout][ld6]
    int64_t ld6;
    const float *out_mean, *out_std;   // [nout] de-standardisation
    const float *add_h;       // kEpiOutPhys: per-row term added to output 2 (h) after de-standardisation
    int log_mask;             // kEpiOutPhys: bit j set = output j was learned as its logarithm
    const float *target;      // kEpiOutLoss: standardised targets [nout][ldt]
    int64_t ldt;
    float loss_scale;         // d loss / d y = loss_scale * (y - target), or loss_scale * sign(y - target) (l1)
    float *loss_part;         // [m_tiles] per-M-tile sum of squared (l1: absolute) errors
    int l1;                   // kEpiOutLoss: 1 = L1 loss, 0 = squared error
    int nout;                 // kEpiOutPhys / kEpiOutLoss: outputs in use (<= 16)
    int *err;                 // set to 1 when a bounded wait runs out
    // kEpiHidden / kEpiDx with tma_out != 0: `out` (and `gd` when written) go
    // out through shared memory and TMA stores of 32 x 64 boxes (128-byte
    // swizzle); tm_out / tm_gd map those matrices with that box
    int tma_out;
    CUtensorMap tm_out, tm_gd;
};

constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;

template <int BN>
struct Cfg {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int STG_BYTES = kEpiWarps * 8192;   // output staging: two 4 KB boxes per epilogue warp
    static constexpr int S_FIT = (232448 - 1024 - STG_BYTES - 12288) / STAGE;
    static constexpr int S = S_FIT < 8 ? S_FIT : 8;
    static constexpr uint32_t TMEM_COLS = (2 * BN) < 32 ? 32 : 2 * BN;   // two accumulator buffers
    static constexpr int BAR_BYTES = 8 * (2 * S + 4) + 16;
    static constexpr int RED_BYTES = 4 * BN * 4 + 64;
    static constexpr int BIAS_BYTES = 1024 * 4;   // bias of up to 1024 output columns
    static constexpr int SMEM = 1024 + S * STAGE + STG_BYTES + BAR_BYTES + RED_BYTES + BIAS_BYTES;
};

// GeLU in its tanh form (Hendrycks & Gimpel 2016),
//   GeLU(z) ~ z/2 (1 + tanh(k (z + c z^3))),  k = sqrt(2/pi), c = 0.044715,
// with the hardware tanh.approx.f32 (one MUFU operation), and its exact
// derivative
//   GeLU'(z) = (1 + t)/2 + z/2 (1 - t^2) k (1 + 3 c z^2),  t = tanh(k (z + c z^3)).
// The tanh form differs from z Phi(z) by at most 5e-4 and tanh.approx has a
// relative error below 2^-10.9; both are under the BF16 rounding of the
// activations (3.9e-3).  Training and inference use this same function.
__device__ __forceinline__ float tanh_approx(float x)
{
    float r;
    asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

constexpr float kGeluK = 0.7978845608028654f;            // sqrt(2/pi)
constexpr float kGeluKC = 0.7978845608028654f * 0.044715f;

__device__ __forceinline__ float gelu_f(float z)
{
    const float z2 = z * z;
    const float t = tanh_approx(z * fmaf(kGeluKC, z2, kGeluK));
    const float hz = 0.5f * z;
    return fmaf(hz, t, hz);
}

// gelu_f of z = a + b on two lanes at once with the packed FP32 instructions
// of sm_100 (FADD2 / FMUL2 / FFMA2): the same operations in the same order as
// gelu_f(a + b), so the same bits, in about half the FP32 instructions.
__device__ __forceinline__ float2 gelu2(float2 a, float2 b)
{
    const float2 z = __fadd2_rn(a, b);
    const float2 z2 = __fmul2_rn(z, z);
    const float2 p = __ffma2_rn(make_float2(kGeluKC, kGeluKC), z2, make_float2(kGeluK, kGeluK));
    const float2 u = __fmul2_rn(z, p);
    const float2 t = make_float2(tanh_approx(u.x), tanh_approx(u.y));
    const float2 hz = __fmul2_rn(make_float2(0.5f, 0.5f), z);
    return __ffma2_rn(hz, t, hz);
}

// gelu_and_grad of z = a + b on two lanes at once (packed FP32): the same
// operations in the same order as the scalar form, so the same bits.
__device__ __forceinline__ void gelu_and_grad2(float2 a, float2 b, float2 &g, float2 &dg)
{
    const float2 z = __fadd2_rn(a, b);
    const float2 z2 = __fmul2_rn(z, z);
    const float2 u = __fmul2_rn(z, __ffma2_rn(make_float2(kGeluKC, kGeluKC), z2, make_float2(kGeluK, kGeluK)));
    const float2 t = make_float2(tanh_approx(u.x), tanh_approx(u.y));
    const float2 hz = __fmul2_rn(make_float2(0.5f, 0.5f), z);
    g = __ffma2_rn(hz, t, hz);
    const float2 dk = __ffma2_rn(make_float2(3.0f * kGeluKC, 3.0f * kGeluKC), z2, make_float2(kGeluK, kGeluK));
    const float2 omt = __ffma2_rn(make_float2(-t.x, -t.y), t, make_float2(1.0f, 1.0f));
    dg = __ffma2_rn(__fmul2_rn(hz, omt), dk, __ffma2_rn(make_float2(0.5f, 0.5f), t, make_float2(0.5f, 0.5f)));
}

__device__ __forceinline__ void gelu_and_grad(float z, float &g, float &dg)
{
    const float z2 = z * z;
    const float t = tanh_approx(z * fmaf(kGeluKC, z2, kGeluK));
    const float hz = 0.5f * z;
    g = fmaf(hz, t, hz);
    const float dk = fmaf(3.0f * kGeluKC, z2, kGeluK);      // d/dz of k (z + c z^3)
    dg = fmaf(hz * fmaf(-t, t, 1.0f), dk, fmaf(0.5f, t, 0.5f));
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

// 16 BF16 of row `row` (0..31), columns 16*c4 .. 16*c4+15 (c4 = 0..3), into a
// 32 x 64 staging box laid out as TMA's 128-byte swizzle: the 16-byte piece j
// of the 128-byte row r sits at piece j ^ (r % 8).
__device__ __forceinline__ void stage_row16_bf16(uint8_t *box, int row, int c4, const float (&v)[16])
{
    const uint4 lo = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                pack_bf16(v[6], v[7]));
    const uint4 hi = make_uint4(pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]), pack_bf16(v[12], v[13]),
                                pack_bf16(v[14], v[15]));
    uint8_t *r = box + row * 128;
    const int j0 = 2 * c4, x = row & 7;
    *reinterpret_cast<uint4 *>(r + ((j0 ^ x) << 4)) = lo;
    *reinterpret_cast<uint4 *>(r + (((j0 + 1) ^ x) << 4)) = hi;
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
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory");
}

// Epilogue of one accumulator tile for one epilogue warp: drain this warp's
// 32 rows x HALF columns from TMEM (loads software-pipelined), apply the
// epilogue, store.  Returns this lane's sum of squared errors (kEpiOutLoss).
template <int BN, int EPI>
__device__ __forceinline__ float epilogue_tile(const GemmArgs &a, uint32_t taddr, int m, bool mval, int n0, int hcol,
                                               int q, int lane, int split, float *red, const float *sbias,
                                               bool active, bool fail, uint8_t *stg, int m0)
{
    constexpr int HALF = (BN >= 32) ? BN / 2 : BN;
    // TMA-store path: this warp's 32 rows x 64 columns of `out` (and of `gd`
    // when written) are staged as 128-byte-swizzled boxes and stored by lane 0,
    // one bulk group per 64 columns; the next group first waits until the
    // previous boxes have been read out of shared memory
    const bool tma = (EPI == kEpiHidden || EPI == kEpiDx) && a.tma_out && (HALF % 64 == 0);
    uint8_t *sh = stg, *sg = stg + 4096;
    float lsum = 0.f;
    if (active && !fail) {
        uint32_t rnext[16];
        umma::tmem_ld16(taddr, rnext);
        // kEpiDx: GeLU'(z) of this lane's row, one chunk ahead (a global load
        // whose latency would otherwise stall every chunk)
        uint4 gq0 = make_uint4(0, 0, 0, 0), gq1 = gq0;
        const __nv_bfloat16 *grow = (EPI == kEpiDx && mval) ? a.gd + (int64_t)m * a.ldg + n0 + hcol : nullptr;
        if (grow) {
            gq0 = reinterpret_cast<const uint4 *>(grow)[0];
            gq1 = reinterpret_cast<const uint4 *>(grow)[1];
        }
#pragma unroll 1
        for (int c = 0; c < HALF / 16; ++c) {
            umma::tmem_ld_wait(rnext);
            uint32_t rr[16];
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) rr[jj] = rnext[jj];
            // next chunk's load is in flight while this one is processed
            if (c + 1 < HALF / 16) umma::tmem_ld16(taddr + (c + 1) * 16, rnext);
            const int nb = n0 + hcol + c * 16;
            uint4 gc0 = gq0, gc1 = gq1;
            if (grow && c + 1 < HALF / 16) {
                gq0 = reinterpret_cast<const uint4 *>(grow + (c + 1) * 16)[0];
                gq1 = reinterpret_cast<const uint4 *>(grow + (c + 1) * 16)[1];
            }
            if (tma && (c & 3) == 0) {
                if (lane == 0) umma::bulk_wait_read0();
                __syncwarp();
            }
            float bias[16];
            if (EPI == kEpiHidden || EPI == kEpiOutPhys || EPI == kEpiOutLoss) {
                const float4 *sb = reinterpret_cast<const float4 *>(sbias + nb);   // broadcast reads
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const float4 b4 = sb[jj];
                    bias[4 * jj] = b4.x; bias[4 * jj + 1] = b4.y; bias[4 * jj + 2] = b4.z; bias[4 * jj + 3] = b4.w;
                }
            }
            float g[16];
            if (EPI == kEpiDx) {
                const uint32_t w[8] = {gc0.x, gc0.y, gc0.z, gc0.w, gc1.x, gc1.y, gc1.z, gc1.w};
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w[k]));
                    g[2 * k] = f.x;
                    g[2 * k + 1] = f.y;
                }
            }
            float v[16];
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) v[jj] = __uint_as_float(rr[jj]);
            if (EPI == kEpiHidden) {
                float gg[16];
                if (a.gd) {
#pragma unroll
                    for (int jj = 0; jj < 16; jj += 2) {
                        float2 g2, d2;
                        gelu_and_grad2(make_float2(v[jj], v[jj + 1]), make_float2(bias[jj], bias[jj + 1]), g2, d2);
                        v[jj] = g2.x; v[jj + 1] = g2.y;
                        gg[jj] = d2.x; gg[jj + 1] = d2.y;
                    }
                } else {
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) v[jj] = gelu_f(v[jj] + bias[jj]);
                }
                if (tma) {
                    stage_row16_bf16(sh, lane, c & 3, v);
                    if (a.gd) stage_row16_bf16(sg, lane, c & 3, gg);
                }
                if (mval) {
                    if (!tma) {
                        store_row16_bf16(a.out + (int64_t)m * a.ldo + nb, v);
                        if (a.gd) store_row16_bf16(a.gd + (int64_t)m * a.ldg + nb, gg);
                    }
                }
            } else if (EPI == kEpiOutPhys) {
                if (mval && nb == 0) {
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        if (jj >= a.nout) break;
                        const float sv = v[jj] + bias[jj];
                        float qv = sv * __ldg(a.out_std + jj) + __ldg(a.out_mean + jj);
                        if (jj == 2 && a.add_h) qv += __ldg(a.add_h + m);
                        a.out6[(int64_t)jj * a.ld6 + m] = ((a.log_mask >> jj) & 1) ? __expf(qv) : qv;
                    }
                }
            } else if (EPI == kEpiOutLoss) {
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    float d = 0.f;
                    if (mval && nb == 0 && jj < a.nout) {
                        const float tv = __ldg(a.target + (int64_t)jj * a.ldt + m);
                        d = isfinite(tv) ? v[jj] + bias[jj] - tv : 0.f;   // non-finite targets are masked
                    }
                    if (a.l1) {
                        lsum += fabsf(d);
                        v[jj] = a.loss_scale * (float)((d > 0.f) - (d < 0.f));
                    } else {
                        lsum += d * d;
                        v[jj] = a.loss_scale * d;
                    }
                }
                if (mval) store_row16_bf16(a.out + (int64_t)m * a.ldo + nb, v);
            } else if (EPI == kEpiDx) {
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) v[jj] = mval ? v[jj] * g[jj] : 0.f;
                if (tma) stage_row16_bf16(sh, lane, c & 3, v);
                if (mval && !tma) store_row16_bf16(a.out + (int64_t)m * a.ldo + nb, v);
            } else {  // kEpiDw, kEpiDwMN
                if (m < a.Mpad) {
                    float4 *dst = reinterpret_cast<float4 *>(a.partial + ((int64_t)split * a.Mpad + m) * a.N + nb);
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj)
                        dst[jj] = make_float4(v[4 * jj], v[4 * jj + 1], v[4 * jj + 2], v[4 * jj + 3]);
                }
            }
            if (tma && (c & 3) == 3) {
                umma::fence_async_smem();   // staging writes visible to the TMA engine
                __syncwarp();
                if (lane == 0) {
                    umma::tma_store_2d(&a.tm_out, sh, nb - 48, m0 + q * 32);
                    if (EPI == kEpiHidden && a.gd) umma::tma_store_2d(&a.tm_gd, sg, nb - 48, m0 + q * 32);
                    umma::bulk_commit();
                }
            }
            if (EPI == kEpiOutLoss || EPI == kEpiDx) {
                const float sv = warp_colsum16(v, lane);
                if ((lane & 1) == 0) red[q * BN + hcol + c * 16 + (lane >> 1)] = sv;
            }
        }
    }
    return lsum;
}

// Tile `t` of the grid-stride walk: K split, M-tile index and N offset.
template <int BN>
__device__ __forceinline__ void tile_of(const GemmArgs &a, int t, int &split, int &mt, int &n0)
{
    const int per_split = a.m_tiles * a.n_tiles;
    split = t / per_split;
    const int r = t % per_split;
    mt = r / a.n_tiles;
    n0 = (r % a.n_tiles) * BN;
}

template <int BN, int EPI>
__global__ void __launch_bounds__(kThreads, 1) gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                           const __grid_constant__ CUtensorMap tmB,
                                                           const __grid_constant__ GemmArgs a)
{
    using C = Cfg<BN>;
    constexpr int HALF = (BN >= 32) ? BN / 2 : BN;   // columns per epilogue warp
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *stg_base = smem + C::S * C::STAGE;   // 1024-aligned: stages are whole KB
    uint64_t *full = reinterpret_cast<uint64_t *>(stg_base + C::STG_BYTES);
    uint64_t *empty = full + C::S;
    uint64_t *acc_full = empty + C::S;     // [2]
    uint64_t *acc_empty = acc_full + 2;    // [2]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
    float *red = reinterpret_cast<float *>(stg_base + C::STG_BYTES + C::BAR_BYTES);   // [4][BN] + 16
    float *sbias = red + 4 * BN + 16;                                                // [N] (N <= 1024)

    static_assert(EPI != kEpiDwMN || BN >= 64, "MN-major operands come in 64-wide boxes");
    constexpr bool kMN = EPI == kEpiDwMN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kb_total = (a.K + BK - 1) / BK;
    const int total = a.m_tiles * a.n_tiles * a.splits;
    const int t_first = blockIdx.x, t_step = gridDim.x;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::S; ++s) {
            umma::mbar_init(&full[s], 1);
            umma::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            umma::mbar_init(&acc_full[b], 1);
            umma::mbar_init(&acc_empty[b], kEpiWarps);
        }
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
        // ------------------------------------------------------- TMA producer
        if (lane == 0) {
            uint32_t it = 0;
            for (int t = t_first; t < total && !fail; t += t_step) {
                int split, mt, n0;
                tile_of<BN>(a, t, split, mt, n0);
                const int m0 = mt * BM;
                const int kb0 = split * a.kb_per_split;
                const int nkb = min(a.kb_per_split, kb_total - kb0);
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % C::S;
                    const uint32_t ph = (it / C::S) & 1u;
                    if (it >= (uint32_t)C::S && !umma::mbar_wait(&empty[s], ph ^ 1u)) { fail = true; break; }
                    uint8_t *st = smem + s * C::STAGE;
                    umma::mbar_arrive_expect_tx(&full[s], C::STAGE);
                    if constexpr (kMN) {
                        // 64 k-rows of 64 M (N) columns per box; blocks of 64 columns 8 KB apart
                        const int kr = (kb0 + kb) * BK;
#pragma unroll
                        for (int i = 0; i < BM / 64; ++i) umma::tma_load_2d(st + i * 8192, &tmA, &full[s], m0 + 64 * i, kr);
#pragma unroll
                        for (int j = 0; j < BN / 64; ++j)
                            umma::tma_load_2d(st + C::A_BYTES + j * 8192, &tmB, &full[s], n0 + 64 * j, kr);
                    } else {
                        umma::tma_load_2d(st, &tmA, &full[s], (kb0 + kb) * BK, m0);
                        umma::tma_load_2d(st + C::A_BYTES, &tmB, &full[s], (kb0 + kb) * BK, n0);
                    }
                }
            }
            // no copy may still be landing in shared memory when the CTA exits
            for (uint32_t k = (it > (uint32_t)C::S ? it - C::S : 0u); k < it; ++k)
                if (!umma::mbar_wait(&full[k % C::S], (k / C::S) & 1u, 200000000LL)) fail = true;
        }
    } else if (warp == 1) {
        // -------------------------------------------------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = kMN ? umma::idesc_bf16_f32_mn(BM, BN) : umma::idesc_bf16_f32(BM, BN);
            uint32_t it = 0, j = 0;
            for (int t = t_first; t < total && !fail; t += t_step, ++j) {
                int split, mt, n0;
                tile_of<BN>(a, t, split, mt, n0);
                const int kb0 = split * a.kb_per_split;
                const int nkb = min(a.kb_per_split, kb_total - kb0);
                const uint32_t buf = j & 1u;
                if (j >= 2 && !umma::mbar_wait(&acc_empty[buf], ((j >> 1) & 1u) ^ 1u)) { fail = true; break; }
                umma::tc_fence_after();
                const uint32_t d_tmem = tmem + buf * BN;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % C::S;
                    const uint32_t ph = (it / C::S) & 1u;
                    if (!umma::mbar_wait(&full[s], ph)) { fail = true; break; }
                    umma::tc_fence_after();
                    const uint32_t sa = umma::smem_u32(smem + s * C::STAGE);
                    const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k) {
                        if constexpr (kMN)   // 16 k-rows of 128 B per step
                            umma::mma_bf16(d_tmem, umma::sdesc_mnmajor_sw128(sa + k * 2048, 8192),
                                           umma::sdesc_mnmajor_sw128(sb + k * 2048, 8192), idesc,
                                           (kb > 0 || k > 0) ? 1u : 0u);
                        else
                            umma::mma_bf16(d_tmem, umma::sdesc_kmajor_sw128(sa + k * 32),
                                           umma::sdesc_kmajor_sw128(sb + k * 32), idesc, (kb > 0 || k > 0) ? 1u : 0u);
                    }
                    umma::mma_commit(&empty[s]);
                }
                umma::mma_commit(&acc_full[buf]);
            }
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const int ew = warp - 2;                   // 0..7
        const int q = warp & 3;                    // TMEM lane quarter this warp may access
        const int hcol = (BN >= 32) ? (ew >> 2) * HALF : 0;   // column half of this warp
        const bool active = (BN >= 32) || (ew < 4);
        const int row = q * 32 + lane;
        if (EPI == kEpiHidden || EPI == kEpiOutPhys || EPI == kEpiOutLoss) {
            for (int col = threadIdx.x - 64; col < a.N; col += 32 * kEpiWarps) sbias[col] = __ldg(a.bias + col);
            named_barrier_epi();
        }
        uint32_t j = 0;
        for (int t = t_first; t < total; t += t_step, ++j) {
            int split, mt, n0;
            tile_of<BN>(a, t, split, mt, n0);
            const bool tile_ok = mt < a.m_tiles;
            const int m0 = mt * BM;
            const int m = m0 + row;
            const bool mval = m < a.M;
            const uint32_t buf = j & 1u;
            // after a timed-out wait this warp skips its work but keeps taking
            // part in the named barriers, so the other epilogue warps finish
            if (!fail && !umma::mbar_wait(&acc_full[buf], (j >> 1) & 1u)) fail = true;
            umma::tc_fence_after();
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + buf * BN + hcol;
            float lsum = epilogue_tile<BN, EPI>(a, taddr, m, mval, n0, hcol, q, lane, split, red, sbias,
                                                      active && tile_ok, fail, stg_base + ew * 8192, m0);
            // the accumulator buffer may be reused once every warp has read it
            umma::tc_fence_before();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&acc_empty[buf]);
            if (EPI == kEpiOutLoss || EPI == kEpiDx) {
                if (EPI == kEpiOutLoss) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
                    if (lane == 0 && active) red[4 * BN + q] = lsum;
                }
                named_barrier_epi();
                const int tt = tile_ok ? threadIdx.x - 64 : BN;
                for (int col = tt; col < BN; col += 32 * kEpiWarps)
                    a.colsum[(int64_t)mt * a.N + n0 + col] =
                        red[col] + red[BN + col] + red[2 * BN + col] + red[3 * BN + col];
                if (EPI == kEpiOutLoss && tile_ok && tt == 0)
                    a.loss_part[mt] = red[4 * BN] + red[4 * BN + 1] + red[4 * BN + 2] + red[4 * BN + 3];
                named_barrier_epi();   // red is reused by the next tile
            }
        }
    }
    if (warp >= 2 && lane == 0) umma::bulk_wait0();   // staged stores complete before shared memory goes
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
