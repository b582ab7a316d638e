// Surrogate MLP (the paper's DNN strategy, Sec. 4): training and inference
// on the tensor cores, with the FP64 Peng-Robinson path as the fallback for
// states outside the training hull.
//
// Network: 13 inputs [log T, p, Y_1..Y_9, T_pc / T, log W] -> H hidden layers
// of width W with
// GeLU -> 6 outputs [log rho, Z, h - h_ig, log cp, log mu, log lambda]; inputs
// and outputs standardised with statistics of the training pool.  The network
// learns the enthalpy departure from the ideal-gas enthalpy h_ig(T, Y) =
// sum_k Y_k h_k(T) / W_k (NASA-7, Sec. 2), which is evaluated exactly (FP32)
// and added back to its output.  Layer l computes
// z = W_l h + b_l with BF16 operands and FP32 accumulation (mlp_gemm.cuh);
// master weights and Adam moments are FP32.
//
// Padded layouts (so that every GEMM is a whole number of 128 x BN x 64
// tiles): inputs K = 11 -> 64, the output layer N = 6 -> 16 (and its weight
// gradient M = 6 -> 128).  Padding entries are zero and stay zero.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "mlp_fused.cuh"
#include "mlp_resident.cuh"
#include "mlp_pingpong.cuh"
#include "mlp_gemm.cuh"
#include "pr_device.cuh"
#include "pr_internal.h"
#include "pr_kernels.cuh"
#include "pr_species.cuh"
#include "surrogate_internal.h"

using namespace mlp;
using prk::SpeciesRec;

namespace {

constexpr int NIN = 13;
constexpr int NOUT6 = 6;       // outputs of the property models (forward, inverse, Bilger)
constexpr int NOUT_MAX = 16;   // output rows of the padded last layer: up to 16 outputs
constexpr int KIN = 64;      // padded input width (one 64-wide k-block)
// Each standardised input enters the first layer as two BF16 numbers, its
// rounding hi = bf16(v) in column k and the remainder lo = bf16(v - hi) in
// column kLoOff + k, both multiplied by the same weight (the FP32
// accumulation adds them): the network sees its inputs to about 16 bits
// instead of BF16's 8, at no tensor-core cost since K = 64 is one k-block
// either way.  (A BF16 log T alone is off by up to 0.35 % in T, which moves
// the viscosity of liquid oxygen by over 1 %.)
constexpr int kLoOff = 16;
static_assert(NIN <= 16 && kLoOff >= 16 && kLoOff + 16 <= KIN, "hi and lo input blocks must fit the padded K");
constexpr int NOP = 16;      // padded output width
constexpr int MOP = 128;     // padded output rows of the last layer's weight gradient
constexpr int NSTAT = NIN + NOUT_MAX;

// Normalisation vector (SG_NORM_FLOATS = 84): in_mean[13] in_std[13]
// out_mean[0..5] out_std[0..5] hull_lo[13] hull_hi[13], then out_mean[6..15]
// and out_std[6..15] of the per-species outputs.
__host__ __device__ constexpr int out_mean_idx(int j) { return j < NOUT6 ? 2 * NIN + j : 64 + (j - NOUT6); }
__host__ __device__ constexpr int out_std_idx(int j) { return j < NOUT6 ? 2 * NIN + NOUT6 + j : 74 + (j - NOUT6); }
static_assert(SG_NORM_FLOATS == 84, "normalisation layout");

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ float uniform01(uint64_t h) { return (float)((h >> 40) * (1.0 / 16777216.0)); }

// Derived features from T and Y: the inverse pseudo-reduced temperature
// T_pc / T (T_pc = sum_k X_k Tc_k, Kay's rule over mole fractions X) and the
// log of the mean molar mass [kg/mol].
__device__ __forceinline__ void derived_features(float T, const float *Y, const void *sp32, float &tpc_over_T,
                                                 float &logW)
{
    const SpeciesRec<float> *sp = static_cast<const SpeciesRec<float> *>(sp32);
    float s = 0.f, st = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float nk = Y[k] * __ldg(&sp[k].inv_W);   // moles per kg
        s += nk;
        st = fmaf(nk, __ldg(&sp[k].Tc), st);
    }
    tpc_over_T = st / (s * T);
    logW = -logf(s);
}

__device__ __forceinline__ float h_ideal(float T, const float (&Y)[9], const void *sp32);

// Box-Cox transform ((x + shift)^lambda - 1) / lambda (log(x + shift) at
// lambda = 0); NaN where x + shift <= 0, which the hull check turns into a
// fallback.
__device__ __forceinline__ float box_cox(float x, float lambda, float shift)
{
    const float u = x + shift;
    if (!(u > 0.f)) return __int_as_float(0x7fc00000);
    return (lambda == 0.f) ? logf(u) : (powf(u, lambda) - 1.f) / lambda;
}

// Features of one cell from its first raw input v0, p and Y (in f[1..10]):
//   forward model (v0 = T):  [log T, p, Y_1..Y_9, T_pc / T, log W];
//   inverse model (v0 = h*): [h* - h_f(Y), p, Y_1..Y_9, log T_pc, log W], where
//   h_f(Y) = sum_k Y_k h_k(298.15 K) / W_k removes the formation enthalpies, so
//   that the first input is the sensible-plus-departure enthalpy;
//   Bilger model (v0 = h*): [h* - h_f(Y), p, BoxCox(Z)] with Bilger's mixture
//   fraction Z of Y (the paper's network inputs, Sec. 4.1-4.2), the other
//   slots zero.
__device__ __forceinline__ void cell_features(const SgDev &d, float v0, float (&f)[NIN])
{
    const int mode = d.mode;
    const void *sp32 = d.sp32;
    float tpc_over_T, logW;
    if (mode == SG_MODE_BILGER) {
        float Yk[9];
        float beta = 0.f;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            Yk[k] = f[2 + k];
            beta = fmaf(__ldg(d.bilger + k), Yk[k], beta);
        }
        const float z = (beta - __ldg(d.bilger + 9)) * __ldg(d.bilger + 10);
        f[0] = v0 - h_ideal(298.15f, Yk, sp32);
        f[2] = box_cox(z, d.bc_lambda, d.bc_shift);
#pragma unroll
        for (int k = 3; k < NIN; ++k) f[k] = 0.f;
        return;
    }
    if (mode == SG_MODE_INVERSE) {
        float Yk[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) Yk[k] = f[2 + k];
        derived_features(1.0f, f + 2, sp32, tpc_over_T, logW);   // T = 1: T_pc itself
        f[0] = v0 - h_ideal(298.15f, Yk, sp32);
        f[11] = logf(tpc_over_T);
    } else {
        derived_features(v0, f + 2, sp32, tpc_over_T, logW);
        f[0] = logf(v0);
        f[11] = tpc_over_T;
    }
    f[12] = logW;
}

// Features of pool row i, x = [v0, p, Y_1..Y_9] (v0 = T, or h* for the inverse model).
__device__ __forceinline__ void features(const float *x, int64_t ldx, int64_t i, const SgDev &d, float (&f)[NIN])
{
    f[1] = __ldg(x + ldx + i);
#pragma unroll
    for (int k = 0; k < 9; ++k) f[2 + k] = __ldg(x + (int64_t)(2 + k) * ldx + i);
    cell_features(d, __ldg(x + i), f);
}

// Mass-specific ideal-gas enthalpy sum_k Y_k h_k(T) / W_k [J/kg] from the
// NASA-7 records (molar h = R (a1 T + a2 T^2/2 + ... + a5 T^5/5 + a6)).
__device__ __forceinline__ float h_ideal(float T, const float (&Y)[9], const void *sp32)
{
    const SpeciesRec<float> *sp = static_cast<const SpeciesRec<float> *>(sp32);
    float h = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float *e = (T < __ldg(&sp[k].T_mid)) ? sp[k].h_lo : sp[k].h_hi;
        float hk = __ldg(e + 4);
#pragma unroll
        for (int j = 3; j >= 0; --j) hk = fmaf(hk, T, __ldg(e + j));
        hk = fmaf(hk, T, __ldg(e + 5));
        h = fmaf(Y[k] * __ldg(&sp[k].inv_W), hk, h);
    }
    return h;
}

// Outputs learned as logarithms (bit j: output j).
constexpr int kLogMaskForward = 0x39;   // rho, cp, mu, lambda
constexpr int kLogMaskInverse = 0x3F;   // all six
constexpr int kLogMaskDk = 0x1FF;       // the nine diffusion coefficients

__host__ __device__ inline int log_mask_of(int mode, int outputs)
{
    if (outputs == SG_OUT_DK) return kLogMaskDk;
    if (outputs == SG_OUT_HK) return 0;
    if (outputs >= SG_OUT_SINGLE) return 1;   // one of the inverse model's six, all logarithms
    return (mode != SG_MODE_FORWARD) ? kLogMaskInverse : kLogMaskForward;
}

// Targets from raw properties and inputs x = [T, p, Y_1..Y_9]:
//   forward model, y = [rho, Z, h, cp, mu, lambda]:
//     [log rho, Z, h - h_ig(T, Y), log cp, log mu, log lambda];
//   inverse and Bilger models, y = [T, rho, psi, mu, alpha, cp]: the six logarithms;
//   per-species outputs (inverse or Bilger inputs), y = D_k [9]: their logarithms,
//   or y = h_k / (R T) [9] as they are;
//   a single property of the inverse set (y = [one of T, rho, psi, mu, alpha, cp]):
//   its logarithm.
__device__ __forceinline__ void targets(const float *x, int64_t ldx, const float *y, int64_t ldy, int64_t i,
                                        const SgDev &d, float (&q)[NOUT_MAX])
{
    const int lm = log_mask_of(d.mode, d.outputs);
#pragma unroll
    for (int j = 0; j < NOUT_MAX; ++j) {
        const float v = (j < d.nout) ? __ldg(y + (int64_t)j * ldy + i) : 0.f;
        q[j] = ((lm >> j) & 1) ? logf(v) : v;
    }
    const void *sp32 = d.sp32;
    if (d.mode != SG_MODE_FORWARD) return;
    float Yk[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Yk[k] = __ldg(x + (int64_t)(2 + k) * ldx + i);
    q[2] -= h_ideal(__ldg(x + i), Yk, sp32);
}

// ------------------------------------------------------------ init params
__global__ void init_params_kernel(SgDev d, uint64_t seed)
{
    const int64_t total = d.n_master;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        ParamRef r = decode_param(d, e);
        float v = 0.f;
        if (r.valid) {
            const float bound = 1.0f / sqrtf((float)(r.layer == 0 ? NIN : d.width));
            v = bound * (2.f * uniform01(splitmix64(seed * 0x100000001B3ull + (uint64_t)e)) - 1.f);
        }
        d.master[e] = v;
        d.adam_m[e] = 0.f;
        d.adam_v[e] = 0.f;
    }
}

// BF16 copy of the weights, W [out][in_pad] (the forward B operand); the
// transposed copies W^T [in][out_pad] (input-gradient B operands) are made from
// it by transpose_w_kernel.
__device__ __forceinline__ void write_bf16_copies(const SgDev &d, const ParamRef &r, float v)
{
    if (r.bias) return;
    // layer 0: padding columns from kLoOff on hold the lo-part weights,
    // written only by the valid weights' own copies below
    if (r.layer == 0 && !r.valid && r.i >= kLoOff) return;
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    d.wb[r.layer][(int64_t)r.o * r.in_pad + r.i] = b;
    if (r.layer == 0 && r.valid) d.wb[0][(int64_t)r.o * r.in_pad + kLoOff + r.i] = b;   // weight of the input's lo part
}

// W^T [in][out_pad_k] of layers 1..L from their BF16 W [out_pad][in_pad], by
// 32 x 32 tiles through shared memory (both sides coalesced).  grid: (in / 32,
// max out_pad / 32, L), block 32 x 8.
__global__ void transpose_w_kernel(SgDev d)
{
    __shared__ __nv_bfloat16 tile[32][33];
    const int l = blockIdx.z + 1;
    const LayerLayout &Ly = d.lay[l];
    const int o0 = blockIdx.y * 32, i0 = blockIdx.x * 32;
    if (o0 >= Ly.out_pad || i0 >= Ly.in_pad) return;
    const int out_pad_k = (l == d.hidden) ? KIN : d.width;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int o = o0 + r;
        tile[r][threadIdx.x] = (o < Ly.out_pad) ? d.wb[l][(int64_t)o * Ly.in_pad + i0 + threadIdx.x]
                                                 : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int o = o0 + threadIdx.x;
        if (o < Ly.out_pad) d.wt[l][(int64_t)(i0 + r) * out_pad_k + o] = tile[threadIdx.x][r];
    }
}

void launch_transpose_w(const SgDev &d, cudaStream_t st)
{
    transpose_w_kernel<<<dim3(d.width / 32, d.width / 32, d.hidden), dim3(32, 8), 0, st>>>(d);
}

__global__ void refresh_bf16_kernel(SgDev d)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < d.n_master; e += (int64_t)gridDim.x * blockDim.x) {
        ParamRef r = decode_param(d, e);
        write_bf16_copies(d, r, d.master[e]);
    }
}

// ----------------------------------------------------------- normalization
// Per-block partial sums (FP64) of the 17 features / targets: sum, sum of
// squares, min, max.
__global__ void norm_partial_kernel(int64_t n, const float *x, int64_t ldx, const float *y, int64_t ldy,
                                    const SgDev d, double *part)
{
    double s[NSTAT], s2[NSTAT], mn[NSTAT], mx[NSTAT];
    double cnt = 0;
#pragma unroll
    for (int k = 0; k < NSTAT; ++k) { s[k] = 0; s2[k] = 0; mn[k] = 1e300; mx[k] = -1e300; }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float f[NIN], q[NOUT_MAX];
        features(x, ldx, i, d, f);
        targets(x, ldx, y, ldy, i, d, q);
        bool fin = true;
#pragma unroll
        for (int k = 0; k < NSTAT; ++k) fin = fin && (k >= NIN + d.nout || isfinite((k < NIN) ? f[k] : q[k - NIN]));
        if (!fin) continue;   // rows with a non-finite feature or target are left out
        cnt += 1;
#pragma unroll
        for (int k = 0; k < NSTAT; ++k) {
            const double v = (k < NIN) ? f[k] : q[k - NIN];
            s[k] += v; s2[k] += v * v; mn[k] = fmin(mn[k], v); mx[k] = fmax(mx[k], v);
        }
    }
    __shared__ double sh[4][NSTAT][8];
    __shared__ double shc[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) shc[warp] = cnt;
#pragma unroll
    for (int k = 0; k < NSTAT; ++k) {
        double a = s[k], b = s2[k], c = mn[k], e = mx[k];
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            c = fmin(c, __shfl_xor_sync(0xffffffffu, c, o));
            e = fmax(e, __shfl_xor_sync(0xffffffffu, e, o));
        }
        if (lane == 0) { sh[0][k][warp] = a; sh[1][k][warp] = b; sh[2][k][warp] = c; sh[3][k][warp] = e; }
    }
    __syncthreads();
    if (threadIdx.x < NSTAT) {
        const int k = threadIdx.x;
        double a = 0, b = 0, c = 1e300, e = -1e300;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += sh[0][k][w]; b += sh[1][k][w]; c = fmin(c, sh[2][k][w]); e = fmax(e, sh[3][k][w]);
        }
        double *p = part + ((int64_t)blockIdx.x * (NSTAT + 1) + k) * 4;
        p[0] = a; p[1] = b; p[2] = c; p[3] = e;
    }
    if (threadIdx.x == 0) {
        double c = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) c += shc[w];
        part[((int64_t)blockIdx.x * (NSTAT + 1) + NSTAT) * 4] = c;
    }
}

// Mean, standard deviation and the training hull (min/max widened by 1 % of
// the range) from the block partials, in the normalisation layout above.
__global__ void norm_final_kernel(int nblocks, const double *part, float *norm)
{
    const int k = threadIdx.x;
    if (k >= NSTAT) return;
    double a = 0, b = 0, c = 1e300, e = -1e300, n = 0;
    for (int blk = 0; blk < nblocks; ++blk) {
        const double *p = part + ((int64_t)blk * (NSTAT + 1) + k) * 4;
        a += p[0]; b += p[1]; c = fmin(c, p[2]); e = fmax(e, p[3]);
        n += part[((int64_t)blk * (NSTAT + 1) + NSTAT) * 4];
    }
    if (!(n > 0)) return;   // no valid row: keep the previous normalisation
    const double mean = a / n;
    double var = b / n - mean * mean;
    double sd = var > 0 ? sqrt(var) : 0.0;
    if (!(sd > 1e-12 * fmax(1.0, fabs(mean)))) sd = 1.0;
    if (k < NIN) {
        norm[k] = (float)mean;
        norm[NIN + k] = (float)sd;
        const double w = 0.01 * (e - c);
        norm[2 * NIN + 2 * NOUT6 + k] = (float)(c - w);
        norm[3 * NIN + 2 * NOUT6 + k] = (float)(e + w);
    } else {
        norm[out_mean_idx(k - NIN)] = (float)mean;
        norm[out_std_idx(k - NIN)] = (float)sd;
    }
}

// The output statistics gathered into one array, mean[16] then std[16], for
// the epilogues and the training targets.
__global__ void outstat_kernel(const float *norm, float *outstat)
{
    const int j = threadIdx.x;
    if (j < NOUT_MAX) {
        outstat[j] = norm[out_mean_idx(j)];
        outstat[NOUT_MAX + j] = norm[out_std_idx(j)];
    }
}

// ------------------------------------------------------------ prep kernels
// lo[k] = v[k] - bf16(v[k]): the part of each input that BF16 drops (exact in
// FP32; stored as BF16 it keeps the input to about 16 significant bits).
__device__ __forceinline__ void split_hi_lo(const float (&v)[16], float (&lo)[16])
{
#pragma unroll
    for (int k = 0; k < 16; ++k) lo[k] = v[k] - __bfloat162float(__float2bfloat16_rn(v[k]));
}

// Training batch: row r takes pool row src (in order when sample_seed == 0 and
// the pool is the batch, else uniformly at random with replacement).
__global__ void prep_train_kernel(SgDev d, int64_t B, int64_t n_pool, const float *x, int64_t ldx, const float *y,
                                  int64_t ldy, uint64_t sample_seed)
{
    const float *nm = d.norm;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < B; r += (int64_t)gridDim.x * blockDim.x) {
        int64_t src = r;
        if (sample_seed != 0 || n_pool != B) src = (int64_t)(splitmix64(sample_seed ^ ((uint64_t)r * 0xD1B54A32D192ED03ull)) % (uint64_t)n_pool);
        float f[NIN], q[NOUT_MAX];
        features(x, ldx, src, d, f);
        targets(x, ldx, y, ldy, src, d, q);
        float v[16], lo[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = (k < NIN) ? (f[k] - nm[k]) / nm[NIN + k] : 0.f;
        split_hi_lo(v, lo);
        store_row16_bf16(d.x0 + r * KIN, v);
        store_row16_bf16(d.x0 + r * KIN + kLoOff, lo);
#pragma unroll
        for (int j = 0; j < NOUT_MAX; ++j)
            if (j < d.nout) d.tgt[(int64_t)j * d.max_batch + r] = (q[j] - d.outstat[j]) / d.outstat[NOUT_MAX + j];
    }
}

// Inference chunk: standardised inputs, training-hull test, compaction of the
// cells outside the hull into `list` (chunk-local indices).
__global__ void prep_infer_kernel(SgDev d, int64_t r0, int64_t mc, const float *T, const float *p, const float *Y,
                                  int64_t ldY, uint8_t *flags, uint8_t *cflags, int32_t *list, unsigned int *count)
{
    const float *nm = d.norm;
    const float *lo = nm + 2 * NIN + 2 * NOUT6, *hi = lo + NIN;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < mc; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = r0 + r;
        float f[NIN];
        const float Ti = __ldg(T + i);   // h* for the inverse model
        f[1] = __ldg(p + i);
#pragma unroll
        for (int k = 0; k < 9; ++k) f[2 + k] = __ldg(Y + (int64_t)k * ldY + i);
        cell_features(d, Ti, f);
        bool out = false;
        float v[16], vlo[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (k < NIN) {
                out = out || !(f[k] >= lo[k] && f[k] <= hi[k]);
                v[k] = (f[k] - nm[k]) / nm[NIN + k];
            } else {
                v[k] = 0.f;
            }
        }
        split_hi_lo(v, vlo);
        store_row16_bf16(d.xi + r * KIN, v);
        store_row16_bf16(d.xi + r * KIN + kLoOff, vlo);
        if (d.mode == SG_MODE_FORWARD) {
            float Yk[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) Yk[k] = f[2 + k];
            d.hig[r] = h_ideal(Ti, Yk, d.sp32);
        }
        if (flags) flags[i] = out ? 1 : 0;
        cflags[r] = out ? 1 : 0;
        if (out) list[atomicAdd(count, 1u)] = (int32_t)r;
    }
}

// Low-confidence cells, appended to the fallback list (cells already on it
// are skipped through the chunk's flags):
//  * equation of state (forward model, tol > 0): the network predicts rho and
//    Z separately, while the equation of state ties them, rho Z R T = p W; a
//    cell whose two outputs disagree by more than `tol` is flagged;
//  * transport (property models, tol_tr > 0): Chung's correlation evaluated
//    in FP32 at the network's own density (and, for the inverse models, its
//    own temperature) and the cell's composition gives mu_c and lambda_c; a
//    cell whose predicted mu or lambda differs from them by more than tol_tr
//    (relative) is flagged.  The correlation's narrow excursions (the polar
//    and association terms of water-rich mixtures) are where the network is
//    least accurate, and a consistent density makes the check sharp there.
__global__ void __launch_bounds__(256) confidence_kernel(SgDev d, int64_t r0, int64_t mc, const float *T,
                                                         const float *p, const float *Y, int64_t ldY,
                                                         const float *out, int64_t ldo, float tol, float tol_tr,
                                                         uint8_t *flags, uint8_t *cflags, int32_t *list,
                                                         unsigned int *count)
{
    __shared__ SpeciesRec<float> s_sp[9];
    __shared__ float s_pair[81];
    {
        const float *src = static_cast<const float *>(d.sp32);
        float *dst = reinterpret_cast<float *>(s_sp);
        for (int j = threadIdx.x; j < (int)(9 * sizeof(SpeciesRec<float>) / 4); j += blockDim.x) dst[j] = src[j];
        for (int j = threadIdx.x; j < 81; j += blockDim.x) s_pair[j] = d.pair32[j];
    }
    __syncthreads();
    const bool fwd = d.mode == SG_MODE_FORWARD;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < mc; r += (int64_t)gridDim.x * blockDim.x) {
        if (cflags[r]) continue;
        const int64_t i = r0 + r;
        bool bad = false;
        if (fwd && tol > 0.f) {
            float s = 0.f;   // moles per kg = 1 / W
#pragma unroll
            for (int k = 0; k < 9; ++k) s = fmaf(__ldg(Y + (int64_t)k * ldY + i), s_sp[k].inv_W, s);
            const float c = out[i] * out[ldo + i] * float(prk::kR) * __ldg(T + i) * s / __ldg(p + i);
            bad = !(fabsf(c - 1.f) <= tol);
        }
        if (!bad && tol_tr > 0.f) {
            prk::Comp<float, 9> c;
            if (prk::load_comp<float, 9>(c, Y, ldY, i, 9, s_sp)) {
                const float Tc = fwd ? __ldg(T + i) : out[i];              // the network's T (inverse models)
                const float rho = fwd ? out[i] : out[ldo + i];
                const float mu = fwd ? out[4 * ldo + i] : out[3 * ldo + i];
                const float lam = fwd ? out[5 * ldo + i] : out[4 * ldo + i] * out[5 * ldo + i];   // alpha cp
                // ideal-gas molar cv (NASA-7) for the conductivity
                float cpm = 0.f;
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const float *a = (Tc < s_sp[k].T_mid) ? s_sp[k].cp_lo : s_sp[k].cp_hi;
                    const float cpk = fmaf(fmaf(fmaf(fmaf(a[4], Tc, a[3]), Tc, a[2]), Tc, a[1]), Tc, a[0]);
                    cpm = fmaf(c.x[k], cpk, cpm);
                }
                prk::Thermo<float> th;
                th.rho_mol = rho / c.Wbar;
                th.cv_ig_molar = cpm - float(prk::kR);
                float mu_c, lam_c;
                prk::transport<float, 9>(c, Tc, th, s_sp, s_pair, d.pr_flags, mu_c, lam_c);
                bad = !(fabsf(mu - mu_c) <= tol_tr * fabsf(mu_c)) || !(fabsf(lam - lam_c) <= tol_tr * fabsf(lam_c));
            }
        }
        if (bad) {
            cflags[r] = 1;
            if (flags) flags[i] = 1;
            list[atomicAdd(count, 1u)] = (int32_t)r;
        }
    }
}

// ---------------------------------------------------------- PR fallback
// FP64 Peng-Robinson properties of the listed cells (float inputs/outputs),
// one thread per listed cell.
template <int NS, bool KIJ>
__global__ void __launch_bounds__(128) fallback_kernel(const int32_t *list, const unsigned int *count, int64_t r0,
                                                       const float *T, const float *p, const float *Y, int64_t ldY,
                                                       float *out, int64_t ldo, const SpeciesRec<double> *sp,
                                                       const double *pair, const double *kij, int N, int flags,
                                                       double tmid_u)
{
    __shared__ SpeciesRec<double> s_sp[NS];
    __shared__ double s_pair[NS * NS];
    __shared__ double s_kij[NS * NS];
    {
        const double *src = reinterpret_cast<const double *>(sp);
        double *dst = reinterpret_cast<double *>(s_sp);
        for (int j = threadIdx.x; j < (int)(NS * sizeof(SpeciesRec<double>) / 8); j += blockDim.x) dst[j] = src[j];
        for (int j = threadIdx.x; j < NS * NS; j += blockDim.x) { s_pair[j] = pair[j]; s_kij[j] = kij[j]; }
    }
    __syncthreads();
    const unsigned int n = *count;
    for (unsigned int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        prk::fallback_cell_fp64<NS, KIJ>(r0 + list[t], T, p, Y, ldY, out, ldo, s_sp, s_pair, s_kij, N, flags,
                                         tmid_u);
}

// FP64 Peng-Robinson fallback of the inverse model for the listed cells: the
// safeguarded FP64 inversion T(h*, p, Y), started from the network's own T
// (clamped to the bracket; from 1000 K for a single-property network other than
// T), then rho, psi, mu, alpha, cp at that T; NaN where the inversion fails.
// sel < 0: all six outputs; sel = j: only property j, into output row 0.
template <int NS, bool KIJ>
__global__ void __launch_bounds__(128) fallback_inverse_kernel(const int32_t *list, const unsigned int *count,
                                                               int64_t r0, const float *H, const float *p,
                                                               const float *Y, int64_t ldY, float *out, int64_t ldo,
                                                               const SpeciesRec<double> *sp, const double *pair,
                                                               const double *kij, int N, int flags, int sel)
{
    __shared__ SpeciesRec<double> s_sp[NS];
    __shared__ double s_pair[NS * NS];
    __shared__ double s_kij[NS * NS];
    {
        const double *src = reinterpret_cast<const double *>(sp);
        double *dst = reinterpret_cast<double *>(s_sp);
        for (int j = threadIdx.x; j < (int)(NS * sizeof(SpeciesRec<double>) / 8); j += blockDim.x) dst[j] = src[j];
        for (int j = threadIdx.x; j < NS * NS; j += blockDim.x) { s_pair[j] = pair[j]; s_kij[j] = kij[j]; }
    }
    __syncthreads();
    const unsigned int n = *count;
    for (unsigned int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int64_t i = r0 + list[t];
        const double hv = (double)__ldg(H + i), pv = (double)__ldg(p + i);
        prk::Comp<double, NS> c;
        bool ok = prk::comp_fp64_of_fp32<NS>(c, Y, ldY, i, N, s_sp) && (pv > 0) && isfinite(hv) && isfinite(pv);
        float o[6];
        for (int q = 0; q < 6; ++q) o[q] = __int_as_float(0x7fc00000);
        if (ok) {
            double T0 = (sel <= 0) ? (double)out[i] : 1000.0;   // the network's T
            if (!(T0 == T0)) T0 = 300.0;
            T0 = fmin(fmax(T0, prk::kTLo), prk::kTHi);
            double T, cpl;
            int it;
            const int st = prk::newton_solve<double, double, NS, KIJ>(c, hv, pv, T0, s_sp, s_kij, 0.0, 60, 1e-12, 1e-6, T,
                                                                     it, cpl);
            if (st == prk::kOk) {
                prk::Thermo<double> th;
                prk::thermo<double, double, NS, KIJ>(c, T, pv, s_sp, s_kij, th);
                if (th.status != prk::kNoRoot) {
                    double mu, lam;
                    prk::transport<double, NS>(c, T, th, s_sp, s_pair, flags, mu, lam);
                    o[0] = (float)T;
                    o[1] = (float)(pv * c.Wbar / (th.Z * prk::kR * T));
                    o[2] = (float)prk::psi_h<double>(th, T, c.Wbar);
                    o[3] = (float)mu;
                    o[4] = (float)(lam / th.cp);
                    o[5] = (float)th.cp;
                }
            }
        }
        if (sel >= 0) {
            out[i] = o[sel < 6 ? sel : 0];
        } else {
#pragma unroll
            for (int q = 0; q < 6; ++q) out[(int64_t)q * ldo + i] = o[q];
        }
    }
}

// Per-species outputs of cells outside the hull: the FP64 inversion T(h, p, Y)
// started from the network's own T estimate is not available here (the
// outputs are per-species quantities), so it starts from 1000 K, then the
// FP64 per-species values at that T: D_k (with the context's correction
// table) or h_k / (R T).  NaN where the inversion fails.
template <int NS, bool KIJ>
__global__ void __launch_bounds__(128) fallback_species_kernel(const int32_t *list, const unsigned int *count,
                                                               int64_t r0, const float *H, const float *p,
                                                               const float *Y, int64_t ldY, float *out, int64_t ldo,
                                                               const SpeciesRec<double> *sp, const double *kij,
                                                               const double *dtab, const double *corr, int cT,
                                                               int cP, int N, int outputs)
{
    __shared__ SpeciesRec<double> s_sp[NS];
    __shared__ double s_kij[NS * NS];
    __shared__ double s_tab[2 * NS + 3 * NS * NS];
    {
        const double *src = reinterpret_cast<const double *>(sp);
        double *dst = reinterpret_cast<double *>(s_sp);
        for (int j = threadIdx.x; j < (int)(NS * sizeof(SpeciesRec<double>) / 8); j += blockDim.x) dst[j] = src[j];
        for (int j = threadIdx.x; j < NS * NS; j += blockDim.x) s_kij[j] = kij[j];
        for (int j = threadIdx.x; j < 2 * NS + 3 * NS * NS; j += blockDim.x) s_tab[j] = dtab[j];
    }
    __syncthreads();
    const unsigned int n = *count;
    for (unsigned int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int64_t i = r0 + list[t];
        const double hv = (double)__ldg(H + i), pv = (double)__ldg(p + i);
        prk::Comp<double, NS> c;
        bool ok = prk::comp_fp64_of_fp32<NS>(c, Y, ldY, i, N, s_sp) && (pv > 0) && isfinite(hv) && isfinite(pv);
        double o[NS];
#pragma unroll
        for (int k = 0; k < NS; ++k) o[k] = __longlong_as_double(0x7ff8000000000000ULL);
        if (ok) {
            double T, cpl;
            int it;
            const int st = prk::newton_solve<double, double, NS, KIJ>(c, hv, pv, 1000.0, s_sp, s_kij, 0.0, 60, 1e-12, 1e-6,
                                                                     T, it, cpl);
            if (st == prk::kOk) {
                if (outputs == SG_OUT_HK) {
                    const double iRT = 1.0 / (prk::kR * T);
#pragma unroll
                    for (int k = 0; k < NS; ++k)
                        if (k < N) o[k] = prs::h_over_RT<double>(T < s_sp[k].T_mid ? s_sp[k].h_lo : s_sp[k].h_hi, T, iRT);
                } else {
                    double y[NS], ysum = 0.0;
#pragma unroll
                    for (int k = 0; k < NS; ++k) {
                        y[k] = (k < N) ? (double)__ldg(Y + (int64_t)k * ldY + i) : 0.0;
                        ysum += y[k];
                    }
                    prs::diffusion_cell<double, NS>(y, c.x, ysum, T, pv, N, s_tab, corr, cT, cP, o);
                }
            }
        }
        for (int k = 0; k < N; ++k) out[(int64_t)k * ldo + i] = (float)o[k];
    }
}

// ------------------------------------------------------------------- Adam
// Bias gradients: one warp per (layer, output) sums the per-M-tile column sums
// of dz (nct of them), lanes striding over the tiles.
__global__ void bias_grad_kernel(SgDev d, int64_t nct)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int l = (int)(wid / d.width), o = (int)(wid % d.width);
    if (l > d.hidden) return;
    const int ncol = d.lay[l].out_pad;
    if (o >= ncol) return;
    const float *cs = d.colsum[l];
    float g = 0.f;
    for (int64_t c = lane; c < nct; c += 32) g += cs[c * ncol + o];
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) g += __shfl_xor_sync(0xffffffffu, g, k);
    if (lane == 0) d.bgrad[(int64_t)l * d.width + o] = g;
}

__global__ void adam_kernel(SgDev d, float lr, float b1, float b2, float eps, int t, int export_only,
                            float *grad_out)
{
    const float bc1 = 1.f - powf(b1, (float)t), bc2 = 1.f - powf(b2, (float)t);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < d.n_master; e += (int64_t)gridDim.x * blockDim.x) {
        ParamRef r = decode_param(d, e);
        if (!r.valid) continue;
        float g = 0.f;
        if (r.bias) {
            g = d.bgrad[(int64_t)r.layer * d.width + r.o];
        } else {
            // split-K partials; four independent sums keep four loads in flight
            const float *pp = d.partial[r.layer] + (int64_t)r.o * r.in_pad + r.i;
            const int64_t plane = (int64_t)d.dw_mpad[r.layer] * r.in_pad;
            const int ns = d.dw_splits[r.layer];
            float g4[4] = {0.f, 0.f, 0.f, 0.f};
            int s = 0;
            for (; s + 4 <= ns; s += 4) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    g4[u] += pp[(s + u) * plane];
                    if (r.layer == 0) g4[u] += pp[(s + u) * plane + kLoOff];   // tied lo weight
                }
            }
            for (; s < ns; ++s) {
                g4[0] += pp[s * plane];
                if (r.layer == 0) g4[0] += pp[s * plane + kLoOff];
            }
            g = (g4[0] + g4[1]) + (g4[2] + g4[3]);
        }
        if (export_only) {
            grad_out[r.flat] = g;
            continue;
        }
        const float m = b1 * d.adam_m[e] + (1.f - b1) * g;
        const float v = b2 * d.adam_v[e] + (1.f - b2) * g * g;
        d.adam_m[e] = m;
        d.adam_v[e] = v;
        const float w = d.master[e] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
        d.master[e] = w;
        write_bf16_copies(d, r, w);
    }
}

// one thread per master element (n_master ~ 10^6: a few thousand blocks)
inline int adam_blocks(const SgDev &d) { return (int)((d.n_master + 255) / 256); }

__global__ void loss_final_kernel(const float *part, int64_t nct, float scale, float *loss_out)
{
    __shared__ float sh[256];
    float s = 0.f;
    for (int64_t c = threadIdx.x; c < nct; c += blockDim.x) s += part[c];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss_out = sh[0] * scale;
}

__global__ void copy_params_kernel(SgDev d, float *flat, int to_flat)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < d.n_master; e += (int64_t)gridDim.x * blockDim.x) {
        ParamRef r = decode_param(d, e);
        if (!r.valid) continue;
        if (to_flat) flat[r.flat] = d.master[e];
        else d.master[e] = flat[r.flat];
    }
}

// --------------------------------------------------------- tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// K-major BF16 operand [rows][inner] with row pitch `pitch` elements, loaded
// in boxes of 64 x box_rows with 128-byte swizzling (out-of-range rows and
// columns read as zero).
bool make_map(CUtensorMap *m, const void *ptr, uint64_t inner, uint64_t rows, uint64_t pitch, uint32_t box_rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {pitch * 2};
    cuuint32_t box[2] = {64, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool make_map_3d(CUtensorMap *m, const void *ptr, uint64_t inner, uint64_t rows, uint64_t depth, uint32_t box_rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {inner, rows, depth};
    cuuint64_t strides[2] = {inner * 2, inner * rows * 2};
    cuuint32_t box[3] = {64, box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int num_sms_current()
{
    static int sms[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 148;
    if (!sms[dev]) cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
    return sms[dev] > 0 ? sms[dev] : 148;
}

// Persistent launch: one CTA per SM (or fewer when there are fewer tiles).
template <int BN, int EPI>
cudaError_t launch_gemm(const CUtensorMap &ta, const CUtensorMap &tb, GemmArgs a, int m_tiles, int n_tiles,
                        int splits, cudaStream_t st)
{
    static int dev_ready[64] = {0};   // per device: shared-memory attribute set
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    a.m_tiles = m_tiles;
    a.n_tiles = n_tiles;
    a.splits = splits;
    const int tiles = m_tiles * n_tiles * splits;
    if (!dev_ready[dev]) {
        cudaError_t e =
            cudaFuncSetAttribute(gemm_kernel<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<BN>::SMEM);
        if (e != cudaSuccess) return e;
        dev_ready[dev] = 1;
    }
    const int sms = num_sms_current();
    gemm_kernel<BN, EPI><<<tiles < sms ? tiles : sms, kThreads, Cfg<BN>::SMEM, st>>>(ta, tb, a);
    return cudaGetLastError();
}

// Widest N tile (256, 128, 64 or 16) that divides N.
inline int pick_bn(int N) { return (N % 256 == 0) ? 256 : (N % 128 == 0) ? 128 : (N % 64 == 0) ? 64 : 16; }

// Dispatch on the N tile width.
template <int EPI>
cudaError_t launch_gemm_n(const CUtensorMap &ta, const CUtensorMap &tb, const GemmArgs &a, int m_tiles, int N,
                          int splits, cudaStream_t st)
{
    switch (pick_bn(N)) {
    case 256: return launch_gemm<256, EPI>(ta, tb, a, m_tiles, N / 256, splits, st);
    case 128: return launch_gemm<128, EPI>(ta, tb, a, m_tiles, N / 128, splits, st);
    case 64: return launch_gemm<64, EPI>(ta, tb, a, m_tiles, N / 64, splits, st);
    default: return launch_gemm<16, EPI>(ta, tb, a, m_tiles, N / 16, splits, st);
    }
}

// Weight-gradient GEMM with MN-major operands: N tiles of 256, 128 or 64.
cudaError_t launch_gemm_dw_mn(const CUtensorMap &ta, const CUtensorMap &tb, GemmArgs a, int m_tiles, int N,
                              int splits, cudaStream_t st)
{
    switch (pick_bn(N)) {
    case 256: return launch_gemm<256, kEpiDwMN>(ta, tb, a, m_tiles, N / 256, splits, st);
    case 128: return launch_gemm<128, kEpiDwMN>(ta, tb, a, m_tiles, N / 128, splits, st);
    case 64: return launch_gemm<64, kEpiDwMN>(ta, tb, a, m_tiles, N / 64, splits, st);
    default: return cudaErrorInvalidValue;
    }
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// One cooperative launch of the fused inference kernel (all CTAs resident:
// they wait on one another's arrival counters) over `units` CTAs or, for
// PAIR, CTA pairs (clusters of two).
template <bool PAIR>
cudaError_t launch_fused(const FusedArgs &fa, int units, cudaStream_t st)
{
    static int dev_ready[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!dev_ready[dev]) {
        cudaError_t e = cudaFuncSetAttribute(mlp_fused_kernel<PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             FusedCfg<PAIR>::kMaxSmem);
        if (e != cudaSuccess) return e;
        if (!PAIR) {
            int occ = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mlp_fused_kernel<PAIR>, kFusedThreads,
                                                              FusedCfg<PAIR>::kMaxSmem);
            if (e != cudaSuccess) return e;
            if (occ < 1) return cudaErrorInvalidConfiguration;
        }
        dev_ready[dev] = 1;
    }
    const long long g = fa.total < units ? fa.total : units;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = 2;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)((PAIR ? 2 : 1) * g), 1, 1);
    cfg.blockDim = dim3(kFusedThreads, 1, 1);
    cfg.dynamicSmemBytes = FusedCfg<PAIR>::smem_bytes(fa.L, fa.W);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = PAIR ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, mlp_fused_kernel<PAIR>, fa);
}

// CTA pairs of the fused kernel that the device holds at once (0: none, or
// cluster launches unavailable).
int fused_pair_clusters(int L, int W)
{
    if (cudaFuncSetAttribute(mlp_fused_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             FusedCfg<true>::kMaxSmem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * num_sms_current(), 1, 1);
    cfg.blockDim = dim3(kFusedThreads, 1, 1);
    cfg.dynamicSmemBytes = FusedCfg<true>::smem_bytes(L, W);
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, mlp_fused_kernel<true>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nc;
}

// Slot lag D between consecutive layers, about three rounds of G concurrent
// units (an item's inputs are released about two rounds after its producer
// item's turn), and the ring size 2 D + 4 (a ring unit is rewritten about
// three rounds after its readers' turn).
void fused_lag(int G, int ips, int &D, int &ring)
{
    const int lagmin = (G + 2 * ips + ips - 1) / ips;   // slots with D ips > G + ips
    const int three_rounds = (3 * G + ips - 1) / ips;
    D = three_rounds > lagmin + 4 ? three_rounds : lagmin + 4;
    ring = 2 * D + 4;
}

// The resident-activation kernel for width W (256 or 512) and this depth (the
// output layer's weights resident in shared memory when they fit).
inline const void *resident_fn(int L, int W)
{
    const bool wo = ResCfg::wout_resident(L, W);
    if (W == 256) return wo ? reinterpret_cast<const void *>(mlp_resident_kernel<256, true>)
                            : reinterpret_cast<const void *>(mlp_resident_kernel<256, false>);
    return wo ? reinterpret_cast<const void *>(mlp_resident_kernel<512, true>)
              : reinterpret_cast<const void *>(mlp_resident_kernel<512, false>);
}

// CTA pairs of the resident-activation kernel the device holds at once (0:
// none, or cluster launches unavailable).
int resident_pairs(int L, int W)
{
    if (cudaFuncSetAttribute(resident_fn(L, W), cudaFuncAttributeMaxDynamicSharedMemorySize, ResCfg::kMaxSmem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * num_sms_current(), 1, 1);
    cfg.blockDim = dim3(kResThreads, 1, 1);
    cfg.dynamicSmemBytes = ResCfg::smem_bytes(L, W, ResCfg::wout_resident(L, W));
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, resident_fn(L, W), &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nc;
}

inline const void *pingpong_fn(int L, int W)
{
    const bool wo = PPCfg::wout_resident(L, W);
    if (W == 256) return wo ? reinterpret_cast<const void *>(mlp_pingpong_kernel<256, true>)
                            : reinterpret_cast<const void *>(mlp_pingpong_kernel<256, false>);
    return wo ? reinterpret_cast<const void *>(mlp_pingpong_kernel<512, true>)
              : reinterpret_cast<const void *>(mlp_pingpong_kernel<512, false>);
}

// CTA pairs of the alternating-activation kernel the device holds at once
// (0: none, or cluster launches unavailable).
int pingpong_pairs(int L, int W)
{
    if (cudaFuncSetAttribute(pingpong_fn(L, W), cudaFuncAttributeMaxDynamicSharedMemorySize, PPCfg::kMaxSmem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * num_sms_current(), 1, 1);
    cfg.blockDim = dim3(kPPThreads, 1, 1);
    cfg.dynamicSmemBytes = PPCfg::smem_bytes(L, W, PPCfg::wout_resident(L, W));
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, pingpong_fn(L, W), &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nc;
}

// One launch of the alternating-activation kernel (as launch_resident).
cudaError_t launch_pingpong(const ResidentArgs &ra, int pairs, cudaStream_t st)
{
    const int R = (ra.M + 255) / 256;
    const int g = R < pairs ? R : pairs;
    const bool wo = PPCfg::wout_resident(ra.L, ra.W);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(2 * g), 1, 1);
    cfg.blockDim = dim3(kPPThreads, 1, 1);
    cfg.dynamicSmemBytes = PPCfg::smem_bytes(ra.L, ra.W, wo);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (ra.W == 256)
        return wo ? cudaLaunchKernelEx(&cfg, mlp_pingpong_kernel<256, true>, ra)
                  : cudaLaunchKernelEx(&cfg, mlp_pingpong_kernel<256, false>, ra);
    return wo ? cudaLaunchKernelEx(&cfg, mlp_pingpong_kernel<512, true>, ra)
              : cudaLaunchKernelEx(&cfg, mlp_pingpong_kernel<512, false>, ra);
}

// One launch of the resident-activation kernel: a pair per block of 256 rows,
// at most `pairs` pairs (each walks its blocks in turn; pairs never wait on
// one another, so no co-residency is needed).
cudaError_t launch_resident(const ResidentArgs &ra, int pairs, cudaStream_t st)
{
    const int R = (ra.M + 255) / 256;
    const int g = R < pairs ? R : pairs;
    const bool wo = ResCfg::wout_resident(ra.L, ra.W);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(2 * g), 1, 1);
    cfg.blockDim = dim3(kResThreads, 1, 1);
    cfg.dynamicSmemBytes = ResCfg::smem_bytes(ra.L, ra.W, wo);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (ra.W == 256)
        return wo ? cudaLaunchKernelEx(&cfg, mlp_resident_kernel<256, true>, ra)
                  : cudaLaunchKernelEx(&cfg, mlp_resident_kernel<256, false>, ra);
    return wo ? cudaLaunchKernelEx(&cfg, mlp_resident_kernel<512, true>, ra)
              : cudaLaunchKernelEx(&cfg, mlp_resident_kernel<512, false>, ra);
}

GemmArgs base_args(sg_model *m)
{
    GemmArgs a;
    memset(&a, 0, sizeof(a));
    a.err = m->d_err;
    return a;
}

}  // namespace

// ===================================================== host-side plumbing
static pr_status build_maps(sg_model *m)
{
    SgDev &d = m->dev;
    const int W = m->width, L = m->hidden;
    const int64_t B = m->max_batch, C = m->chunk;
    bool ok = true;
    // weights (forward B operands): one box holds a whole N tile of the GEMMs with N = W
    const uint32_t bw = (uint32_t)pick_bn(W);
    ok = ok && make_map(&m->tm_w[0], d.wb[0], KIN, W, KIN, bw);
    for (int l = 1; l < L; ++l) ok = ok && make_map(&m->tm_w[l], d.wb[l], W, W, W, bw);
    ok = ok && make_map(&m->tm_w[L], d.wb[L], W, NOP, W, 16);
    // transposed weights (input-gradient B operands)
    for (int l = 1; l < L; ++l) ok = ok && make_map(&m->tm_wt[l], d.wt[l], W, W, W, bw);
    ok = ok && make_map(&m->tm_wt[L], d.wt[L], KIN, W, KIN, bw);
    // training activations
    ok = ok && make_map(&m->tm_x0, d.x0, KIN, B, KIN, 128);
    ok = ok && make_map(&m->tmn_x0, d.x0, KIN, B, KIN, 64);
    for (int l = 0; l < L; ++l) {
        ok = ok && make_map(&m->tm_h[l], d.h[l], W, B, W, 128);
        ok = ok && make_map(&m->tmn_h[l], d.h[l], W, B, W, 64);
        ok = ok && make_map(&m->tm_dz[l], d.dz[l], W, B, W, 128);
        ok = ok && make_map(&m->tmn_dz[l], d.dz[l], W, B, W, 64);
    }
    ok = ok && make_map(&m->tm_dzo, d.dzo, KIN, B, KIN, 128);
    ok = ok && make_map(&m->tmn_dzo, d.dzo, KIN, B, KIN, 64);
    // inference
    ok = ok && make_map(&m->tm_xi, d.xi, KIN, C, KIN, 128);
    ok = ok && make_map(&m->tm_hi[0], d.hi[0], W, C, W, 128);
    ok = ok && make_map(&m->tm_hi[1], d.hi[1], W, C, W, 128);
    // epilogue stores
    for (int l = 0; l < L; ++l) {
        ok = ok && make_map(&m->ts_h[l], d.h[l], W, B, W, 32);
        ok = ok && make_map(&m->ts_g[l], d.g[l], W, B, W, 32);
        ok = ok && make_map(&m->ts_dz[l], d.dz[l], W, B, W, 32);
    }
    ok = ok && make_map(&m->ts_hi[0], d.hi[0], W, C, W, 32);
    ok = ok && make_map(&m->ts_hi[1], d.hi[1], W, C, W, 32);
    // fused inference
    if (m->fused_ok) {
        ok = ok && make_map(&m->tmf_w[0], d.wb[0], KIN, W, KIN, kFusedBN);
        for (int l = 1; l < L; ++l) ok = ok && make_map(&m->tmf_w[l], d.wb[l], W, W, W, kFusedBN);
        m->tmf_w[L] = m->tm_w[L];
        if (m->fused_pair_ok) {   // each CTA of a pair loads half of every weight tile
            ok = ok && make_map(&m->tmp_w[0], d.wb[0], KIN, W, KIN, kFusedBN / 2);
            for (int l = 1; l < L; ++l) ok = ok && make_map(&m->tmp_w[l], d.wb[l], W, W, W, kFusedBN / 2);
            ok = ok && make_map(&m->tmp_w[L], d.wb[L], W, NOP, W, kFusedOutBN / 2);
        }
        if (m->res_pairs > 0) {   // resident activations: each CTA of a pair loads half of every N-tile
            ok = ok && make_map(&m->tmr_w[0], d.wb[0], KIN, W, KIN, (uint32_t)(W / 4));
            for (int l = 1; l < L; ++l) ok = ok && make_map(&m->tmr_w[l], d.wb[l], W, W, W, (uint32_t)(W / 4));
            ok = ok && make_map(&m->tmr_w[L], d.wb[L], W, NOP, W, 8);
        }
        if (m->pp_pairs > 0) {   // alternating activations: a CTA's 64 rows of every 128-row N-tile
            ok = ok && make_map(&m->tmq_w[0], d.wb[0], KIN, W, KIN, (uint32_t)(kPPBN / 2));
            for (int l = 1; l < L; ++l) ok = ok && make_map(&m->tmq_w[l], d.wb[l], W, W, W, (uint32_t)(kPPBN / 2));
            ok = ok && make_map(&m->tmq_w[L], d.wb[L], W, NOP, W, 8);
        }
        const int64_t rr = (int64_t)m->fused_ring_rows * 128;
        ok = ok && make_map_3d(&m->tmf_ring_ld, m->ring, W, rr, L, 128);
        ok = ok && make_map_3d(&m->tmf_ring_st, m->ring, W, rr, L, 32);
    }
    if (!ok) {
        prgb::set_error("surrogate: cuTensorMapEncodeTiled unavailable or failed");
        return PR_ECUDA;
    }
    return PR_OK;
}

static void free_model(sg_model *m)
{
    if (!m) return;
    for (void *p : m->allocs) cudaFree(p);
    for (cudaEvent_t e : m->tev) cudaEventDestroy(e);
    delete m;
}

extern "C" {

pr_status surrogate_create(pr_ctx *ctx, const sg_config *cfg, uint64_t seed, sg_model **out)
{
    PR_CHECK_ARG(ctx && cfg && out, "surrogate_create: null argument");
    *out = nullptr;
    PR_CHECK_ARG(ctx->n_species == 9, "surrogate_create: the surrogate takes 9 species, context has %d", ctx->n_species);
    PR_CHECK_ARG(cfg->width == 512 || cfg->width == 256 || cfg->width == 128 || cfg->width == 1024,
                 "surrogate_create: width must be 128, 256, 512 or 1024");
    PR_CHECK_ARG(cfg->hidden_layers >= 1 && cfg->hidden_layers <= SG_MAX_HIDDEN, "surrogate_create: hidden_layers 1..%d",
                 SG_MAX_HIDDEN);
    PR_CHECK_ARG(cfg->max_batch >= 128 && cfg->max_batch % 128 == 0 && cfg->max_batch <= (1 << 22),
                 "surrogate_create: max_batch must be a multiple of 128 in [128, 4194304]");
    PR_CHECK_ARG(cfg->infer_chunk >= 128 && cfg->infer_chunk % 128 == 0 && cfg->infer_chunk <= (1 << 24),
                 "surrogate_create: infer_chunk must be a multiple of 128 in [128, 16777216]");
    sg_model *m = new (std::nothrow) sg_model();
    if (!m) { prgb::set_error("surrogate_create: host allocation failed"); return PR_ENOMEM; }
    m->ctx = ctx;
    m->seed = seed;
    m->width = cfg->width;
    m->hidden = cfg->hidden_layers;
    m->max_batch = cfg->max_batch;
    m->chunk = cfg->infer_chunk;
    m->step = 0;
    m->norm_blocks = 2 * ctx->num_sms;
    SgDev &d = m->dev;
    memset(&d, 0, sizeof(d));
    d.width = m->width;
    d.hidden = m->hidden;
    d.max_batch = m->max_batch;
    d.sp32 = ctx->d_sp32;
    d.pair32 = ctx->d_pair32;
    d.pr_flags = ctx->flags;
    d.bilger = ctx->d_bilger32;
    d.bc_lambda = 1.0f;      // Box-Cox of Bilger's Z: linear until surrogate_set_boxcox
    d.bc_shift = 1e-3f;
    d.nout = NOUT6;
    d.outputs = SG_OUT_PROPS;
    const int W = m->width, L = m->hidden;
    const int64_t B = m->max_batch, C = m->chunk;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
        if (e != cudaSuccess) return;
        e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) {
            m->allocs.push_back(*p);
            e = cudaMemset(*p, 0, bytes);
        }
    };
    // parameter layout: per layer W [out_pad][in_pad] then b [out_pad]
    int64_t off = 0, flat = 0;
    for (int l = 0; l <= L; ++l) {
        const int in = (l == 0) ? NIN : W, in_pad = (l == 0) ? KIN : W;
        const int out = (l == L) ? NOUT6 : W, out_pad = (l == L) ? NOP : W;
        d.lay[l] = {off, off + (int64_t)out_pad * in_pad, in, in_pad, out, out_pad, flat};
        off += (int64_t)out_pad * in_pad + out_pad;
        flat += (int64_t)out * in + out;
    }
    d.n_master = off;
    d.n_flat = flat;
    alloc((void **)&d.master, off * 4);
    alloc((void **)&d.adam_m, off * 4);
    alloc((void **)&d.adam_v, off * 4);
    for (int l = 0; l <= L; ++l) {
        alloc((void **)&d.wb[l], (size_t)d.lay[l].out_pad * d.lay[l].in_pad * 2);
        if (l > 0) {
            const int out_pad_k = (l == L) ? KIN : W;   // K of the input-gradient GEMM
            alloc((void **)&d.wt[l], (size_t)d.lay[l].in_pad * out_pad_k * 2);
        }
    }
    alloc((void **)&d.norm, SG_NORM_FLOATS * 4);
    alloc((void **)&d.outstat, 2 * NOUT_MAX * 4);
    alloc((void **)&d.x0, B * KIN * 2);
    alloc((void **)&d.tgt, (int64_t)NOUT_MAX * B * 4);
    for (int l = 0; l < L; ++l) {
        alloc((void **)&d.h[l], B * W * 2);
        alloc((void **)&d.g[l], B * W * 2);
        alloc((void **)&d.dz[l], B * W * 2);
    }
    alloc((void **)&d.dzo, B * KIN * 2);
    // weight-gradient partials: splits chosen so that tiles x splits ~ SM count
    const int kb = (int)(B / 64);
    for (int l = 0; l <= L; ++l) {
        const int mp = (l == L) ? MOP : W;
        const int np = d.lay[l].in_pad;
        const int bn = pick_bn(np);
        const int tiles = (mp / 128) * (np / bn);
        int splits = ctx->num_sms / tiles;
        splits = splits < 1 ? 1 : (splits > kb ? kb : splits);
        const int kps = (kb + splits - 1) / splits;
        splits = (kb + kps - 1) / kps;
        d.dw_splits[l] = splits;
        d.dw_kps[l] = kps;
        d.dw_mpad[l] = mp;
        alloc((void **)&d.partial[l], (size_t)splits * mp * np * 4);
        const int ncol = (l == L) ? NOP : W;
        alloc((void **)&d.colsum[l], (size_t)(B / 128) * ncol * 4);
        if (l == 0) alloc((void **)&d.bgrad, (size_t)(L + 1) * W * 4);
    }
    alloc((void **)&d.loss_part, (B / 128) * 4);
    alloc((void **)&m->d_loss, 4);
    alloc((void **)&m->d_err, 4);
    alloc((void **)&m->d_normpart, (size_t)m->norm_blocks * (NSTAT + 1) * 4 * 8);
    alloc((void **)&d.xi, C * KIN * 2);
    alloc((void **)&d.hig, C * 4);
    // fused inference (mlp_fused.cuh), with single-CTA tiles or CTA pairs
    m->fused_ok = (W % kFusedBN == 0) && W <= 1024 && L <= SG_MAX_HIDDEN &&
                  FusedCfg<false>::smem_bytes(L, W) <= FusedCfg<false>::kMaxSmem;
    if (m->fused_ok) {
        const int ips = L * (W / kFusedBN) + 1;
        fused_lag(ctx->num_sms, ips, m->fused_D, m->fused_ring);
        m->fused_ring_rows = m->fused_ring;
        m->fused_clusters = (FusedCfg<true>::smem_bytes(L, W) <= FusedCfg<true>::kMaxSmem) ? fused_pair_clusters(L, W) : 0;
        m->fused_pair_ok = m->fused_clusters > 0;
        if (m->fused_pair_ok) {
            fused_lag(m->fused_clusters, ips, m->fused_D2, m->fused_ring2);
            if (2 * m->fused_ring2 > m->fused_ring_rows) m->fused_ring_rows = 2 * m->fused_ring2;
        }
        alloc((void **)&m->ring, (size_t)L * m->fused_ring_rows * 128 * W * 2);
        alloc((void **)&m->d_done, (size_t)ceil_div(C, 128) * (L + 1) * 4);
        m->res_pairs = ResCfg::supports(L, W) ? resident_pairs(L, W) : 0;
        m->pp_pairs = PPCfg::supports(L, W) ? pingpong_pairs(L, W) : 0;
    }
    m->fused_on = m->res_pairs > 0 ? 3 : m->fused_ok;   // resident activations where the shape allows
    alloc((void **)&d.hi[0], C * W * 2);
    alloc((void **)&d.hi[1], C * W * 2);
    alloc((void **)&m->d_list, C * 4);
    alloc((void **)&m->d_count, 16);
    alloc((void **)&m->d_flags, C);
    if (e == cudaSuccess) {
        // default normalisation: identity, unbounded hull
        float nm[SG_NORM_FLOATS];
        for (int k = 0; k < SG_NORM_FLOATS; ++k) nm[k] = 0.f;
        for (int k = 0; k < NIN; ++k) { nm[NIN + k] = 1.f; nm[2 * NIN + 2 * NOUT6 + k] = -3e38f; nm[3 * NIN + 2 * NOUT6 + k] = 3e38f; }
        for (int j = 0; j < NOUT_MAX; ++j) nm[out_std_idx(j)] = 1.f;
        e = cudaMemcpy(d.norm, nm, sizeof(nm), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            outstat_kernel<<<1, 32>>>(d.norm, d.outstat);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        init_params_kernel<<<256, 256>>>(d, seed ? seed : 1);
        refresh_bf16_kernel<<<256, 256>>>(d);
        launch_transpose_w(d, 0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        prgb::set_error("surrogate_create: %s", cudaGetErrorString(e));
        free_model(m);
        return e == cudaErrorMemoryAllocation ? PR_ENOMEM : PR_ECUDA;
    }
    pr_status s = build_maps(m);
    if (s) { free_model(m); return s; }
    *out = m;
    return PR_OK;
}

void surrogate_destroy(sg_model *m)
{
    if (!m) return;
    cudaDeviceSynchronize();
    free_model(m);
}

int64_t surrogate_num_params(const sg_model *m) { return m ? m->dev.n_flat : -1; }

pr_status surrogate_get_params(const sg_model *m, float *host_dst, int64_t n)
{
    PR_CHECK_ARG(m && host_dst && n == m->dev.n_flat, "surrogate_get_params: bad arguments");
    float *tmp = nullptr;
    PR_CUDA_TRY(cudaDeviceSynchronize());
    PR_CUDA_TRY(cudaMalloc(&tmp, n * 4));
    copy_params_kernel<<<256, 256>>>(m->dev, tmp, 1);
    cudaError_t e = cudaMemcpy(host_dst, tmp, n * 4, cudaMemcpyDeviceToHost);
    cudaFree(tmp);
    PR_CUDA_TRY(e);
    return PR_OK;
}

pr_status surrogate_set_params(sg_model *m, const float *host_src, int64_t n)
{
    PR_CHECK_ARG(m && host_src && n == m->dev.n_flat, "surrogate_set_params: bad arguments");
    float *tmp = nullptr;
    PR_CUDA_TRY(cudaDeviceSynchronize());
    PR_CUDA_TRY(cudaMalloc(&tmp, n * 4));
    cudaError_t e = cudaMemcpy(tmp, host_src, n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        copy_params_kernel<<<256, 256>>>(m->dev, tmp, 0);
        refresh_bf16_kernel<<<256, 256>>>(m->dev);
        launch_transpose_w(m->dev, 0);
        e = cudaDeviceSynchronize();
    }
    cudaFree(tmp);
    PR_CUDA_TRY(e);
    return PR_OK;
}

pr_status surrogate_get_normalization(const sg_model *m, float *host_dst)
{
    PR_CHECK_ARG(m && host_dst, "surrogate_get_normalization: null argument");
    PR_CUDA_TRY(cudaDeviceSynchronize());
    PR_CUDA_TRY(cudaMemcpy(host_dst, m->dev.norm, SG_NORM_FLOATS * 4, cudaMemcpyDeviceToHost));
    return PR_OK;
}

pr_status surrogate_set_normalization(sg_model *m, const float *host_src)
{
    PR_CHECK_ARG(m && host_src, "surrogate_set_normalization: null argument");
    for (int k = 0; k < NIN; ++k)
        PR_CHECK_ARG(host_src[NIN + k] > 0, "surrogate_set_normalization: input std must be > 0");
    for (int j = 0; j < m->dev.nout; ++j)
        PR_CHECK_ARG(host_src[out_std_idx(j)] > 0, "surrogate_set_normalization: output std must be > 0");
    PR_CUDA_TRY(cudaDeviceSynchronize());
    PR_CUDA_TRY(cudaMemcpy(m->dev.norm, host_src, SG_NORM_FLOATS * 4, cudaMemcpyHostToDevice));
    outstat_kernel<<<1, 32>>>(m->dev.norm, m->dev.outstat);
    PR_CUDA_TRY(cudaGetLastError());
    return PR_OK;
}

pr_status surrogate_fit_normalization(sg_model *m, int64_t n, const float *x, int64_t ldx, const float *y,
                                      int64_t ldy, void *stream)
{
    PR_CHECK_ARG(m && x && y && n > 0 && ldx >= n && ldy >= n, "surrogate_fit_normalization: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    norm_partial_kernel<<<m->norm_blocks, 256, 0, st>>>(n, x, ldx, y, ldy, m->dev, m->d_normpart);
    norm_final_kernel<<<1, 32, 0, st>>>(m->norm_blocks, m->d_normpart, m->dev.norm);
    outstat_kernel<<<1, 32, 0, st>>>(m->dev.norm, m->dev.outstat);
    PR_CUDA_TRY(cudaGetLastError());
    return PR_OK;
}

// forward + backward of one batch already prepared in the training buffers
static pr_status fwd_bwd(sg_model *m, int64_t B, cudaStream_t st)
{
    SgDev &d = m->dev;
    const int W = m->width, L = m->hidden;
    const int mt = ceil_div(B, 128);
    cudaError_t e = cudaSuccess;
    // forward, hidden layers
    for (int l = 0; l < L; ++l) {
        GemmArgs a = base_args(m);
        a.M = (int)B; a.N = W; a.K = (l == 0) ? KIN : W; a.kb_per_split = a.K / 64;
        a.bias = d.master + d.lay[l].b_off;
        a.out = d.h[l]; a.ldo = W; a.gd = d.g[l]; a.ldg = W;
        a.tma_out = 1; a.tm_out = m->ts_h[l]; a.tm_gd = m->ts_g[l];
        const CUtensorMap &ta = (l == 0) ? m->tm_x0 : m->tm_h[l - 1];
        e = launch_gemm_n<kEpiHidden>(ta, m->tm_w[l], a, mt, W, 1, st);
        if (e != cudaSuccess) break;
    }
    if (e != cudaSuccess) { prgb::set_error("forward: %s", cudaGetErrorString(e)); return PR_ECUDA; }
    // output layer + loss + dz of the output
    {
        GemmArgs a = base_args(m);
        a.M = (int)B; a.N = NOP; a.K = W; a.kb_per_split = W / 64;
        a.bias = d.master + d.lay[L].b_off;
        a.target = d.tgt; a.ldt = d.max_batch;
        a.l1 = m->loss_l1;
        a.loss_scale = (m->loss_l1 ? 1.0f : 2.0f) / (float)(B * d.nout);
        a.nout = d.nout;
        a.out = d.dzo; a.ldo = KIN;
        a.colsum = d.colsum[L]; a.loss_part = d.loss_part;
        e = launch_gemm<16, kEpiOutLoss>(m->tm_h[L - 1], m->tm_w[L], a, mt, 1, 1, st);
        if (e != cudaSuccess) { prgb::set_error("loss: %s", cudaGetErrorString(e)); return PR_ECUDA; }
    }
    // input gradients: dz_{l-1} = (dz_l W_l) * GeLU'(z_{l-1})
    for (int l = L; l >= 1; --l) {
        GemmArgs a = base_args(m);
        a.M = (int)B; a.N = W; a.K = (l == L) ? KIN : W; a.kb_per_split = a.K / 64;
        a.gd = d.g[l - 1]; a.ldg = W;
        a.out = d.dz[l - 1]; a.ldo = W;
        a.tma_out = 1; a.tm_out = m->ts_dz[l - 1];
        a.colsum = d.colsum[l - 1];
        const CUtensorMap &ta = (l == L) ? m->tm_dzo : m->tm_dz[l];
        e = launch_gemm_n<kEpiDx>(ta, m->tm_wt[l], a, mt, W, 1, st);
        if (e != cudaSuccess) { prgb::set_error("dx: %s", cudaGetErrorString(e)); return PR_ECUDA; }
    }
    // weight gradients: dW_l = dz_l^T h_{l-1}, K = batch, split along K; both
    // operands read MN-major from the batch-major dz and h
    for (int l = 0; l <= L; ++l) {
        GemmArgs a = base_args(m);
        const int mp = d.dw_mpad[l], np = d.lay[l].in_pad;
        a.M = mp; a.Mpad = mp; a.N = np; a.K = (int)B; a.kb_per_split = d.dw_kps[l];
        a.partial = d.partial[l];
        const int splits = ceil_div(ceil_div(B, 64), d.dw_kps[l]);
        const CUtensorMap &ta = (l == L) ? m->tmn_dzo : m->tmn_dz[l];
        const CUtensorMap &tb = (l == 0) ? m->tmn_x0 : m->tmn_h[l - 1];
        e = launch_gemm_dw_mn(ta, tb, a, mp / 128, np, splits, st);
        if (e != cudaSuccess) { prgb::set_error("dw: %s", cudaGetErrorString(e)); return PR_ECUDA; }
        m->last_splits[l] = splits;
    }
    return PR_OK;
}

static pr_status train_common(sg_model *m, int64_t batch, int64_t n_pool, const float *x, int64_t ldx, const float *y,
                              int64_t ldy, uint64_t seed, float lr, float *loss_out, float *grad_out, void *stream)
{
    PR_CHECK_ARG(m && x && y, "surrogate_train_step: null argument");
    PR_CHECK_ARG(batch >= 128 && batch % 128 == 0 && batch <= m->max_batch,
                 "surrogate_train_step: batch must be a multiple of 128 and <= max_batch (%lld)", (long long)m->max_batch);
    PR_CHECK_ARG(n_pool >= batch && ldx >= n_pool && ldy >= n_pool, "surrogate_train_step: pool sizes");
    PR_CHECK_ARG(std::isfinite(lr) && lr >= 0.f, "surrogate_train_step: bad lr");
    cudaStream_t st = (cudaStream_t)stream;
    SgDev &d = m->dev;
    const int blocks = ceil_div(batch, 256);
    prep_train_kernel<<<blocks < 2048 ? blocks : 2048, 256, 0, st>>>(d, batch, n_pool, x, ldx, y, ldy, seed);
    PR_CUDA_TRY(cudaGetLastError());
    // the dw GEMMs split K over dw_kps k-blocks: make sure the splits fit the batch
    for (int l = 0; l <= m->hidden; ++l) d.dw_splits[l] = ceil_div(ceil_div(batch, 64), d.dw_kps[l]);
    pr_status s = fwd_bwd(m, batch, st);
    if (s) return s;
    const int64_t nct = batch / 128;
    if (grad_out) {
        bias_grad_kernel<<<(int)(((int64_t)(m->hidden + 1) * m->width * 32 + 255) / 256), 256, 0, st>>>(d, nct);
        adam_kernel<<<adam_blocks(d), 256, 0, st>>>(d, 0.f, 0.9f, 0.999f, 1e-8f, 1, 1, grad_out);
    } else {
        m->step += 1;
        bias_grad_kernel<<<(int)(((int64_t)(m->hidden + 1) * m->width * 32 + 255) / 256), 256, 0, st>>>(d, nct);
        adam_kernel<<<adam_blocks(d), 256, 0, st>>>(d, lr, 0.9f, 0.999f, 1e-8f, (int)m->step, 0, nullptr);
        launch_transpose_w(d, st);
    }
    float *lo = loss_out ? loss_out : m->d_loss;
    loss_final_kernel<<<1, 256, 0, st>>>(d.loss_part, nct, 1.0f / (float)(batch * d.nout), lo);
    PR_CUDA_TRY(cudaGetLastError());
    return PR_OK;
}

pr_status surrogate_train_step(sg_model *m, int64_t batch, int64_t n_pool, const float *x, int64_t ldx,
                               const float *y, int64_t ldy, uint64_t sample_seed, float lr, float *loss_out,
                               void *stream)
{
    return train_common(m, batch, n_pool, x, ldx, y, ldy, sample_seed, lr, loss_out, nullptr, stream);
}

pr_status surrogate_loss_grad(sg_model *m, int64_t batch, const float *x, int64_t ldx, const float *y, int64_t ldy,
                              float *loss_out, float *grad_out, void *stream)
{
    PR_CHECK_ARG(grad_out != nullptr, "surrogate_loss_grad: grad_out is NULL");
    return train_common(m, batch, batch, x, ldx, y, ldy, 0, 0.f, loss_out, grad_out, stream);
}

// The next (start, stop) event pair of SG_OPT_TIME_MLP, created on first use.
static cudaError_t mlp_timer_pair(sg_model *m, cudaEvent_t &t0, cudaEvent_t &t1)
{
    while ((int)m->tev.size() < 2 * (m->tev_used + 1)) {
        cudaEvent_t e;
        const cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        m->tev.push_back(e);
    }
    t0 = m->tev[2 * m->tev_used];
    t1 = m->tev[2 * m->tev_used + 1];
    ++m->tev_used;
    return cudaSuccess;
}

pr_status surrogate_infer(sg_model *m, int64_t n, const float *T, const float *p, const float *Y, int64_t ldY,
                          float *out, int64_t ldo, uint8_t *used_fallback, void *stream)
{
    PR_CHECK_ARG(m != nullptr, "surrogate_infer: null model");
    PR_CHECK_ARG(n >= 0, "surrogate_infer: n < 0");
    if (n == 0) return PR_OK;
    PR_CHECK_ARG(T && p && Y && out, "surrogate_infer: null array");
    PR_CHECK_ARG(ldY >= n && ldo >= n, "surrogate_infer: ldY/ldo < n");
    PR_CHECK_ARG(prgb::aligned(T, 4) && prgb::aligned(p, 4) && prgb::aligned(Y, 4) && prgb::aligned(out, 4),
                 "surrogate_infer: misaligned array");
    cudaStream_t st = (cudaStream_t)stream;
    SgDev &d = m->dev;
    pr_ctx *ctx = m->ctx;
    const int W = m->width, L = m->hidden;
    for (int64_t r0 = 0; r0 < n; r0 += m->chunk) {
        const int64_t mc = (n - r0 < m->chunk) ? (n - r0) : m->chunk;
        const int mt = ceil_div(mc, 128);
        PR_CUDA_TRY(cudaMemsetAsync(m->d_count, 0, 4, st));
        const int pb = ceil_div(mc, 256);
        prep_infer_kernel<<<pb < 4096 ? pb : 4096, 256, 0, st>>>(d, r0, mc, T, p, Y, ldY, used_fallback,
                                                                 m->d_flags, m->d_list, m->d_count);
        PR_CUDA_TRY(cudaGetLastError());
        cudaEvent_t tm0 = nullptr, tm1 = nullptr;
        if (m->time_mlp) {
            PR_CUDA_TRY(mlp_timer_pair(m, tm0, tm1));
            PR_CUDA_TRY(cudaEventRecord(tm0, st));
        }
        if ((m->fused_on == 3 && m->res_pairs > 0) || (m->fused_on == 4 && m->pp_pairs > 0)) {
            // every layer in one launch, activations resident in shared memory
            // (mlp_resident.cuh), or alternating between tensor and shared
            // memory (mlp_pingpong.cuh)
            const bool pp = m->fused_on == 4;
            ResidentArgs ra;
            memset(&ra, 0, sizeof(ra));
            ra.tm_x = m->tm_xi;
            for (int l = 0; l <= L; ++l) {
                ra.tm_w[l] = pp ? m->tmq_w[l] : m->tmr_w[l];
                ra.bias[l] = d.master + d.lay[l].b_off;
            }
            ra.M = (int)mc; ra.L = L; ra.W = W;
            ra.out6 = out + r0; ra.ld6 = ldo;
            ra.out_mean = d.outstat; ra.out_std = d.outstat + NOUT_MAX;
            ra.add_h = (d.mode != SG_MODE_FORWARD) ? nullptr : d.hig;
            ra.log_mask = log_mask_of(d.mode, d.outputs);
            ra.nout = d.nout;
            ra.err = m->d_err;
            ra.wait_cycles = m->wait_cycles > 0 ? m->wait_cycles : 4000000000LL;
            ra.stall_test = m->stall_test;
            if (pp) PR_CUDA_TRY(launch_pingpong(ra, m->pp_pairs, st));
            else PR_CUDA_TRY(launch_resident(ra, m->res_pairs, st));
        } else if (m->fused_on) {
            // every layer in one cooperative launch (mlp_fused.cuh): single
            // CTAs, or CTA pairs when asked for and the device takes them
            bool pair = m->fused_on == 2 && m->fused_pair_ok;
            FusedArgs fa;
            memset(&fa, 0, sizeof(fa));
            fa.tm_x = m->tm_xi;
            fa.tm_ring_ld = m->tmf_ring_ld;
            fa.tm_ring_st = m->tmf_ring_st;
            for (int l = 0; l <= L; ++l) fa.bias[l] = d.master + d.lay[l].b_off;
            fa.M = (int)mc; fa.L = L; fa.W = W;
            fa.n_t = W / kFusedBN; fa.ips = L * fa.n_t + 1;
            fa.out6 = out + r0; fa.ld6 = ldo;
            fa.out_mean = d.outstat; fa.out_std = d.outstat + NOUT_MAX;
            fa.add_h = (d.mode != SG_MODE_FORWARD) ? nullptr : d.hig;
            fa.log_mask = log_mask_of(d.mode, d.outputs);
            fa.nout = d.nout;
            fa.done = m->d_done; fa.err = m->d_err;
            fa.wait_cycles = m->wait_cycles > 0 ? m->wait_cycles : 4000000000LL;
            fa.stall_test = m->stall_test;
            PR_CUDA_TRY(cudaMemsetAsync(m->d_done, 0, (size_t)mt * (L + 1) * 4, st));
            cudaError_t e = cudaSuccess;
            if (pair) {
                for (int l = 0; l <= L; ++l) fa.tm_w[l] = m->tmp_w[l];
                fa.R = ceil_div(mt, 2); fa.D = m->fused_D2; fa.ring = m->fused_ring2;
                fa.total = (long long)(fa.R + (long long)L * fa.D) * fa.ips;
                e = launch_fused<true>(fa, m->fused_clusters, st);
                if (e != cudaSuccess) {   // a configuration the device refuses: single CTAs from now on
                    cudaGetLastError();
                    m->fused_pair_ok = 0;
                    pair = false;
                }
            }
            if (!pair) {
                for (int l = 0; l <= L; ++l) fa.tm_w[l] = m->tmf_w[l];
                fa.R = mt; fa.D = m->fused_D; fa.ring = m->fused_ring;
                fa.total = (long long)(fa.R + (long long)L * fa.D) * fa.ips;
                e = launch_fused<false>(fa, num_sms_current(), st);
            }
            PR_CUDA_TRY(e);
        }
        for (int l = 0; l < L && !m->fused_on; ++l) {
            GemmArgs a = base_args(m);
            a.M = (int)mc; a.N = W; a.K = (l == 0) ? KIN : W; a.kb_per_split = a.K / 64;
            a.bias = d.master + d.lay[l].b_off;
            a.out = d.hi[l & 1]; a.ldo = W;
            a.tma_out = 1; a.tm_out = m->ts_hi[l & 1];
            const CUtensorMap &ta = (l == 0) ? m->tm_xi : m->tm_hi[(l - 1) & 1];
            PR_CUDA_TRY((launch_gemm_n<kEpiHidden>(ta, m->tm_w[l], a, mt, W, 1, st)));
        }
        if (!m->fused_on) {
            GemmArgs a = base_args(m);
            a.M = (int)mc; a.N = NOP; a.K = W; a.kb_per_split = W / 64;
            a.bias = d.master + d.lay[L].b_off;
            a.out6 = out + r0; a.ld6 = ldo;
            a.out_mean = d.outstat; a.out_std = d.outstat + NOUT_MAX;
            a.add_h = (d.mode != SG_MODE_FORWARD) ? nullptr : d.hig;
            a.log_mask = log_mask_of(d.mode, d.outputs);
            a.nout = d.nout;
            PR_CUDA_TRY((launch_gemm<16, kEpiOutPhys>(m->tm_hi[(L - 1) & 1], m->tm_w[L], a, mt, 1, 1, st)));
        }
        if (m->time_mlp) PR_CUDA_TRY(cudaEventRecord(tm1, st));
        const float ctol = (d.mode == SG_MODE_FORWARD) ? m->conf_tol : 0.f;
        const float ttol = (d.outputs == SG_OUT_PROPS) ? m->tr_tol : 0.f;
        if (ctol > 0.f || ttol > 0.f) {
            confidence_kernel<<<pb < 4096 ? pb : 4096, 256, 0, st>>>(d, r0, mc, T, p, Y, ldY, out, ldo, ctol, ttol,
                                                                     used_fallback, m->d_flags, m->d_list, m->d_count);
            PR_CUDA_TRY(cudaGetLastError());
        }
        // FP64 Peng-Robinson for the cells outside the training hull (and the low-confidence ones)
        const int fb = ctx->num_sms * 4;
        const SpeciesRec<double> *sp64 = (const SpeciesRec<double> *)ctx->d_sp64;
        const int sel = (d.outputs >= SG_OUT_SINGLE) ? d.outputs - SG_OUT_SINGLE : -1;
        if (d.outputs == SG_OUT_DK || d.outputs == SG_OUT_HK) {
            if (ctx->has_kij)
                fallback_species_kernel<9, true><<<fb, 128, 0, st>>>(m->d_list, m->d_count, r0, T, p, Y, ldY, out,
                                                                     ldo, sp64, ctx->d_kij64, ctx->d_dtab64,
                                                                     ctx->d_corr64, ctx->corr_nT, ctx->corr_nP,
                                                                     ctx->n_species, d.outputs);
            else
                fallback_species_kernel<9, false><<<fb, 128, 0, st>>>(m->d_list, m->d_count, r0, T, p, Y, ldY, out,
                                                                      ldo, sp64, ctx->d_kij64, ctx->d_dtab64,
                                                                      ctx->d_corr64, ctx->corr_nT, ctx->corr_nP,
                                                                      ctx->n_species, d.outputs);
        } else if (d.mode != SG_MODE_FORWARD) {
            if (ctx->has_kij)
                fallback_inverse_kernel<9, true><<<fb, 128, 0, st>>>(m->d_list, m->d_count, r0, T, p, Y, ldY, out,
                                                                     ldo, sp64, ctx->d_pair64, ctx->d_kij64,
                                                                     ctx->n_species, ctx->flags, sel);
            else
                fallback_inverse_kernel<9, false><<<fb, 128, 0, st>>>(m->d_list, m->d_count, r0, T, p, Y, ldY, out,
                                                                      ldo, sp64, ctx->d_pair64, ctx->d_kij64,
                                                                      ctx->n_species, ctx->flags, sel);
        } else if (ctx->has_kij)
            fallback_kernel<9, true><<<fb, 128, 0, st>>>(m->d_list, m->d_count, r0, T, p, Y, ldY, out, ldo,
                                                         (const SpeciesRec<double> *)ctx->d_sp64, ctx->d_pair64,
                                                         ctx->d_kij64, ctx->n_species, ctx->flags, ctx->tmid_u);
        else
            fallback_kernel<9, false><<<fb, 128, 0, st>>>(m->d_list, m->d_count, r0, T, p, Y, ldY, out, ldo,
                                                          (const SpeciesRec<double> *)ctx->d_sp64, ctx->d_pair64,
                                                          ctx->d_kij64, ctx->n_species, ctx->flags, ctx->tmid_u);
        PR_CUDA_TRY(cudaGetLastError());
    }
    return PR_OK;
}

}  // extern "C"

int sg_mode_of(const sg_model *m) { return m->dev.mode; }

extern "C" {

pr_status surrogate_get_option(const sg_model *m, int option, int *value)
{
    PR_CHECK_ARG(m != nullptr && value != nullptr, "surrogate_get_option: null argument");
    switch (option) {
    case SG_OPT_FUSED_INFER:
        *value = !m->fused_on                            ? 0
                 : (m->fused_on == 4 && m->pp_pairs > 0)  ? 4
                 : (m->fused_on == 3 && m->res_pairs > 0) ? 3
                 : (m->fused_on == 2 && m->fused_pair_ok) ? 2
                                                          : 1;
        return PR_OK;
    case SG_OPT_MODE: *value = m->dev.mode; return PR_OK;
    case SG_OPT_WAIT_LIMIT_KCYCLES: *value = (int)(m->wait_cycles / 1000); return PR_OK;
    case SG_OPT_TEST_STALL: *value = m->stall_test; return PR_OK;
    case SG_OPT_LOSS: *value = m->loss_l1 ? SG_LOSS_L1 : SG_LOSS_REL_MSE; return PR_OK;
    case SG_OPT_CONFIDENCE_PPM: *value = (int)(m->conf_tol * 1e6f + 0.5f); return PR_OK;
    case SG_OPT_TRANSPORT_CONFIDENCE_PPM: *value = (int)(m->tr_tol * 1e6f + 0.5f); return PR_OK;
    case SG_OPT_OUTPUTS: *value = m->dev.outputs; return PR_OK;
    case SG_OPT_TIME_MLP: *value = m->time_mlp; return PR_OK;
    default: break;
    }
    PR_CHECK_ARG(false, "surrogate_get_option: unknown option %d", option);
    return PR_EINVAL;
}

pr_status surrogate_set_option(sg_model *m, int option, int value)
{
    PR_CHECK_ARG(m != nullptr, "surrogate_set_option: null model");
    switch (option) {
    case SG_OPT_FUSED_INFER:
        PR_CHECK_ARG(value == 0 || ((value == 1 || value == 2) && m->fused_ok) || (value == 3 && m->res_pairs > 0) ||
                         (value == 4 && m->pp_pairs > 0),
                     "surrogate_set_option: fused inference needs a width that is a multiple of 256, <= 1024, "
                     "and its biases within shared memory; resident activations need a width of 256 or 512 "
                     "and cluster launches");
        m->fused_on = value;
        return PR_OK;
    case SG_OPT_WAIT_LIMIT_KCYCLES:
        PR_CHECK_ARG(value >= 0, "surrogate_set_option: wait limit must be >= 0");
        m->wait_cycles = 1000LL * value;
        return PR_OK;
    case SG_OPT_TEST_STALL:
        m->stall_test = value != 0;
        return PR_OK;
    case SG_OPT_OUTPUTS: {
        PR_CHECK_ARG(value >= SG_OUT_PROPS && value <= SG_OUT_SINGLE + 5, "surrogate_set_option: bad outputs %d", value);
        PR_CHECK_ARG(value == SG_OUT_PROPS || m->dev.mode != SG_MODE_FORWARD,
                     "surrogate_set_option: per-species and single-property outputs need the inverse or Bilger "
                     "inputs (h, p, Y)");
        SgDev &d = m->dev;
        d.outputs = value;
        d.nout = (value == SG_OUT_PROPS) ? NOUT6 : (value >= SG_OUT_SINGLE) ? 1 : m->ctx->n_species;
        // the last layer's output count changes the exported parameter count;
        // start the weights afresh
        LayerLayout &LL = d.lay[d.hidden];
        d.n_flat = LL.flat_off + (int64_t)d.nout * LL.in + d.nout;
        LL.out = d.nout;
        PR_CUDA_TRY(cudaDeviceSynchronize());
        init_params_kernel<<<256, 256>>>(d, m->seed ? m->seed : 1);
        refresh_bf16_kernel<<<256, 256>>>(d);
        launch_transpose_w(d, 0);
        PR_CUDA_TRY(cudaDeviceSynchronize());
        m->step = 0;
        return PR_OK;
    }
    case SG_OPT_CONFIDENCE_PPM:
        PR_CHECK_ARG(value >= 0, "surrogate_set_option: confidence tolerance must be >= 0");
        m->conf_tol = 1e-6f * (float)value;
        return PR_OK;
    case SG_OPT_TRANSPORT_CONFIDENCE_PPM:
        PR_CHECK_ARG(value >= 0, "surrogate_set_option: transport confidence tolerance must be >= 0");
        m->tr_tol = 1e-6f * (float)value;
        return PR_OK;
    case SG_OPT_TIME_MLP:
        PR_CHECK_ARG(value == 0 || value == 1, "surrogate_set_option: SG_OPT_TIME_MLP takes 0 or 1");
        m->time_mlp = value;
        m->tev_used = 0;
        return PR_OK;
    case SG_OPT_LOSS:
        PR_CHECK_ARG(value == SG_LOSS_REL_MSE || value == SG_LOSS_L1, "surrogate_set_option: bad loss %d", value);
        m->loss_l1 = value == SG_LOSS_L1;
        return PR_OK;
    case SG_OPT_MODE:
        PR_CHECK_ARG(value == SG_MODE_FORWARD || value == SG_MODE_INVERSE || value == SG_MODE_BILGER,
                     "surrogate_set_option: bad mode %d", value);
        PR_CHECK_ARG(value != SG_MODE_BILGER || m->ctx->has_bilger,
                     "surrogate_set_option: SG_MODE_BILGER needs the context's element table (pr_set_bilger)");
        PR_CHECK_ARG(value != SG_MODE_FORWARD || m->dev.outputs == SG_OUT_PROPS,
                     "surrogate_set_option: the forward model has no per-species or single-property outputs");
        m->dev.mode = value;
        m->dev.bilger = m->ctx->d_bilger32;
        return PR_OK;
    default:
        PR_CHECK_ARG(false, "surrogate_set_option: unknown option %d", option);
    }
    return PR_EINVAL;
}

pr_status surrogate_set_boxcox(sg_model *m, double lambda, double shift)
{
    PR_CHECK_ARG(m != nullptr, "surrogate_set_boxcox: null model");
    PR_CHECK_ARG(std::isfinite(lambda) && std::fabs(lambda) <= 10.0, "surrogate_set_boxcox: lambda outside [-10, 10]");
    PR_CHECK_ARG(std::isfinite(shift) && shift > 0.0 && shift <= 1.0, "surrogate_set_boxcox: shift outside (0, 1]");
    m->dev.bc_lambda = (float)lambda;
    m->dev.bc_shift = (float)shift;
    return PR_OK;
}

pr_status surrogate_sync_status(sg_model *m)
{
    PR_CHECK_ARG(m != nullptr, "surrogate_sync_status: null model");
    PR_CUDA_TRY(cudaDeviceSynchronize());
    int err = 0;
    PR_CUDA_TRY(cudaMemcpy(&err, m->d_err, 4, cudaMemcpyDeviceToHost));
    if (err) {
        PR_CUDA_TRY(cudaMemset(m->d_err, 0, 4));
        prgb::set_error("surrogate: a tensor-core kernel gave up waiting on a barrier (results invalid)");
        return PR_ETIMEOUT;
    }
    return PR_OK;
}

// Checkpoint: "PRSG" v1 | width hidden step | n_master | master, adam_m, adam_v (FP32) | normalisation.
pr_status surrogate_save(const sg_model *m, const char *path)
{
    PR_CHECK_ARG(m && path, "surrogate_save: null argument");
    const int64_t n = m->dev.n_master;
    std::vector<float> buf(3 * n + SG_NORM_FLOATS);
    PR_CUDA_TRY(cudaDeviceSynchronize());
    PR_CUDA_TRY(cudaMemcpy(buf.data(), m->dev.master, n * 4, cudaMemcpyDeviceToHost));
    PR_CUDA_TRY(cudaMemcpy(buf.data() + n, m->dev.adam_m, n * 4, cudaMemcpyDeviceToHost));
    PR_CUDA_TRY(cudaMemcpy(buf.data() + 2 * n, m->dev.adam_v, n * 4, cudaMemcpyDeviceToHost));
    PR_CUDA_TRY(cudaMemcpy(buf.data() + 3 * n, m->dev.norm, SG_NORM_FLOATS * 4, cudaMemcpyDeviceToHost));
    FILE *f = fopen(path, "wb");
    if (!f) { prgb::set_error("surrogate_save: cannot open %s", path); return PR_EINVAL; }
    const char magic[4] = {'P', 'R', 'S', 'G'};
    // format 5: 13 inputs (with T_pc / T and log W); the enthalpy output is the
    // departure from the ideal-gas enthalpy; the mode word carries the output
    // set in its second byte; the Box-Cox parameters of Bilger's Z follow the
    // counts; the normalisation has SG_NORM_FLOATS entries (64 before format 5)
    const int32_t hdr[4] = {5, m->width, m->hidden, m->dev.mode | (m->dev.outputs << 8)};
    const int64_t step = m->step;
    const float bc[2] = {m->dev.bc_lambda, m->dev.bc_shift};
    bool ok = fwrite(magic, 1, 4, f) == 4 && fwrite(hdr, 4, 4, f) == 4 && fwrite(&step, 8, 1, f) == 1 &&
              fwrite(&n, 8, 1, f) == 1 && fwrite(bc, 4, 2, f) == 2 && fwrite(buf.data(), 4, buf.size(), f) == buf.size();
    ok = (fclose(f) == 0) && ok;
    if (!ok) { prgb::set_error("surrogate_save: write failed"); return PR_EINVAL; }
    return PR_OK;
}

pr_status surrogate_load(sg_model *m, const char *path)
{
    PR_CHECK_ARG(m && path, "surrogate_load: null argument");
    FILE *f = fopen(path, "rb");
    if (!f) { prgb::set_error("surrogate_load: cannot open %s", path); return PR_EINVAL; }
    char magic[4];
    int32_t hdr[4];
    int64_t step = 0, n = 0;
    bool ok = fread(magic, 1, 4, f) == 4 && memcmp(magic, "PRSG", 4) == 0 && fread(hdr, 4, 4, f) == 4 &&
              fread(&step, 8, 1, f) == 1 && fread(&n, 8, 1, f) == 1;
    const int32_t mode_word = m->dev.mode | (m->dev.outputs << 8);
    ok = ok && hdr[0] >= 3 && hdr[0] <= 5 && hdr[1] == m->width && hdr[2] == m->hidden && hdr[3] == mode_word &&
         n == m->dev.n_master;
    float bc[2] = {m->dev.bc_lambda, m->dev.bc_shift};   // format 3 carries none
    if (ok && hdr[0] >= 4) ok = fread(bc, 4, 2, f) == 2;
    const int norm_floats = (hdr[0] >= 5) ? SG_NORM_FLOATS : 64;
    std::vector<float> buf;
    if (ok) {
        buf.resize(3 * n + SG_NORM_FLOATS);
        ok = fread(buf.data(), 4, 3 * n + norm_floats, f) == (size_t)(3 * n + norm_floats);
        // older formats: the statistics of outputs 6..15 as the identity
        for (int j = NOUT6; j < NOUT_MAX && norm_floats < SG_NORM_FLOATS; ++j) {
            buf[3 * n + out_mean_idx(j)] = 0.f;
            buf[3 * n + out_std_idx(j)] = 1.f;
        }
    }
    fclose(f);
    if (!ok) { prgb::set_error("surrogate_load: %s is not a checkpoint of this model", path); return PR_EINVAL; }
    PR_CUDA_TRY(cudaDeviceSynchronize());
    PR_CUDA_TRY(cudaMemcpy(m->dev.master, buf.data(), n * 4, cudaMemcpyHostToDevice));
    PR_CUDA_TRY(cudaMemcpy(m->dev.adam_m, buf.data() + n, n * 4, cudaMemcpyHostToDevice));
    PR_CUDA_TRY(cudaMemcpy(m->dev.adam_v, buf.data() + 2 * n, n * 4, cudaMemcpyHostToDevice));
    PR_CUDA_TRY(cudaMemcpy(m->dev.norm, buf.data() + 3 * n, SG_NORM_FLOATS * 4, cudaMemcpyHostToDevice));
    m->dev.bc_lambda = bc[0];
    m->dev.bc_shift = bc[1];
    outstat_kernel<<<1, 32>>>(m->dev.norm, m->dev.outstat);
    refresh_bf16_kernel<<<256, 256>>>(m->dev);
    launch_transpose_w(m->dev, 0);
    PR_CUDA_TRY(cudaDeviceSynchronize());
    m->step = step;
    return PR_OK;
}

pr_status surrogate_mlp_time(sg_model *m, double *ms, int64_t *launches)
{
    PR_CHECK_ARG(m && ms && launches, "surrogate_mlp_time: null argument");
    double t = 0.0;
    if (m->tev_used > 0) PR_CUDA_TRY(cudaEventSynchronize(m->tev[2 * m->tev_used - 1]));
    for (int k = 0; k < m->tev_used; ++k) {
        float e = 0.f;
        PR_CUDA_TRY(cudaEventElapsedTime(&e, m->tev[2 * k], m->tev[2 * k + 1]));
        t += e;
    }
    *ms = t;
    *launches = m->tev_used;
    m->tev_used = 0;
    return PR_OK;
}

pr_status mlp_gemm_bf16(int64_t M, int64_t N, int64_t K, const void *A, int64_t lda, const void *B, int64_t ldb,
                        float *D, int64_t ldd, int *err_flag, void *stream)
{
    PR_CHECK_ARG(A && B && D && err_flag, "mlp_gemm_bf16: null argument");
    PR_CHECK_ARG(M >= 1 && M <= (1 << 30) && K >= 64 && K % 64 == 0 && K <= (1 << 30),
                 "mlp_gemm_bf16: need M >= 1 and K a positive multiple of 64");
    PR_CHECK_ARG(N == 16 || N == 64 || (N % 128 == 0 && N <= 65536), "mlp_gemm_bf16: N must be 16, 64 or a multiple of 128");
    PR_CHECK_ARG(lda >= K && ldb >= K && ldd >= N && lda % 8 == 0 && ldb % 8 == 0 && ldd % 4 == 0,
                 "mlp_gemm_bf16: leading dimensions (lda, ldb multiples of 8; ldd of 4)");
    PR_CHECK_ARG(prgb::aligned(A, 16) && prgb::aligned(B, 16) && prgb::aligned(D, 16), "mlp_gemm_bf16: 16-byte alignment");
    const int bn = pick_bn((int)N);
    CUtensorMap ta, tb;
    if (!make_map(&ta, A, K, M, lda, 128) || !make_map(&tb, B, K, N, ldb, bn)) {
        prgb::set_error("mlp_gemm_bf16: tensor map encoding failed");
        return PR_ECUDA;
    }
    GemmArgs a;
    memset(&a, 0, sizeof(a));
    a.M = (int)M; a.Mpad = (int)M; a.N = (int)ldd; a.K = (int)K; a.kb_per_split = (int)(K / 64);
    a.partial = D;
    a.err = err_flag;
    cudaStream_t st = (cudaStream_t)stream;
    const int gx = ceil_div(M, 128), gy = (int)(N / bn);
    cudaError_t e;
    e = launch_gemm_n<kEpiDw>(ta, tb, a, gx, (int)N, 1, st);
    (void)gy;
    PR_CUDA_TRY(e);
    return PR_OK;
}

}  // extern "C"
