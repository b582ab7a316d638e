// Internal state of the surrogate MLP (device buffers, parameter layout,
// tensor maps).  Shared by surrogate.cu and the serving loop.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "pr_internal.h"

#define SG_MAX_HIDDEN 8
// SG_NORM_FLOATS comes from prgb300.h

// Parameter layout of one layer inside the padded FP32 master array.
struct LayerLayout {
    int64_t w_off, b_off;   // offsets of W [out_pad][in_pad] and b [out_pad]
    int in, in_pad, out, out_pad;
    int64_t flat_off;       // offset in the unpadded (W [out][in], b [out]) export order
};

// Everything the kernels need, passed by value.
struct SgDev {
    int width, hidden;
    int64_t max_batch;
    LayerLayout lay[SG_MAX_HIDDEN + 1];
    int64_t n_master, n_flat;
    float *master, *adam_m, *adam_v;
    __nv_bfloat16 *wb[SG_MAX_HIDDEN + 1];   // W [out_pad][in_pad]
    __nv_bfloat16 *wt[SG_MAX_HIDDEN + 1];   // W^T [in][K of the input-gradient GEMM]
    float *norm;                            // SG_NORM_FLOATS
    float *outstat;                         // output mean[16] then std[16], gathered from norm
    int nout;                               // outputs of the model: 6, or 9 per-species ones
    int outputs;                            // SG_OUT_PROPS, SG_OUT_DK, SG_OUT_HK or SG_OUT_SINGLE + j
    // training activations, batch-major [B][.] (the weight-gradient GEMMs read
    // them MN-major, so no transposed copies)
    __nv_bfloat16 *x0;
    float *tgt;                             // standardised targets [6][B]
    __nv_bfloat16 *h[SG_MAX_HIDDEN], *g[SG_MAX_HIDDEN];
    __nv_bfloat16 *dz[SG_MAX_HIDDEN];
    __nv_bfloat16 *dzo;                     // output-layer dz [B][64]
    float *partial[SG_MAX_HIDDEN + 1];      // weight-gradient partials [split][Mpad][in_pad]
    int dw_splits[SG_MAX_HIDDEN + 1], dw_kps[SG_MAX_HIDDEN + 1], dw_mpad[SG_MAX_HIDDEN + 1];
    float *colsum[SG_MAX_HIDDEN + 1];       // per-CTA column sums of dz [B/128][out_pad]
    float *bgrad;                           // bias gradients [hidden + 1][width] (reduced colsum)
    float *loss_part;                       // [B/128]
    // inference chunk buffers
    __nv_bfloat16 *xi, *hi[2];
    float *hig;                             // ideal-gas enthalpy of the chunk's cells [chunk]
    int mode;                               // SG_MODE_FORWARD, SG_MODE_INVERSE or SG_MODE_BILGER
    const void *sp32;                       // the context's FP32 species records (NASA-7 data)
    const float *pair32;                    // the context's FP32 Chung pair table [9][9]
    int pr_flags;                           // the context's PR_FLAG_* (transport rule)
    const float *bilger;                    // SG_MODE_BILGER: the context's b_k [9], beta_ox, 1/range
    float bc_lambda, bc_shift;              // SG_MODE_BILGER: Box-Cox of Z, ((Z + shift)^lambda - 1) / lambda
};

struct ParamRef {
    bool valid, bias;
    int layer, o, i;
    int in_pad, out_pad_n, out_pad_k;
    int64_t flat;
};

__device__ __forceinline__ ParamRef decode_param(const SgDev &d, int64_t e)
{
    ParamRef r;
    int l = 0;
    while (l < d.hidden && e >= d.lay[l + 1].w_off) ++l;
    const LayerLayout &L = d.lay[l];
    r.layer = l;
    r.in_pad = L.in_pad;
    r.out_pad_n = L.out_pad;
    r.out_pad_k = (l == d.hidden) ? 64 : d.width;
    if (e < L.b_off) {
        const int64_t k = e - L.w_off;
        r.bias = false;
        r.o = (int)(k / L.in_pad);
        r.i = (int)(k % L.in_pad);
        r.valid = r.o < L.out && r.i < L.in;
        r.flat = L.flat_off + (int64_t)r.o * L.in + r.i;
    } else {
        r.bias = true;
        r.o = (int)(e - L.b_off);
        r.i = 0;
        r.valid = r.o < L.out;
        r.flat = L.flat_off + (int64_t)L.out * L.in + r.o;
    }
    return r;
}

struct sg_model {
    pr_ctx *ctx;
    uint64_t seed;                          // of the initial weights
    int width, hidden;
    int64_t max_batch, chunk;
    int64_t step;
    int norm_blocks;
    SgDev dev;
    float *d_loss;
    int *d_err;
    double *d_normpart;
    int32_t *d_list;
    unsigned int *d_count;
    uint8_t *d_flags;
    int last_splits[SG_MAX_HIDDEN + 1];
    CUtensorMap tm_w[SG_MAX_HIDDEN + 1], tm_wt[SG_MAX_HIDDEN + 1];
    CUtensorMap tm_x0, tm_h[SG_MAX_HIDDEN], tm_dz[SG_MAX_HIDDEN], tm_dzo, tm_xi, tm_hi[2];
    // weight-gradient operands read MN-major: x0, h, dz, dzo with 64 x 64 boxes
    CUtensorMap tmn_x0, tmn_h[SG_MAX_HIDDEN], tmn_dz[SG_MAX_HIDDEN], tmn_dzo;
    // epilogue TMA-store maps (32-row boxes): h, GeLU'(z), dz, inference h
    CUtensorMap ts_h[SG_MAX_HIDDEN], ts_g[SG_MAX_HIDDEN], ts_dz[SG_MAX_HIDDEN], ts_hi[2];
    // fused inference (mlp_fused.cuh): activation ring, its maps, the weight
    // maps with 256-row boxes, per-(row block, layer) arrival counters
    int fused_ok, fused_on, fused_D, fused_ring;   // single-CTA tiles: slot lag, ring row blocks
    int fused_pair_ok, fused_D2, fused_ring2;      // CTA-pair tiles: slot lag, ring units of two row blocks
    int fused_clusters;                     // CTA pairs resident at once
    int fused_ring_rows;                    // row blocks per layer of the ring buffer
    long long wait_cycles;                  // bounded-wait limit of the fused kernel
    int stall_test;                         // SG_OPT_TEST_STALL
    int loss_l1;                            // SG_OPT_LOSS == SG_LOSS_L1
    float conf_tol;                         // SG_OPT_CONFIDENCE_PPM / 1e6; 0: off
    float tr_tol;                           // SG_OPT_TRANSPORT_CONFIDENCE_PPM / 1e6; 0: off
    __nv_bfloat16 *ring;                    // [L][fused_ring_rows * 128][W]
    uint32_t *d_done;
    CUtensorMap tmf_w[SG_MAX_HIDDEN + 1], tmf_ring_ld, tmf_ring_st;
    CUtensorMap tmp_w[SG_MAX_HIDDEN + 1];  // CTA pairs: half-height weight boxes
    // resident-activation inference (mlp_resident.cuh): CTA pairs held at
    // once (0: not available for this shape), weight boxes of W / 4 rows
    int res_pairs;
    CUtensorMap tmr_w[SG_MAX_HIDDEN + 1];
    // activations alternating between tensor and shared memory
    // (mlp_pingpong.cuh): CTA pairs the device holds at once, and the weight
    // maps (boxes of 64 rows: a CTA's half of a 128-row N-tile)
    int pp_pairs;
    CUtensorMap tmq_w[SG_MAX_HIDDEN + 1];
    std::vector<void *> allocs;
    // SG_OPT_TIME_MLP: event pairs (start, stop) around the MLP launches,
    // reused; the first 2 tev_used of them hold intervals not yet read
    int time_mlp;
    int tev_used;
    std::vector<cudaEvent_t> tev;
};
