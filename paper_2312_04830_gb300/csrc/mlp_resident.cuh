// Inference of the whole surrogate MLP with the activations resident in
// shared memory: a CTA pair (cta_group::2 MMAs, M = 256) takes a block of 256
// rows through every layer before it moves to its next block, each CTA keeping
// its 128 rows' activation (128 x W BF16, in the 128-byte-swizzled K-major
// layout the MMA reads) in its own shared memory.  Only the weights stream
// from L2, each CTA loading its half of every N-tile (the pair MMA's B split
// along N), so the L2 traffic is the weights once per 256 rows and nothing
// else: no activation leaves the SM, and no CTA waits on another pair.
//
// Each hidden layer's output (N = W) is computed as two N-tiles of BN = W / 2
// columns, accumulated in tensor memory at columns [0, BN) and [BN, 2 BN)
// (all 512 columns for W = 512).  Layer l + 1 reads the activation that layer
// l's epilogue writes in place, so the order of the MMAs is chosen for the
// epilogue to overlap them:
//   N-tile 0 of layer l      (all K)
//   N-tile 1 of layer l, K-blocks of the first half  -> the first half of the
//        activation is free: the epilogue of N-tile 0 writes it meanwhile
//   N-tile 1, second half    -> the epilogue of N-tile 1 follows
//   N-tile 0 of layer l + 1, first half (needs the first epilogue), second
//        half (needs the second), ...
// The input layer (K = 64, the standardised inputs as a TMA tile in a buffer
// of their own) and the output layer (N = 16, accumulated in the first 16 columns of
// the second accumulator) are interleaved with the neighbouring row blocks:
//   input N-tile 0 of block r, output layer of block r - 1, input N-tile 1 of
//   block r, hidden layers of block r, ...
// Barriers: a stage ring (full / empty) and the input buffer (x_full /
// x_empty) between the TMA producers and the MMA issuer; MMA completion
// (tcgen05.commit, multicast to both CTAs) tells the epilogues that an
// N-tile is ready and the activation half it overwrites is no longer read
// (`hid`), or that the output layer is done (`outf`); one arrival per CTA on
// the leader's barriers, after a named barrier of that CTA's epilogue warps,
// tells the MMA issuer that an activation half is written and its
// accumulator read (`epi_done`), or that the output accumulator has been read
// (`out_done`).  The issuing thread does as little as possible between MMAs
// (the tensor core does not queue far ahead of it): stage indices and
// phases advance by increments and shared-memory descriptors by 64-bit adds.
// Every wait is bounded; a failed wait sets the error flag, and every role
// then stops, lets its copies and MMAs in flight complete, and returns (the
// epilogue warps keep their trip counts, so their named barriers always
// complete).
#pragma once

#include "mlp_gemm.cuh"

namespace mlp {

constexpr int kResEpiWarps = 16;                       // four per TMEM lane quarter
constexpr int kResThreads = 64 + 32 * kResEpiWarps;    // producer, MMA issuer, epilogue
constexpr int kResOutBN = 16;                          // padded output width
constexpr int kResStages = 4;                          // weight stages (four measured faster than five)

struct ResidentArgs {
    CUtensorMap tm_x;                     // standardised inputs [rows][64], box 64 x 128
    CUtensorMap tm_w[kFusedMaxLayers];    // W_l [out][in]: box 64 x (W / 4) (hidden, this CTA's half of
                                          // an N-tile), 64 x 8 (output layer)
    const float *bias[kFusedMaxLayers];   // b_l [out_pad]
    int M;                                // rows of the chunk
    int L;                                // hidden layers
    int W;                                // width: 256 or 512
    float *out6;                          // [nout][ld6] physical outputs of the chunk's rows
    long long ld6;
    const float *out_mean, *out_std;      // [nout] de-standardisation
    int nout;                             // outputs in use (<= 16)
    const float *add_h;                   // per-row term added to output 2 (h), or NULL
    int log_mask;                         // bit j set = output j was learned as its logarithm
    int *err;                             // set to 1 when a bounded wait runs out
    long long wait_cycles;                // limit of every bounded wait
    int stall_test;                       // test hook: the MMA issuer waits for one epilogue too many
};

// Shared memory: the activation (128 x W BF16), the input tile (128 x 64
// BF16), the stage ring, the output layer's weights when they fit (this CTA's
// 8 rows x W, loaded once), the barriers, the biases of every layer.
struct ResCfg {
    static constexpr int kMaxSmem = 232448;   // 227 KB opt-in per CTA
    static constexpr int STAGE = 16384;       // this CTA's half of a weight K-block (at most 128 x 64 BF16)
    static constexpr int XBYTES = 16384;      // 128 x 64 BF16 input tile
    static constexpr int BAR_BYTES = 256;
    __host__ __device__ static int act_bytes(int W) { return 128 * W * 2; }
    __host__ __device__ static int bias_bytes(int L, int W) { return (L * W + kResOutBN) * 4; }
    __host__ __device__ static int wout_bytes(int W) { return (W / 64) * 1024; }   // 8 rows x W BF16
    __host__ __device__ static int smem_bytes(int L, int W, bool wo)
    {
        return 1024 + act_bytes(W) + XBYTES + kResStages * STAGE + (wo ? wout_bytes(W) : 0) + BAR_BYTES +
               bias_bytes(L, W);
    }
    // widths this kernel takes: two N-tiles of W / 2 columns fill at most the
    // 512 TMEM columns
    static bool supports(int L, int W)
    {
        return (W == 256 || W == 512) && L >= 1 && L < kFusedMaxLayers && smem_bytes(L, W, false) <= kMaxSmem;
    }
    // the output layer's weights stay in shared memory (else they stream
    // through the stage ring like the others)
    static bool wout_resident(int L, int W) { return smem_bytes(L, W, true) <= kMaxSmem; }
};

// Position in the stage ring: index and phase parity, advanced by increments
struct RingPos {
    uint32_t s = 0, ph = 0;
    __device__ __forceinline__ void next()
    {
        if (++s == (uint32_t)kResStages) {
            s = 0;
            ph ^= 1u;
        }
    }
};

// Named barrier among `threads` threads (id 1..15; id 0 is __syncthreads)
__device__ __forceinline__ void named_sync(uint32_t id, uint32_t threads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// GeLU(acc + b) of 16 accumulator columns, as BF16 into the resident
// activation (K-blocks of 128 rows x 128 B, 16-byte chunks swizzled by the
// row's index within its 8-row atom, as TMA's 128-byte swizzle places them).
// rx: shared address of the row's 128-byte line XOR (row & 7) << 4, so that
// chunk j of the line lies at rx ^ (j << 4); j0: the first of the two chunks.
__device__ __forceinline__ void act_chunk(const uint32_t (&r)[16], const float *sb, uint32_t rx, int j0)
{
    const float4 *b4 = reinterpret_cast<const float4 *>(sb);
    uint32_t pk[8];
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
        const float4 b = b4[jj];
        const float2 g0 = gelu2(make_float2(__uint_as_float(r[4 * jj]), __uint_as_float(r[4 * jj + 1])),
                                make_float2(b.x, b.y));
        const float2 g1 = gelu2(make_float2(__uint_as_float(r[4 * jj + 2]), __uint_as_float(r[4 * jj + 3])),
                                make_float2(b.z, b.w));
        pk[2 * jj] = pack_bf16(g0.x, g0.y);
        pk[2 * jj + 1] = pack_bf16(g1.x, g1.y);
    }
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(rx ^ (uint32_t)(j0 << 4)), "r"(pk[0]), "r"(pk[1]),
                 "r"(pk[2]), "r"(pk[3])
                 : "memory");
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(rx ^ (uint32_t)((j0 + 1) << 4)), "r"(pk[4]),
                 "r"(pk[5]), "r"(pk[6]), "r"(pk[7])
                 : "memory");
}

// The epilogue of one warp's NCOL columns of an N-tile: TMEM loads of 16
// columns double-buffered, everything unrolled (column offsets are
// immediates); rx as for act_chunk, for the first column.  (Loads of 32 or
// all columns per wait measured slower: they spill at 96 registers.)
template <int NCOL>
__device__ __forceinline__ void act_columns(uint32_t taddr, const float *sb, uint32_t rx)
{
    uint32_t ra[16], rb[16];
    umma::tmem_ld16(taddr, ra);
#pragma unroll
    for (int c = 0; c < NCOL; c += 32) {
        umma::tmem_ld_wait(ra);
        umma::tmem_ld16(taddr + c + 16, rb);
        act_chunk(ra, sb + c, rx, c / 8);
        umma::tmem_ld_wait(rb);
        if (c + 32 < NCOL) umma::tmem_ld16(taddr + c + 32, ra);
        act_chunk(rb, sb + c + 16, rx, c / 8 + 2);
    }
}

template <int W, bool WO>
__global__ void __launch_bounds__(kResThreads, 1) mlp_resident_kernel(const __grid_constant__ ResidentArgs a)
{
    static_assert(W == 256 || W == 512, "resident activations: width 256 or 512");
    constexpr int S = kResStages;
    constexpr int BN = W / 2, nkb = W / 64, NCOL = BN / 4;
    constexpr uint32_t kStageDesc = ResCfg::STAGE >> 4;   // descriptor address units per stage / K-block
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int L = a.L;
    uint8_t *act = smem;
    uint8_t *xbuf = smem + ResCfg::act_bytes(W);
    uint8_t *stage = xbuf + ResCfg::XBYTES;
    uint8_t *wout = stage + S * ResCfg::STAGE;   // (WO) the output layer's weights, K-blocks of 8 x 64
    uint64_t *full = reinterpret_cast<uint64_t *>(wout + (WO ? ResCfg::wout_bytes(W) : 0));
    uint64_t *empty = full + S;
    uint64_t *x_full = empty + S;     // input tile landed (both CTAs')
    uint64_t *x_empty = x_full + 1;   // input tile no longer read
    uint64_t *hid = x_empty + 1;      // [2] N-tile b ready, activation half b no longer read
    uint64_t *outf = hid + 2;         // output layer done
    uint64_t *epi_done = outf + 1;    // [2] (leader) activation half b written, accumulator b read
    uint64_t *out_done = epi_done + 2;   // (leader) output accumulator read
    uint64_t *drain = out_done + 1;      // (leader) every MMA issued has completed
    uint64_t *w_full = drain + 1;        // (WO) the output layer's weights landed (both CTAs')
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(w_full + 1);
    float *sbias = reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(full) + ResCfg::BAR_BYTES);   // [L W + 16]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = umma::cluster_ctarank();
    const bool leader = rank == 0;
    const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
    const int R = (a.M + 255) / 256;                                  // row blocks of 256
    const int nr = pair < R ? (R - pair + npairs - 1) / npairs : 0;   // this pair's row blocks
    const long long wc = a.wait_cycles;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            umma::mbar_init(&full[s], 1);
            umma::mbar_init(&empty[s], 1);
        }
        umma::mbar_init(x_full, 1);
        umma::mbar_init(x_empty, 1);
        umma::mbar_init(&hid[0], 1);
        umma::mbar_init(&hid[1], 1);
        umma::mbar_init(outf, 1);
        umma::mbar_init(&epi_done[0], 2);
        umma::mbar_init(&epi_done[1], 2);
        umma::mbar_init(out_done, 2);
        umma::mbar_init(drain, 1);
        umma::mbar_init(w_full, 1);
        *tmem_slot = 0u;
        umma::fence_mbar_init();
        umma::tma_prefetch_desc(&a.tm_x);
    }
    for (int e = threadIdx.x; e < L * W + kResOutBN; e += blockDim.x) {
        const int l = (e < L * W) ? e / W : L;
        const int n = (e < L * W) ? e - l * W : e - L * W;
        sbias[e] = __ldg(a.bias[l] + n);
    }
    __syncthreads();
    if (warp == 1) {
        umma::tmem_alloc_pair(tmem_slot, 512);
        umma::tmem_relinquish_pair();
    }
    umma::tc_fence_before();
    __syncthreads();
    umma::cluster_sync();   // both CTAs' barriers initialised before any copy or MMA signals them
    umma::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool fail = false;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer (each CTA)
        if (lane == 0) {
            RingPos rp;
            uint32_t it = 0, nx = 0;
            const uint32_t wbytes = 2u * (uint32_t)(BN / 2) * 128u;   // the pair's halves of a weight K-block
            const int hrow = (int)rank * (BN / 2);                       // this CTA's rows of an N-tile
            auto put = [&](const CUtensorMap *tm, int c0, int c1, uint32_t bytes) {
                if (fail) return;
                if (it >= (uint32_t)S && !umma::mbar_wait(&empty[rp.s], rp.ph ^ 1u, wc)) {
                    fail = true;
                    return;
                }
                if (leader) umma::mbar_arrive_expect_tx(&full[rp.s], bytes);
                umma::tma_load_2d_pair(stage + rp.s * ResCfg::STAGE, tm, umma::mapa_shared(umma::smem_u32(&full[rp.s]), 0u),
                                       c0, c1);
                ++it;
                rp.next();
            };
            auto put_out = [&]() {
                if (!WO)
                    for (int k = 0; k < nkb; ++k) put(&a.tm_w[L], k * 64, (int)rank * 8, 2u * 8u * 128u);
            };
            if (WO && nr > 0) {   // the output layer's weights, once
                if (leader) umma::mbar_arrive_expect_tx(w_full, 2u * (uint32_t)ResCfg::wout_bytes(W));
                for (int k = 0; k < nkb; ++k)
                    umma::tma_load_2d_pair(wout + k * 1024, &a.tm_w[L], umma::mapa_shared(umma::smem_u32(w_full), 0u),
                                           k * 64, (int)rank * 8);
            }
            for (int i = 0; i < nr && !fail; ++i) {
                const int r = pair + i * npairs;
                // the input tile, once the previous block's input layer has read it
                if (i > 0 && !umma::mbar_wait(x_empty, (uint32_t)(i - 1) & 1u, wc)) {
                    fail = true;
                    break;
                }
                if (leader) umma::mbar_arrive_expect_tx(x_full, 2u * (uint32_t)ResCfg::XBYTES);
                umma::tma_load_2d_pair(xbuf, &a.tm_x, umma::mapa_shared(umma::smem_u32(x_full), 0u), 0,
                                       r * 256 + (int)rank * 128);
                ++nx;
                put(&a.tm_w[0], 0, hrow, wbytes);
                if (i > 0) put_out();
                put(&a.tm_w[0], 0, BN + hrow, wbytes);
                for (int l = 1; l < L; ++l)
                    for (int b = 0; b < 2; ++b)
                        for (int k = 0; k < nkb; ++k) put(&a.tm_w[l], k * 64, b * BN + hrow, wbytes);
            }
            if (nr > 0) put_out();
            const uint32_t it_end = it;
            // the leader's MMAs read this CTA's stages: every use is released
            // before the CTA may exit
            for (int j = 0; j < S && !fail; ++j) {
                if (it >= (uint32_t)S && !umma::mbar_wait(&empty[rp.s], rp.ph ^ 1u, wc)) fail = true;
                ++it;
                rp.next();
            }
            // no copy may still be landing in shared memory at exit (the
            // peer's copies complete on the leader's barriers)
            if (leader) {
                for (uint32_t k = (it_end > (uint32_t)S ? it_end - S : 0u); k < it_end; ++k)
                    if (!umma::mbar_wait(&full[k % S], (k / S) & 1u, 200000000LL)) fail = true;
                if (nx > 0 && !umma::mbar_wait(x_full, (uint32_t)(nx - 1) & 1u, 200000000LL)) fail = true;
                if (WO && nr > 0 && !umma::mbar_wait(w_full, 0u, 200000000LL)) fail = true;
            }
            if (fail) atomicExch(a.err, 1);
        }
    } else if (warp == 1) {
        // ----------------------------------------------- MMA issuer (leader)
        if (lane == 0 && leader) {
            RingPos rp;
            uint32_t ne0 = 0, ne1 = 0, no = 0, nxf = 0;
            const uint32_t id_h = umma::idesc_bf16_f32(256, BN), id_o = umma::idesc_bf16_f32(256, kResOutBN);
            const uint32_t acc0 = tmem, acc1 = tmem + (uint32_t)BN;
            const uint64_t d_act = umma::sdesc_kmajor_sw128(umma::smem_u32(act));
            const uint64_t d_x = umma::sdesc_kmajor_sw128(umma::smem_u32(xbuf));
            const uint64_t d_st = umma::sdesc_kmajor_sw128(umma::smem_u32(stage));
            const uint64_t d_wo = umma::sdesc_kmajor_sw128(umma::smem_u32(wout));
            uint32_t nwo = 0;
            auto wait_bar = [&](uint64_t *bar, uint32_t &n) {
                if (!fail && !umma::mbar_wait(bar, n & 1u, wc)) fail = true;
                ++n;
                umma::tc_fence_after();
            };
            // the next stage, once landed: its descriptor
            auto take = [&]() -> uint64_t {
                if (!fail && !umma::mbar_wait(&full[rp.s], rp.ph, wc)) fail = true;
                umma::tc_fence_after();
                return d_st + (uint64_t)(rp.s * kStageDesc);
            };
            // release the stage just read, once the MMAs reading it complete
            auto give = [&]() {
                umma::mma_commit_pair_mc(&empty[rp.s], (uint16_t)0x3);
                rp.next();
            };
            // one K-block: four K = 16 MMAs (descriptor address +32 B each)
            auto kblock = [&](uint32_t d, uint64_t da, uint64_t db, uint32_t id, bool acc_in) {
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    umma::mma_bf16_pair(d, da + 2 * kk, db + 2 * kk, id, (acc_in || kk > 0) ? 1u : 0u);
            };
            // both activation halves written (epi_done[0] waited before); with
            // `next`, the next block's first epilogue may start once the first
            // half of the activation has been read
            auto output_layer = [&](bool next) {
                wait_bar(&epi_done[1], ne1);
                if (WO && nwo == 0) wait_bar(w_full, nwo);
                for (int k = 0; k < nkb && !fail; ++k) {
                    if (WO) {
                        kblock(acc1, d_act + (uint64_t)(k * kStageDesc), d_wo + (uint64_t)(k * 64), id_o, k > 0);
                    } else {
                        const uint64_t db = take();
                        if (fail) break;
                        kblock(acc1, d_act + (uint64_t)(k * kStageDesc), db, id_o, k > 0);
                        give();
                    }
                    if (next && k == nkb / 2 - 1) umma::mma_commit_pair_mc(&hid[0], (uint16_t)0x3);
                }
                if (!fail) umma::mma_commit_pair_mc(outf, (uint16_t)0x3);
            };
            for (int i = 0; i < nr && !fail; ++i) {
                if (i > 0) wait_bar(&epi_done[0], ne0);   // accumulator 0 read by the last layer's epilogue
                wait_bar(x_full, nxf);
                uint64_t db = take();
                if (fail) break;
                kblock(acc0, d_x, db, id_h, false);
                give();
                if (i > 0)
                    output_layer(true);   // of the previous row block
                else
                    umma::mma_commit_pair_mc(&hid[0], (uint16_t)0x3);
                if (fail) break;
                if (i > 0) wait_bar(out_done, no);
                db = take();
                if (fail) break;
                kblock(acc1, d_x, db, id_h, false);
                give();
                umma::mma_commit_pair_mc(x_empty, (uint16_t)0x3);
                umma::mma_commit_pair_mc(&hid[1], (uint16_t)0x3);
                for (int l = 1; l < L && !fail; ++l) {
                    for (int k = 0; k < nkb && !fail; ++k) {
                        if (k == 0) {
                            wait_bar(&epi_done[0], ne0);
                            if (a.stall_test && i == 0 && l == 1) wait_bar(&epi_done[0], ne0);   // never arrives
                        }
                        if (k == nkb / 2) wait_bar(&epi_done[1], ne1);
                        db = take();
                        if (fail) break;
                        kblock(acc0, d_act + (uint64_t)(k * kStageDesc), db, id_h, k > 0);
                        give();
                    }
                    for (int k = 0; k < nkb && !fail; ++k) {
                        db = take();
                        if (fail) break;
                        kblock(acc1, d_act + (uint64_t)(k * kStageDesc), db, id_h, k > 0);
                        give();
                        if (k == nkb / 2 - 1) umma::mma_commit_pair_mc(&hid[0], (uint16_t)0x3);
                    }
                    if (!fail) umma::mma_commit_pair_mc(&hid[1], (uint16_t)0x3);
                }
            }
            if (nr > 0 && !fail) {
                wait_bar(&epi_done[0], ne0);
                output_layer(false);
            }
            // every MMA issued has completed before tensor memory is freed
            umma::mma_commit_pair_mc(drain, (uint16_t)0x1);
            if (!umma::mbar_wait(drain, 0u, 200000000LL)) fail = true;
            if (fail) atomicExch(a.err, 1);
        }
    } else {
        // ------------------------------------------------ epilogue (each CTA)
        const int ew = warp - 2;        // 0..15
        const int q = warp & 3;         // TMEM lane quarter this warp may access
        const int cg = ew >> 2;         // column quarter of an N-tile
        const int row = q * 32 + lane;  // this thread's row of the CTA's 128
        const uint32_t lanes = (uint32_t)(q * 32) << 16;
        const uint32_t act_row = umma::smem_u32(act) + (uint32_t)(row * 128);
        const uint32_t epi_c0 = umma::mapa_shared(umma::smem_u32(&epi_done[0]), 0u);
        const uint32_t epi_c1 = umma::mapa_shared(umma::smem_u32(&epi_done[1]), 0u);
        const uint32_t out_c = umma::mapa_shared(umma::smem_u32(out_done), 0u);
        uint32_t nh[2] = {0u, 0u}, nof = 0u;
        // failed waits are not retried, but the trip counts stay the same, so
        // every named barrier completes
        auto wait_bar = [&](uint64_t *bar, uint32_t &n) {
            if (!fail && !umma::mbar_wait(bar, n & 1u, wc)) fail = true;
            ++n;
            fail = __any_sync(0xffffffffu, fail);   // warp-uniform: tcgen05.ld needs the whole warp
            umma::tc_fence_after();
        };
        // warps 2..5 (one per lane quarter): de-standardised outputs of row block r
        // (the per-row term and the first 8 outputs' bias, scale and shift are
        // loaded before the wait; the rest is read after it)
        auto output_epilogue = [&](int r, bool signal) {
            const int m = r * 256 + (int)rank * 128 + row;
            const float hadd = (a.add_h && m < a.M) ? __ldg(a.add_h + m) : 0.f;
            const float *sb = sbias + L * W;
            float ob[8], os[8], om[8];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                ob[jj] = sb[jj];
                os[jj] = __ldg(a.out_std + jj);
                om[jj] = __ldg(a.out_mean + jj);
            }
            wait_bar(outf, nof);
            if (!fail) {
                uint32_t rr[16];
                umma::tmem_ld16(tmem + lanes + (uint32_t)BN, rr);
                umma::tmem_ld_wait(rr);
                if (m < a.M) {
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        if (jj >= a.nout) break;
                        float qv = jj < 8 ? (__uint_as_float(rr[jj]) + ob[jj & 7]) * os[jj & 7] + om[jj & 7]
                                          : (__uint_as_float(rr[jj]) + sb[jj]) * __ldg(a.out_std + jj) +
                                                __ldg(a.out_mean + jj);
                        if (jj == 2) qv += hadd;
                        a.out6[(long long)jj * a.ld6 + m] = ((a.log_mask >> jj) & 1) ? __expf(qv) : qv;
                    }
                }
            }
            umma::tc_fence_before();
            named_sync(2, 128);
            if (signal && ew == 0 && lane == 0 && !fail) umma::mbar_arrive_cluster(out_c);
        };
        for (int i = 0; i < nr; ++i) {
            if (i > 0 && ew < 4) output_epilogue(pair + (i - 1) * npairs, true);
            for (int l = 0; l < L; ++l) {
                for (int b = 0; b < 2; ++b) {
                    wait_bar(&hid[b], nh[b]);
                    if (!fail) {
                        const int n0 = b * BN + cg * NCOL;   // first column of this warp
                        // its line: K-block n0 / 64, 16-byte chunk (n0 % 64) / 8, swizzled by row % 8
                        const uint32_t rx = (act_row + (uint32_t)((n0 >> 6) * 16384)) ^
                                            (uint32_t)(((row & 7) ^ ((n0 & 63) >> 3)) << 4);
                        act_columns<NCOL>(tmem + lanes + (uint32_t)n0, sbias + l * W + n0, rx);
                    }
                    umma::fence_async_smem();   // the activation writes, visible to the tensor core
                    umma::tc_fence_before();
                    named_sync(1, 32 * kResEpiWarps);
                    if (ew == 0 && lane == 0 && !fail) umma::mbar_arrive_cluster(b ? epi_c1 : epi_c0);
                }
            }
        }
        if (nr > 0 && ew < 4) output_epilogue(pair + (nr - 1) * npairs, false);
        if (fail && lane == 0) atomicExch(a.err, 1);
    }
    __syncwarp();
    umma::tc_fence_before();
    __syncthreads();
    // the pair's MMAs, barrier signals and remote arrivals are all done before
    // either CTA frees its tensor memory or exits
    umma::cluster_sync();
    if (warp == 1) {
        __syncwarp();
        umma::tc_fence_after();
        umma::tmem_dealloc_pair(tmem, 512);
    }
}

}  // namespace mlp
