// Inference of the whole surrogate MLP with the activation alternating
// between tensor memory and shared memory.  As in the resident-activation
// kernel (mlp_resident.cuh), a CTA pair (cta_group::2 MMAs, M = 256) takes a
// block of 256 rows through every layer, each CTA holding its 128 rows, and
// only the weights stream from L2.  Here no layer writes over its own input:
// layer l's output (GeLU, BF16) goes to tensor memory when l is even and to
// shared memory when l is odd, and layer l + 1 reads it from there as the MMA's
// A operand (tcgen05.mma with A in tensor memory, or the 128-byte-swizzled
// K-major tile in shared memory).  A layer's epilogue can therefore start on
// an N-tile as soon as that N-tile's MMAs are done, while the tensor core
// works on the next N-tile; the next layer's first N-tile waits, K-block by
// K-block, only for the epilogues that wrote those columns.
//
// Tensor memory (512 columns of 128 lanes): the BF16 activation in columns
// [0, W / 2) (two values of consecutive K per column, a row per lane), and
// two accumulators of 128 columns at 256 and 384.  Each layer is computed in
// N-tiles of 128 columns, alternating between the two accumulators; the
// output layer (N = 16) is one more N-tile.  The tiles of all layers and
// blocks are counted in one sequence g; tile g uses accumulator g % 2, and
// its epilogue's completion is an arrival on edone[g % 2] (phase g / 2), so
// tile g + 2 waits for edone of tile g before it accumulates there.
//
// Hazards the schedule leaves to the MMA completion order: an epilogue writes
// a buffer only after its own tile's MMAs complete (tcgen05.commit tracks
// every MMA issued before), and the MMAs that last read that buffer (the
// layer before, or the previous block's) were issued earlier.
//
// Weights: each CTA loads its 64 rows of a 128-row N-tile, two K-blocks of 64
// per stage (16 KB stages, four of them: one barrier poll, fence and commit
// of the MMA issuer per eight MMAs, which hides that bookkeeping behind the
// 128-column MMAs; the input layer's stage holds two N-tiles' single
// K-blocks); the output layer's 8 rows per CTA stay in shared memory when
// they fit.  Every wait is bounded; a failed wait
// sets the error flag, the roles stop, and the epilogue warps keep their trip
// counts so their named barrier always completes.
#pragma once

#include "mlp_resident.cuh"

namespace mlp {

constexpr int kPPEpiWarps = 16;                      // four per TMEM lane quarter
constexpr int kPPThreads = 64 + 32 * kPPEpiWarps;    // producer, MMA issuer, epilogue
constexpr int kPPBN = 128;                           // N-tile width
constexpr int kPPStages = 4;
constexpr int kPPStage = 16384;                      // two halves of this CTA's 64 rows x 64 K of a weight N-tile
constexpr int kPPHalf = 8192;
constexpr uint32_t kPPAccCol = 256;                  // first accumulator column

// Shared memory: the activation (128 x W BF16), the input tile (128 x 64
// BF16), the stage ring, the output layer's weights when they fit, the
// barriers, the biases of every layer.
struct PPCfg {
    static constexpr int kMaxSmem = 232448;
    static constexpr int XBYTES = 16384;
    static constexpr int BAR_BYTES = 256;
    __host__ __device__ static int act_bytes(int W) { return 128 * W * 2; }
    __host__ __device__ static int bias_bytes(int L, int W) { return (L * W + kResOutBN) * 4; }
    __host__ __device__ static int wout_bytes(int W) { return (W / 64) * 1024; }
    __host__ __device__ static int smem_bytes(int L, int W, bool wo)
    {
        return 1024 + act_bytes(W) + XBYTES + kPPStages * kPPStage + (wo ? wout_bytes(W) : 0) + BAR_BYTES +
               bias_bytes(L, W);
    }
    static bool supports(int L, int W)
    {
        return (W == 256 || W == 512) && L >= 1 && L < kFusedMaxLayers && smem_bytes(L, W, false) <= kMaxSmem;
    }
    static bool wout_resident(int L, int W) { return smem_bytes(L, W, true) <= kMaxSmem; }
};

struct PPRing {
    uint32_t s = 0, ph = 0;
    __device__ __forceinline__ void next()
    {
        if (++s == (uint32_t)kPPStages) {
            s = 0;
            ph ^= 1u;
        }
    }
};

// GeLU(acc + b) of 16 accumulator columns, as 8 BF16 pairs (the same
// arithmetic as the other inference kernels)
__device__ __forceinline__ void pp_pack(const uint32_t (&r)[16], const float *sb, uint32_t *pk)
{
    const float4 *b4 = reinterpret_cast<const float4 *>(sb);
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
}

// two 16-byte chunks of a row's 128-byte line (rx: the line's address XOR
// (row & 7) << 4, the 128-byte swizzle), u0 the first chunk
__device__ __forceinline__ void pp_store_smem(uint32_t rx, int u0, const uint32_t *pk)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(rx ^ (uint32_t)(u0 << 4)), "r"(pk[0]), "r"(pk[1]),
                 "r"(pk[2]), "r"(pk[3])
                 : "memory");
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(rx ^ (uint32_t)((u0 + 1) << 4)), "r"(pk[4]),
                 "r"(pk[5]), "r"(pk[6]), "r"(pk[7])
                 : "memory");
}

template <int W, bool WO>
__global__ void __launch_bounds__(kPPThreads, 1) mlp_pingpong_kernel(const __grid_constant__ ResidentArgs a)
{
    static_assert(W == 256 || W == 512, "width 256 or 512");
    constexpr int S = kPPStages;
    constexpr int NT = W / kPPBN, nkb = W / 64;   // N-tiles of a layer, K-blocks of the activation
    constexpr uint32_t kBlkDesc = 16384u >> 4;    // descriptor units per activation K-block
    constexpr uint32_t kStageDesc = (uint32_t)kPPStage >> 4;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int L = a.L;
    uint8_t *act = smem;
    uint8_t *xbuf = smem + PPCfg::act_bytes(W);
    uint8_t *stage = xbuf + PPCfg::XBYTES;
    uint8_t *wout = stage + S * kPPStage;
    uint64_t *full = reinterpret_cast<uint64_t *>(wout + (WO ? PPCfg::wout_bytes(W) : 0));
    uint64_t *empty = full + S;
    uint64_t *x_full = empty + S;
    uint64_t *x_empty = x_full + 1;
    uint64_t *afull = x_empty + 1;   // [2] accumulator p's tile computed (both CTAs)
    uint64_t *edone = afull + 2;     // [2] (leader) tile g's epilogue done, g % 2 = p
    uint64_t *drain = edone + 2;     // (leader) every MMA issued has completed
    uint64_t *w_full = drain + 1;    // (WO) the output layer's weights landed
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(w_full + 1);
    float *sbias = reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(full) + PPCfg::BAR_BYTES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = umma::cluster_ctarank();
    const bool leader = rank == 0;
    const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
    const int R = (a.M + 255) / 256;
    const int nr = pair < R ? (R - pair + npairs - 1) / npairs : 0;
    const long long wc = a.wait_cycles;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            umma::mbar_init(&full[s], 1);
            umma::mbar_init(&empty[s], 1);
        }
        umma::mbar_init(x_full, 1);
        umma::mbar_init(x_empty, 1);
        umma::mbar_init(&afull[0], 1);
        umma::mbar_init(&afull[1], 1);
        umma::mbar_init(&edone[0], 2);
        umma::mbar_init(&edone[1], 2);
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
    umma::cluster_sync();
    umma::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool fail = false;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer (each CTA)
        if (lane == 0) {
            PPRing rp;
            uint32_t it = 0, nx = 0;
            const uint32_t wbytes = 2u * 2u * 64u * 128u;   // both CTAs' two K-blocks of a stage
            const int hrow = (int)rank * (kPPBN / 2);
            // one stage: the boxes at (k0, r0) and (k1, r1) in its two halves
            auto put = [&](const CUtensorMap *tm, int k0, int r0, int k1, int r1, uint32_t bytes) {
                if (fail) return;
                if (it >= (uint32_t)S && !umma::mbar_wait(&empty[rp.s], rp.ph ^ 1u, wc)) {
                    fail = true;
                    return;
                }
                if (leader) umma::mbar_arrive_expect_tx(&full[rp.s], bytes);
                const uint32_t bar = umma::mapa_shared(umma::smem_u32(&full[rp.s]), 0u);
                umma::tma_load_2d_pair(stage + rp.s * kPPStage, tm, bar, k0, r0);
                umma::tma_load_2d_pair(stage + rp.s * kPPStage + kPPHalf, tm, bar, k1, r1);
                ++it;
                rp.next();
            };
            if (WO && nr > 0) {
                if (leader) umma::mbar_arrive_expect_tx(w_full, 2u * (uint32_t)PPCfg::wout_bytes(W));
                for (int k = 0; k < nkb; ++k)
                    umma::tma_load_2d_pair(wout + k * 1024, &a.tm_w[L], umma::mapa_shared(umma::smem_u32(w_full), 0u),
                                           k * 64, (int)rank * 8);
            }
            for (int i = 0; i < nr && !fail; ++i) {
                const int r = pair + i * npairs;
                if (i > 0 && !umma::mbar_wait(x_empty, (uint32_t)(i - 1) & 1u, wc)) {
                    fail = true;
                    break;
                }
                if (leader) umma::mbar_arrive_expect_tx(x_full, 2u * (uint32_t)PPCfg::XBYTES);
                umma::tma_load_2d_pair(xbuf, &a.tm_x, umma::mapa_shared(umma::smem_u32(x_full), 0u), 0,
                                       r * 256 + (int)rank * 128);
                ++nx;
                for (int j = 0; j < NT; j += 2) put(&a.tm_w[0], 0, j * kPPBN + hrow, 0, (j + 1) * kPPBN + hrow, wbytes);
                for (int l = 1; l < L; ++l)
                    for (int j = 0; j < NT; ++j)
                        for (int k = 0; k < nkb; k += 2)
                            put(&a.tm_w[l], k * 64, j * kPPBN + hrow, (k + 1) * 64, j * kPPBN + hrow, wbytes);
                if (!WO)
                    for (int k = 0; k < nkb; k += 2)
                        put(&a.tm_w[L], k * 64, (int)rank * 8, (k + 1) * 64, (int)rank * 8, 2u * 2u * 8u * 128u);
            }
            const uint32_t it_end = it;
            for (int j = 0; j < S && !fail; ++j) {
                if (it >= (uint32_t)S && !umma::mbar_wait(&empty[rp.s], rp.ph ^ 1u, wc)) fail = true;
                ++it;
                rp.next();
            }
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
            PPRing rp;
            uint32_t g = 0, ev = 0, nxf = 0, nwo = 0;
            const uint32_t id_h = umma::idesc_bf16_f32(256, kPPBN), id_o = umma::idesc_bf16_f32(256, kResOutBN);
            const uint32_t actT = tmem, acc0 = tmem + kPPAccCol;
            const uint64_t d_act = umma::sdesc_kmajor_sw128(umma::smem_u32(act));
            const uint64_t d_x = umma::sdesc_kmajor_sw128(umma::smem_u32(xbuf));
            const uint64_t d_st = umma::sdesc_kmajor_sw128(umma::smem_u32(stage));
            const uint64_t d_wo = umma::sdesc_kmajor_sw128(umma::smem_u32(wout));
            // every epilogue event up to tile e, in order
            auto wait_ev = [&](uint32_t e) {
                while (!fail && ev <= e) {
                    if (!umma::mbar_wait(&edone[ev & 1u], (ev >> 1) & 1u, wc)) fail = true;
                    ++ev;
                }
                umma::tc_fence_after();
            };
            auto take = [&]() -> uint64_t {
                if (!fail && !umma::mbar_wait(&full[rp.s], rp.ph, wc)) fail = true;
                umma::tc_fence_after();
                return d_st + (uint64_t)(rp.s * kStageDesc);
            };
            auto give = [&]() {
                umma::mma_commit_pair_mc(&empty[rp.s], (uint16_t)0x3);
                rp.next();
            };
            // one K-block (four K = 16 MMAs) with A in shared memory or in
            // tensor memory (8 columns per K = 16)
            auto kblock_s = [&](uint32_t d, uint64_t da, uint64_t db, uint32_t id, bool acc_in) {
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    umma::mma_bf16_pair(d, da + 2 * kk, db + 2 * kk, id, (acc_in || kk > 0) ? 1u : 0u);
            };
            auto kblock_t = [&](uint32_t d, uint32_t ta, uint64_t db, uint32_t id, bool acc_in) {
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    umma::mma_bf16_pair_ts(d, ta + 8u * kk, db + 2 * kk, id, (acc_in || kk > 0) ? 1u : 0u);
            };
            // a tile from the previous layer's output (in tensor memory when
            // that layer's index is even); the first tile of a layer waits,
            // per pair of K-blocks, for the epilogue that wrote them
            auto tile = [&](int lsrc, uint32_t prev_first, bool first_of_layer, bool output) {
                if (g >= 2) wait_ev(g - 2);   // the accumulator read by tile g - 2's epilogue
                const uint32_t d = acc0 + (g & 1u) * kPPBN;
                const bool fromT = (lsrc & 1) == 0;
                if (output && WO && nwo == 0) {
                    if (!fail && !umma::mbar_wait(w_full, 0u, wc)) fail = true;
                    ++nwo;
                    umma::tc_fence_after();
                }
                const uint32_t id = output ? id_o : id_h;
#pragma unroll 1
                for (int k = 0; k < nkb && !fail; k += 2) {   // two K-blocks per stage
                    if (first_of_layer) wait_ev(prev_first + (uint32_t)(k >> 1));
                    if (fail) break;
                    uint64_t db0, db1;
                    if (output && WO) {
                        db0 = d_wo + (uint64_t)(k * 64);
                        db1 = db0 + 64;
                    } else {
                        db0 = take();
                        if (fail) break;
                        db1 = db0 + (uint64_t)(kPPHalf >> 4);
                    }
                    if (fromT) {
                        kblock_t(d, actT + 32u * (uint32_t)k, db0, id, k > 0);
                        kblock_t(d, actT + 32u * (uint32_t)(k + 1), db1, id, true);
                    } else {
                        kblock_s(d, d_act + (uint64_t)(k * kBlkDesc), db0, id, k > 0);
                        kblock_s(d, d_act + (uint64_t)((k + 1) * kBlkDesc), db1, id, true);
                    }
                    if (!(output && WO)) give();
                }
                if (!fail) umma::mma_commit_pair_mc(&afull[g & 1u], (uint16_t)0x3);
                ++g;
            };
            for (int i = 0; i < nr && !fail; ++i) {
                if (!fail && !umma::mbar_wait(x_full, nxf & 1u, wc)) fail = true;
                ++nxf;
                umma::tc_fence_after();
                // input layer: K = 64 from the input tile, two N-tiles per stage
                for (int j = 0; j < NT && !fail; j += 2) {
                    const uint64_t db = take();
                    if (fail) break;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (g >= 2) wait_ev(g - 2);
                        if (fail) break;
                        kblock_s(acc0 + (g & 1u) * kPPBN, d_x, db + (uint64_t)(h * (kPPHalf >> 4)), id_h, false);
                        umma::mma_commit_pair_mc(&afull[g & 1u], (uint16_t)0x3);
                        ++g;
                    }
                    give();
                }
                if (fail) break;
                umma::mma_commit_pair_mc(x_empty, (uint16_t)0x3);
                for (int l = 1; l < L && !fail; ++l) {
                    const uint32_t prev_first = g - (uint32_t)NT;
                    if (a.stall_test && i == 0 && l == 1) wait_ev(g);   // the epilogue of a tile never issued
                    for (int j = 0; j < NT && !fail; ++j) tile(l - 1, prev_first, j == 0, false);
                }
                if (!fail) tile(L - 1, g - (uint32_t)NT, true, true);
            }
            umma::mma_commit_pair_mc(drain, (uint16_t)0x1);
            if (!umma::mbar_wait(drain, 0u, 200000000LL)) fail = true;
            if (fail) atomicExch(a.err, 1);
        }
    } else {
        // ------------------------------------------------ epilogue (each CTA)
        const int ew = warp - 2;        // 0..15
        const int q = warp & 3;         // TMEM lane quarter
        const int cg = ew >> 2;         // column quarter of an N-tile (32 columns)
        const int row = q * 32 + lane;
        const uint32_t lanes = (uint32_t)(q * 32) << 16;
        const uint32_t act_row = umma::smem_u32(act) + (uint32_t)(row * 128);
        const uint32_t swz = (uint32_t)((row & 7) << 4);
        uint32_t g = 0;
        const uint32_t edone_c[2] = {umma::mapa_shared(umma::smem_u32(&edone[0]), 0u),
                                     umma::mapa_shared(umma::smem_u32(&edone[1]), 0u)};
        auto wait_tile = [&]() {
            if (!fail && !umma::mbar_wait(&afull[g & 1u], (g >> 1) & 1u, wc)) fail = true;
            fail = __any_sync(0xffffffffu, fail);
            umma::tc_fence_after();
        };
        auto finish_tile = [&]() {
            umma::tc_fence_before();
            named_sync(1, 32 * kPPEpiWarps);
            if (ew == 0 && lane == 0 && !fail) umma::mbar_arrive_cluster(edone_c[g & 1u]);
            ++g;
        };
        for (int i = 0; i < nr; ++i) {
            const int r = pair + i * npairs;
            for (int l = 0; l < L; ++l) {
                const bool toT = (l & 1) == 0;
                for (int j = 0; j < NT; ++j) {
                    wait_tile();
                    if (!fail) {
                        const int c0 = j * kPPBN + cg * 32;   // this warp's first output column
                        const uint32_t ta = tmem + kPPAccCol + (g & 1u) * kPPBN + lanes + (uint32_t)(cg * 32);
                        uint32_t ra[16], rb[16], pk[16];
                        umma::tmem_ld16(ta, ra);
                        umma::tmem_ld16(ta + 16, rb);
                        umma::tmem_ld_wait(ra);
                        pp_pack(ra, sbias + l * W + c0, pk);
                        umma::tmem_ld_wait(rb);
                        pp_pack(rb, sbias + l * W + c0 + 16, pk + 8);
                        if (toT) {
                            umma::tmem_st16(tmem + lanes + (uint32_t)(c0 >> 1), pk);
                            umma::tmem_st_wait();
                        } else {
                            const uint32_t rx = (act_row + (uint32_t)((c0 >> 6) * 16384)) ^ swz;
                            const int u0 = (c0 & 63) >> 3;
                            pp_store_smem(rx, u0, pk);
                            pp_store_smem(rx, u0 + 2, pk + 8);
                            umma::fence_async_smem();   // visible to the tensor core
                        }
                    }
                    finish_tile();
                }
            }
            // output layer: this warp's 4 of the 16 output columns
            {
                const int m = r * 256 + (int)rank * 128 + row;
                const int j0 = 4 * cg;
                const float hadd = (cg == 0 && a.add_h && m < a.M) ? __ldg(a.add_h + m) : 0.f;
                wait_tile();
                if (!fail) {
                    uint32_t rr[4];
                    umma::tmem_ld4(tmem + kPPAccCol + (g & 1u) * kPPBN + lanes + (uint32_t)j0, rr);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(rr[0]), "+r"(rr[1]), "+r"(rr[2]), "+r"(rr[3])
                                 :
                                 : "memory");
                    if (m < a.M) {
                        const float *sb = sbias + L * W;
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            const int col = j0 + jj;
                            if (col >= a.nout) break;
                            float qv = (__uint_as_float(rr[jj]) + sb[col]) * __ldg(a.out_std + col) +
                                       __ldg(a.out_mean + col);
                            if (col == 2) qv += hadd;
                            a.out6[(long long)col * a.ld6 + m] = ((a.log_mask >> col) & 1) ? __expf(qv) : qv;
                        }
                    }
                }
                finish_tile();
            }
        }
        if (fail && lane == 0) atomicExch(a.err, 1);
    }
    __syncwarp();
    umma::tc_fence_before();
    __syncthreads();
    umma::cluster_sync();
    if (warp == 1) {
        __syncwarp();
        umma::tc_fence_after();
        umma::tmem_dealloc_pair(tmem, 512);
    }
}

}  // namespace mlp
