// Fused inference of the whole surrogate MLP over a chunk of rows in one
// persistent launch: every layer of every 128-row block is a work item, and
// the activations between layers live in rings of row blocks in global memory
// small enough to stay in L2, so that they never travel to DRAM and the
// per-layer launch ramp-up and drain are paid once per chunk.
//
// Items.  A row block r has items (r, l, j) for the hidden layers l < L and
// their N-tiles j (N-tile 256, n_t = W / 256 per layer) and one item (r, L, 0)
// for the output layer (N = 16, 6 used).  Items are numbered slot by slot:
// slot s holds, for every layer l, the items of row block r = s - l D, so a
// layer runs D slots behind the one before it and its inputs were produced
// about D x ips items earlier (ips = L n_t + 1 items per slot, D x ips about
// three rounds of the grid).  CTA c takes items c, c + G, c + 2G, ... (G =
// grid size) in that order; every role of the CTA (TMA producer, MMA issuer,
// epilogue) walks the same sequence.
//
// Rings.  Layer l < L writes its output into ring l (RING row blocks; block r
// uses row block r mod RING), which layer l + 1 reads.  A ring row block lives
// D slots from its write to its read, and is rewritten RING slots after its
// write; RING = 2 D + 4 leaves its readers about three rounds to finish.
//
// Dependencies, through per-(row block, layer) arrival counters in global
// memory: each epilogue warp adds 1 when its part of an item is complete and
// visible (hidden items: after its TMA stores have completed, released at gpu
// scope; output items: once the accumulator has been read).  Item (r, l) may
// start once layer l - 1 of block r has all its arrivals (its input) and, for
// a hidden layer, layer l + 1 of block r - RING has all of its arrivals (the
// readers of the ring row block it is about to overwrite).  Both are items of
// earlier slots.  A dependency warp walks the CTA's items ahead of the TMA
// producer, takes these acquire round trips and the proxy fence, and
// publishes how many items are ready in shared memory, so the producer never
// stalls on a global-memory round trip.  Every wait is bounded and gives up
// early once any CTA has failed.
//
// Progress.  The launch is cooperative (all CTAs resident) and every item
// waits only on strictly earlier items.  An epilogue warp releases a hidden
// item's arrival once its stores have completed: at once, or - to keep the
// store latency off its path - after the accumulator of the CTA's next item is
// ready, but only when that next item depends on nothing at or after the
// released one.  So the earliest unfinished item can always proceed.
#pragma once

#include "mlp_gemm.cuh"

namespace mlp {

constexpr int kFusedMaxLayers = 9;   // up to 8 hidden layers + the output layer
constexpr int kFusedBN = 256;        // N-tile of the hidden layers
constexpr int kFusedOutBN = 16;      // padded output width
constexpr int kFusedEpiWarps = 16;   // four per TMEM lane quarter, 64 columns each
constexpr int kFusedDepWarp = 2 + kFusedEpiWarps;   // after the producer, the MMA issuer and the epilogue
constexpr int kFusedThreads = 64 + 32 * kFusedEpiWarps + 32;
constexpr int kFusedCols = kFusedBN * 4 / kFusedEpiWarps;   // columns of a hidden tile per epilogue warp

struct FusedArgs {
    CUtensorMap tm_x;                     // standardised inputs [rows][64], box 64 x 128
    CUtensorMap tm_ring_ld;               // rings [L][RING * 128][W], box 64 x 128 x 1
    CUtensorMap tm_ring_st;               // the same, box 64 x 32 x 1 (epilogue TMA stores)
    CUtensorMap tm_w[kFusedMaxLayers];    // W_l [out_pad][in_pad]: box 64 x 256 (hidden), 64 x 16 (output)
    const float *bias[kFusedMaxLayers];   // b_l [out_pad]
    int M;                                // rows of the chunk
    int R;                                // row blocks, ceil(M / 128)
    int L;                                // hidden layers
    int W;                                // width, a multiple of 256
    int D;                                // slot lag between consecutive layers
    int ring;                             // row blocks per ring (RING)
    int n_t;                              // N-tiles per hidden layer (W / 256)
    int ips;                              // items per slot, L n_t + 1
    long long total;                      // items, (R + L D) ips
    float *out6;                          // [nout][ld6] physical outputs of the chunk's rows
    long long ld6;
    const float *out_mean, *out_std;      // [nout] de-standardisation
    int nout;                             // outputs in use (<= 16)
    const float *add_h;                   // per-row term added to output 2 (h), or NULL
    int log_mask;                         // bit j set = output j was learned as its logarithm
    uint32_t *done;                       // [R][L + 1] arrival counters, zero at launch
    int *err;                             // set to 1 when a bounded wait runs out
    long long wait_cycles;                // limit of every bounded wait
    int stall_test;                       // test hook: layer 1 of row block 0 waits for one arrival too many
};

// Shared-memory plan.  Single CTAs: stages of a 128 x 64 input tile and a
// 256 x 64 weight tile.  CTA pairs: each CTA's stage holds its 128 input rows
// and half (128 rows) of the weight tile, the pair's MMA reading both CTAs'
// stages; a stage is two thirds the size, so four fit.
template <bool PAIR>
struct FusedCfg {
    static constexpr int A_BYTES = BM * BK * 2;                          // 16 KB
    static constexpr int B_BYTES = (PAIR ? kFusedBN / 2 : kFusedBN) * BK * 2;   // 16 or 32 KB
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int S = PAIR ? 4 : 3;
    static constexpr int STG_BYTES = kFusedEpiWarps * 4096;   // one 32 x 64 BF16 box per epilogue warp
    static constexpr int BAR_BYTES = 256;   // 2 S + 4 mbarriers, the TMEM address, the ready count
    static constexpr uint32_t TMEM_COLS = 2 * kFusedBN;   // two accumulator buffers
    static constexpr int kMaxSmem = 232448;               // 227 KB opt-in per CTA
    static int smem_bytes(int L, int W) { return 1024 + S * STAGE + STG_BYTES + BAR_BYTES + (L * W + 16) * 4; }
};

struct FusedItem {
    bool valid;
    int r, l, j;
};

__device__ __forceinline__ FusedItem fused_item(const FusedArgs &a, long long i)
{
    FusedItem t;
    const long long s = i / a.ips;
    const int k = (int)(i - s * a.ips);
    if (k < a.L * a.n_t) {
        t.l = k / a.n_t;
        t.j = k - t.l * a.n_t;
    } else {
        t.l = a.L;
        t.j = 0;
    }
    const long long r = s - (long long)t.l * a.D;
    t.valid = r >= 0 && r < a.R;
    t.r = (int)r;
    return t;
}

// Largest in-slot index of layer l's items.
__device__ __forceinline__ int fused_kmax(const FusedArgs &a, int l) { return l < a.L ? l * a.n_t + a.n_t - 1 : a.L * a.n_t; }

// Largest item index that item t waits on (-1 if none).
__device__ __forceinline__ long long fused_maxdep(const FusedArgs &a, const FusedItem &t)
{
    long long m = -1;
    if (t.l > 0) m = ((long long)t.r + (long long)(t.l - 1) * a.D) * a.ips + fused_kmax(a, t.l - 1);
    if (t.l < a.L && t.r >= a.ring) {
        const long long d2 = ((long long)(t.r - a.ring) + (long long)(t.l + 1) * a.D) * a.ips + fused_kmax(a, t.l + 1);
        m = d2 > m ? d2 : m;
    }
    return m;
}

// Arrivals that complete layer l of a row block.
__device__ __forceinline__ uint32_t fused_target(const FusedArgs &a, int l)
{
    return (uint32_t)(l < a.L ? kFusedEpiWarps * a.n_t : kFusedEpiWarps);
}

// Wait until *p >= target (acquire, gpu scope); false when ~max_cycles pass
// or another CTA has reported a failure.
__device__ __forceinline__ bool wait_count(const uint32_t *p, uint32_t target, const int *err,
                                           long long max_cycles = 4000000000LL)
{
    if (umma::ld_acquire_gpu(p) >= target) return true;
    const long long t0 = clock64();
    while (true) {
        if (umma::ld_acquire_gpu(p) >= target) return true;
        if (*reinterpret_cast<const volatile int *>(err)) return false;
        const long long dt = clock64() - t0;
        if (dt > max_cycles) return false;
        if (dt > 20000) __nanosleep(64);
    }
}

// Wait until the dependency warp has cleared `n` items (false after
// ~max_cycles, or at once when it reported a failed wait).
__device__ __forceinline__ bool wait_ready(const uint32_t *dep_ready, uint32_t n, long long max_cycles)
{
    uint32_t v = umma::ld_acquire_cta_shared(dep_ready);
    if (v >= n) return v != ~0u;
    const long long t0 = clock64();
    while (true) {
        v = umma::ld_acquire_cta_shared(dep_ready);
        if (v >= n) return v != ~0u;
        const long long dt = clock64() - t0;
        if (dt > max_cycles) return false;
        if (dt > 20000) __nanosleep(32);
    }
}

// One 16-column chunk of a hidden item's epilogue for this lane's row: GeLU of
// accumulator + bias, BF16, into the warp's staging box (chunk c % 4 of it;
// the box must be free again at c % 4 == 0).
__device__ __forceinline__ void hidden_chunk(const uint32_t (&r)[16], const float *sb, uint8_t *stg, int lane, int c)
{
    if ((c & 3) == 0) {
        if (lane == 0) umma::bulk_wait_read0();
        __syncwarp();
    }
    const float4 *b4 = reinterpret_cast<const float4 *>(sb);
    float v[16];
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
        const float4 b = b4[jj];
        const float2 g0 = gelu2(make_float2(__uint_as_float(r[4 * jj]), __uint_as_float(r[4 * jj + 1])),
                                make_float2(b.x, b.y));
        const float2 g1 = gelu2(make_float2(__uint_as_float(r[4 * jj + 2]), __uint_as_float(r[4 * jj + 3])),
                                make_float2(b.z, b.w));
        v[4 * jj] = g0.x;
        v[4 * jj + 1] = g0.y;
        v[4 * jj + 2] = g1.x;
        v[4 * jj + 3] = g1.y;
    }
    stage_row16_bf16(stg, lane, c & 3, v);
}

template <bool PAIR>
__global__ void __launch_bounds__(kFusedThreads, 1) mlp_fused_kernel(const __grid_constant__ FusedArgs a)
{
    using C = FusedCfg<PAIR>;
    constexpr int CT = PAIR ? 2 : 1;   // CTAs per unit of 128 CT rows
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *stg_base = smem + C::S * C::STAGE;
    uint64_t *full = reinterpret_cast<uint64_t *>(stg_base + C::STG_BYTES);
    uint64_t *empty = full + C::S;
    uint64_t *acc_full = empty + C::S;     // [2]
    uint64_t *acc_empty = acc_full + 2;    // [2]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
    uint32_t *dep_ready = tmem_slot + 1;   // items whose dependencies hold; ~0u after a failed wait
    float *sbias = reinterpret_cast<float *>(stg_base + C::STG_BYTES + C::BAR_BYTES);   // [L W + 16]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = a.L, W = a.W;
    const uint32_t rank = PAIR ? umma::cluster_ctarank() : 0u;
    const bool leader = rank == 0;
    const long long g0 = PAIR ? (blockIdx.x >> 1) : blockIdx.x;   // this CTA's (pair's) first item
    const long long gs = PAIR ? (gridDim.x >> 1) : gridDim.x;     // item stride

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::S; ++s) {
            umma::mbar_init(&full[s], 1);
            umma::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            umma::mbar_init(&acc_full[b], 1);
            umma::mbar_init(&acc_empty[b], CT * kFusedEpiWarps);
        }
        *tmem_slot = 0u;
        *dep_ready = 0u;
        umma::fence_mbar_init();
        umma::tma_prefetch_desc(&a.tm_x);
    }
    // biases of every layer, once per CTA
    for (int e = threadIdx.x; e < L * W + kFusedOutBN; e += blockDim.x) {
        const int l = (e < L * W) ? e / W : L;
        const int n = (e < L * W) ? e - l * W : e - L * W;
        sbias[e] = __ldg(a.bias[l] + n);
    }
    __syncthreads();
    if (warp == 1) {
        if constexpr (PAIR) {
            umma::tmem_alloc_pair(tmem_slot, C::TMEM_COLS);
            umma::tmem_relinquish_pair();
        } else {
            umma::tmem_alloc(tmem_slot, C::TMEM_COLS);
            umma::tmem_relinquish();
        }
    }
    umma::tc_fence_before();
    __syncthreads();
    // the peer signals this CTA's barriers: they must be initialised before
    // either CTA of the pair issues a load
    if constexpr (PAIR) umma::cluster_sync();
    umma::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool fail = false;
    const uint32_t *done = a.done;
    uint32_t *done_w = a.done;
    const int stride_l = L + 1;

    if (warp == 0) {
        // ------------------------------------------------------- TMA producer
        if (lane == 0) {
            uint32_t it = 0, nready = 0;
            for (long long i = g0; i < a.total && !fail; i += gs) {
                const FusedItem t = fused_item(a, i);
                if (!t.valid) continue;
                // the dependency warp has acquired this item's inputs (and
                // fenced them for the TMA loads)
                if (!wait_ready(dep_ready, ++nready, a.wait_cycles)) { fail = true; break; }
                const bool out_l = t.l == L;
                const int nkb = (t.l == 0) ? 1 : W / BK;
                const int bn = (out_l ? kFusedOutBN : kFusedBN) / CT;   // weight rows this CTA loads
                const uint32_t bytes = CT * (C::A_BYTES + bn * BK * 2);  // the pair's (or CTA's) stage
                const int unit_blk = (t.l == 0) ? t.r : (t.r % a.ring);
                const int arow = (unit_blk * CT + (int)rank) * BM;
                const int brow = (out_l ? 0 : t.j * kFusedBN) + (int)rank * bn;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % C::S;
                    const uint32_t ph = (it / C::S) & 1u;
                    if (it >= (uint32_t)C::S && !umma::mbar_wait(&empty[s], ph ^ 1u, a.wait_cycles)) {
                        fail = true;
                        break;
                    }
                    uint8_t *st = smem + s * C::STAGE;
                    if (leader) umma::mbar_arrive_expect_tx(&full[s], bytes);
                    if constexpr (PAIR) {
                        // both CTAs' tiles complete on the leader's barrier
                        const uint32_t fb = umma::mapa_shared(umma::smem_u32(&full[s]), 0u);
                        if (t.l == 0)
                            umma::tma_load_2d_pair(st, &a.tm_x, fb, kb * BK, arow);
                        else
                            umma::tma_load_3d_pair(st, &a.tm_ring_ld, fb, kb * BK, arow, t.l - 1);
                        umma::tma_load_2d_pair(st + C::A_BYTES, &a.tm_w[t.l], fb, kb * BK, brow);
                    } else {
                        if (t.l == 0)
                            umma::tma_load_2d(st, &a.tm_x, &full[s], kb * BK, arow);
                        else
                            umma::tma_load_3d(st, &a.tm_ring_ld, &full[s], kb * BK, arow, t.l - 1);
                        umma::tma_load_2d(st + C::A_BYTES, &a.tm_w[t.l], &full[s], kb * BK, brow);
                    }
                }
            }
            if constexpr (PAIR) {
                // the leader's MMAs read this CTA's stages: every use must be
                // released before the CTA may exit
                if (!fail)
                    for (uint32_t k = it; k < it + (uint32_t)C::S; ++k)
                        if (k >= (uint32_t)C::S &&
                            !umma::mbar_wait(&empty[k % C::S], ((k / C::S) & 1u) ^ 1u, 200000000LL)) {
                            fail = true;
                            break;
                        }
            }
            // no copy may still be landing in shared memory when the CTA exits
            // (the peer's copies complete on the leader's barriers)
            if (leader)
                for (uint32_t k = (it > (uint32_t)C::S ? it - C::S : 0u); k < it; ++k)
                    if (!umma::mbar_wait(&full[k % C::S], (k / C::S) & 1u, 200000000LL)) fail = true;
            if (fail) atomicExch(a.err, 1);
        }
    } else if (warp == 1) {
        // -------------------------------------------------------- MMA issuer
        if (lane == 0 && leader) {
            uint32_t it = 0, jacc = 0;
            for (long long i = g0; i < a.total && !fail; i += gs) {
                const FusedItem t = fused_item(a, i);
                if (!t.valid) continue;
                const bool out_l = t.l == L;
                const int nkb = (t.l == 0) ? 1 : W / BK;
                const uint32_t idesc = out_l ? umma::idesc_bf16_f32(CT * BM, kFusedOutBN)
                                             : umma::idesc_bf16_f32(CT * BM, kFusedBN);
                const uint32_t buf = jacc & 1u;
                if (jacc >= 2 && !umma::mbar_wait(&acc_empty[buf], ((jacc >> 1) & 1u) ^ 1u, a.wait_cycles)) {
                    fail = true;
                    break;
                }
                umma::tc_fence_after();
                const uint32_t d_tmem = tmem + buf * kFusedBN;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % C::S;
                    const uint32_t ph = (it / C::S) & 1u;
                    if (!umma::mbar_wait(&full[s], ph, a.wait_cycles)) { fail = true; break; }
                    umma::tc_fence_after();
                    const uint32_t sa = umma::smem_u32(smem + s * C::STAGE);
                    const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k) {
                        if constexpr (PAIR)
                            umma::mma_bf16_pair(d_tmem, umma::sdesc_kmajor_sw128(sa + k * 32),
                                                umma::sdesc_kmajor_sw128(sb + k * 32), idesc, (kb > 0 || k > 0) ? 1u : 0u);
                        else
                            umma::mma_bf16(d_tmem, umma::sdesc_kmajor_sw128(sa + k * 32),
                                           umma::sdesc_kmajor_sw128(sb + k * 32), idesc, (kb > 0 || k > 0) ? 1u : 0u);
                    }
                    if constexpr (PAIR)
                        umma::mma_commit_pair_mc(&empty[s], (uint16_t)0x3);
                    else
                        umma::mma_commit(&empty[s]);
                }
                if (fail) break;
                if constexpr (PAIR)
                    umma::mma_commit_pair_mc(&acc_full[buf], (uint16_t)0x3);
                else
                    umma::mma_commit(&acc_full[buf]);
                ++jacc;
            }
            if (fail) atomicExch(a.err, 1);
        }
    } else if (warp == kFusedDepWarp) {
        // ------------------------------------------------- dependency warp
        if (lane == 0) {
            uint32_t nready = 0;
            for (long long i = g0; i < a.total; i += gs) {
                const FusedItem t = fused_item(a, i);
                if (!t.valid) continue;
                bool ok = true;
                if (t.l > 0)   // the input: layer l - 1 of this unit
                    ok = wait_count(done + (long long)t.r * stride_l + (t.l - 1),
                                    CT * fused_target(a, t.l - 1) + ((a.stall_test && t.r == 0 && t.l == 1) ? 1u : 0u),
                                    a.err, a.wait_cycles);
                if (ok && t.l < L && t.r >= a.ring)   // the ring unit's previous readers
                    ok = wait_count(done + (long long)(t.r - a.ring) * stride_l + (t.l + 1), CT * fused_target(a, t.l + 1),
                                    a.err, a.wait_cycles);
                if (!ok) {
                    umma::st_release_cta_shared(dep_ready, ~0u);
                    atomicExch(a.err, 1);
                    break;
                }
                umma::fence_proxy_async_global();   // the producers' stores, seen by this CTA's TMA loads
                umma::st_release_cta_shared(dep_ready, ++nready);
            }
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const int ew = warp - 2;                   // 0..15
        const int q = warp & 3;                    // TMEM lane quarter this warp may access
        const int hcol = (ew >> 2) * kFusedCols;
        uint8_t *stg = stg_base + ew * 4096;
        uint32_t *pending = nullptr;   // arrival counter of a hidden item whose release is deferred
        uint32_t jacc = 0;
        for (long long i = g0; i < a.total; i += gs) {
            const FusedItem t = fused_item(a, i);
            if (!t.valid) continue;
            const uint32_t buf = jacc & 1u;
            ++jacc;
            // after a timed-out wait this warp skips its work but keeps walking
            // the items (the other warps never wait on it)
            if (!fail && !umma::mbar_wait(&acc_full[buf], ((jacc - 1) >> 1) & 1u, a.wait_cycles)) fail = true;
            fail = __any_sync(0xffffffffu, fail);   // warp-uniform: tcgen05.ld needs the whole warp
            umma::tc_fence_after();
            if (pending) {   // the deferred item's stores have had this item's main loop to land
                if (lane == 0) {
                    umma::bulk_wait0();
                    umma::fence_proxy_async_global();
                    umma::red_release_gpu_add(pending, 1u);
                }
                pending = nullptr;
            }
            const int m0 = (t.r * CT + (int)rank) * BM;
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + buf * kFusedBN;
            // the accumulator buffer is free once every epilogue warp of the
            // pair (or CTA) has read it
            const uint32_t acc_empty_c = PAIR ? umma::mapa_shared(umma::smem_u32(&acc_empty[buf]), 0u) : 0u;
            if (t.l < L) {
                // hidden layer: GeLU(acc + b) -> BF16 -> swizzled box -> TMA store into the ring
                const float *sb = sbias + t.l * W + t.j * kFusedBN + hcol;
                const int ring_row = ((t.r % a.ring) * CT + (int)rank) * BM + q * 32;
                if (!fail) {
                    // 4 chunks of 16 columns; TMEM loads double-buffered in ra / rb
                    uint32_t ra[16], rb[16];
                    umma::tmem_ld16(taddr + hcol, ra);
#pragma unroll 1
                    for (int c = 0; c < kFusedCols / 16; c += 2) {
                        umma::tmem_ld_wait(ra);
                        umma::tmem_ld16(taddr + hcol + (c + 1) * 16, rb);
                        hidden_chunk(ra, sb + c * 16, stg, lane, c);
                        umma::tmem_ld_wait(rb);
                        if (c + 2 < kFusedCols / 16) umma::tmem_ld16(taddr + hcol + (c + 2) * 16, ra);
                        hidden_chunk(rb, sb + (c + 1) * 16, stg, lane, c + 1);
                    }
                    umma::fence_async_smem();   // staging writes visible to the TMA engine
                    __syncwarp();
                    if (lane == 0) {
                        umma::tma_store_3d(&a.tm_ring_st, stg, t.j * kFusedBN + hcol, ring_row, t.l);
                        umma::bulk_commit();
                    }
                }
                umma::tc_fence_before();
                __syncwarp();
                if (lane == 0) {   // the next item's MMAs may start
                    if constexpr (PAIR)
                        umma::mbar_arrive_cluster(acc_empty_c);
                    else
                        umma::mbar_arrive(&acc_empty[buf]);
                }
                // defer the release when the next item waits on nothing at or after this one
                uint32_t *ctr = done_w + (long long)t.r * stride_l + t.l;
                long long nx = i + gs;
                FusedItem tn;
                tn.valid = false;
                for (; nx < a.total; nx += gs) {
                    tn = fused_item(a, nx);
                    if (tn.valid) break;
                }
                if (tn.valid && fused_maxdep(a, tn) < i) {
                    pending = ctr;
                } else if (lane == 0) {
                    umma::bulk_wait0();   // this warp's stores of the item are done
                    umma::fence_proxy_async_global();
                    umma::red_release_gpu_add(ctr, 1u);
                }
            } else {
                // output layer: de-standardise -> physical properties (warps of
                // the first column half; the others only arrive)
                if (!fail && ew < 4) {   // warps 2..5: one per TMEM lane quarter
                    uint32_t rr[16];
                    umma::tmem_ld16(taddr, rr);
                    umma::tmem_ld_wait(rr);
                    const int m = m0 + q * 32 + lane;
                    if (m < a.M) {
                        const float *sb = sbias + L * W;
#pragma unroll
                        for (int jj = 0; jj < 16; ++jj) {
                            if (jj >= a.nout) break;
                            float qv = (__uint_as_float(rr[jj]) + sb[jj]) * __ldg(a.out_std + jj) + __ldg(a.out_mean + jj);
                            if (jj == 2 && a.add_h) qv += __ldg(a.add_h + m);
                            a.out6[(long long)jj * a.ld6 + m] = ((a.log_mask >> jj) & 1) ? __expf(qv) : qv;
                        }
                    }
                }
                umma::tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if constexpr (PAIR)
                        umma::mbar_arrive_cluster(acc_empty_c);
                    else
                        umma::mbar_arrive(&acc_empty[buf]);
                    umma::red_release_gpu_add(done_w + (long long)t.r * stride_l + L, 1u);
                }
            }
        }
        if (pending && lane == 0) {
            umma::bulk_wait0();
            umma::fence_proxy_async_global();
            umma::red_release_gpu_add(pending, 1u);
        }
        if (lane == 0) umma::bulk_wait0();
        if (fail && lane == 0) atomicExch(a.err, 1);
    }
    __syncwarp();
    umma::tc_fence_before();
    __syncthreads();
    // the pair's MMAs, barrier signals and remote arrivals are all done before
    // either CTA frees its tensor memory or exits
    if constexpr (PAIR) umma::cluster_sync();
    if (warp == 1) {
        __syncwarp();
        umma::tc_fence_after();
        if constexpr (PAIR)
            umma::tmem_dealloc_pair(tmem, C::TMEM_COLS);
        else
            umma::tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

}  // namespace mlp
