// Continuous-batching property server.
//
// Clients (simulations) submit requests -- forward properties of a field of
// cells, or T from h -- with FP32 arrays in host memory and a precision.  A
// worker thread:
//   1. admits queued requests in arrival order while their device buffers fit
//      in the HBM budget (a first-fit arena allocated once at creation), and
//      copies their inputs to the device on a copy stream;
//   2. cuts admitted requests into fixed-size chunks and fills batches of up
//      to `max_slots` chunks of one (kind, precision) taken round-robin from
//      every admitted request of that path, so that work of many requests
//      shares each launch and requests that arrive later join the batches
//      still being formed;
//   3. runs each batch by replaying a CUDA graph captured for its path and
//      slot count (bucketed to powers of two): the graph copies the batch's
//      descriptor table (one entry per chunk: request buffers, offset, count)
//      into device memory, gathers the chunks into contiguous staging arrays
//      (FP64 ones for the FP64 paths), runs the surrogate (with its PR
//      fallback) or the PR path on them, and scatters the results back into
//      each request's buffers;
//   4. copies each finished request's outputs back to the host, frees its
//      arena space and records its latency (submit to completion).
// The worker holds the request lock only to take new submissions and to
// publish completions; every CUDA call runs outside it, so serve_submit and
// serve_poll never wait behind a launch.
// Per-row results do not depend on which other rows share a batch, so a
// request's result is the same alone and in the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "pr_internal.h"

namespace {

constexpr int NSP = 9;
constexpr int kNumPrec = 4;                // SV_PREC_SERVER, SV_PREC_FP64, SV_PREC_MIXED, SV_PREC_FP32
constexpr int kNumPaths = 2 * kNumPrec;    // (kind, precision)
constexpr double kRtolFp64 = 1e-12;        // stop tolerance of the FP64 inversion path
constexpr double kRtolFp32 = 1e-6;         // of the FP32 and mixed ones

struct SvSlot {
    const float *T, *p, *Y, *h;   // request inputs (device, arena)
    float *out;                   // props: [6][ld]; T-from-h: T [ld]
    int32_t *status;              // T-from-h status [ld]
    int64_t ld;                   // cells of the request
    int64_t off;                  // first cell of the chunk
    int32_t count;                // cells of the chunk
    int32_t kind;
};

// Gather the batch's chunks into contiguous staging arrays (FP32 request
// data, widened for the FP64 paths).  Rows past a chunk's count get a fixed
// valid state (they are computed and discarded).
template <typename R>
__global__ void gather_kernel(const SvSlot *tab, int nslots, int chunk, int kind, R *T, R *p, R *Y, R *h,
                              int64_t ldst)
{
    const int64_t rows = (int64_t)nslots * chunk;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        const SvSlot s = tab[r / chunk];
        const int64_t o = r % chunk;
        if (o < s.count) {
            const int64_t i = s.off + o;
            T[r] = (R)s.T[i];
            p[r] = (R)s.p[i];
            for (int k = 0; k < NSP; ++k) Y[k * ldst + r] = (R)s.Y[k * s.ld + i];
            if (kind == SV_T_FROM_H) h[r] = (R)s.h[i];
        } else {
            T[r] = R(300);
            p[r] = R(1.0e7);
            for (int k = 0; k < NSP; ++k) Y[k * ldst + r] = (k == 1) ? R(1) : R(0);
            if (kind == SV_T_FROM_H) h[r] = R(0);
        }
    }
}

// Results back into each request's FP32 buffers (rounded from the FP64 paths).
template <typename R>
__global__ void scatter_kernel(const SvSlot *tab, int nslots, int chunk, int kind, const R *out, const int32_t *st,
                               int64_t ldst)
{
    const int64_t rows = (int64_t)nslots * chunk;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        const SvSlot s = tab[r / chunk];
        const int64_t o = r % chunk;
        if (o >= s.count) continue;
        const int64_t i = s.off + o;
        if (kind == SV_PROPS) {
            for (int q = 0; q < 6; ++q) s.out[q * s.ld + i] = (float)out[q * ldst + r];
        } else {
            s.out[i] = (float)out[r];
            s.status[i] = st[r];
        }
    }
}

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with 256-byte granularity.
class Arena {
  public:
    explicit Arena(size_t size) : size_(size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = (bytes + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = (bytes + 255) & ~size_t(255);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

  private:
    size_t size_, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

enum ReqState { kQueued, kAdmitted, kDraining, kDone };

struct Req {
    uint64_t ticket;
    sv_request r;
    double t_submit = 0, t_done = 0;
    // advanced by the worker; kDone (with result and t_done) is published
    // under the server's lock
    std::atomic<int> state{kQueued};
    size_t off = 0, bytes = 0;
    float *dT = nullptr, *dp = nullptr, *dY = nullptr, *dh = nullptr, *dout = nullptr;
    int32_t *dst = nullptr;
    int64_t next = 0;           // next cell to put into a batch
    cudaEvent_t ev_in = nullptr, ev_done = nullptr;
    pr_status result = PR_OK;
};

size_t req_bytes(const sv_request &r)
{
    const size_t n = (size_t)r.n;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    if (r.kind == SV_PROPS) return al(4 * n) * 2 + al(4 * n * NSP) + al(4 * n * 6);
    return al(4 * n) * 4 + al(4 * n * NSP) + al(4 * n);
}

}  // namespace

struct sv_server {
    pr_ctx *ctx;
    sg_model *model;
    sv_config cfg;
    char *arena_base = nullptr;
    Arena *arena = nullptr;                  // worker only
    cudaStream_t s_compute = nullptr, s_copy = nullptr;
    // staging (shared by consecutive batches on the compute stream): FP32
    // and, for the FP64 paths, FP64
    float *stT = nullptr, *stp = nullptr, *stY = nullptr, *sth = nullptr, *stout = nullptr;
    double *sdT = nullptr, *sdp = nullptr, *sdY = nullptr, *sdh = nullptr, *sdout = nullptr;
    int32_t *stst = nullptr, *stit = nullptr;
    int64_t st_rows = 0;
    // double-buffered descriptor tables and their graphs per bucket
    SvSlot *h_tab[2] = {nullptr, nullptr}, *d_tab[2] = {nullptr, nullptr};
    cudaEvent_t tab_free[2] = {nullptr, nullptr};
    cudaEvent_t ev_batch = nullptr;
    int tab_next = 0;
    std::vector<int> buckets;
    std::vector<cudaGraphExec_t> graphs[kNumPaths][2];   // [kind * kNumPrec + precision][table]
    // shared with the callers, under mu
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> queue;                 // submitted, not yet taken by the worker
    std::map<uint64_t, Req *> all;
    uint64_t next_ticket = 1;
    sv_stats stats;
    // worker only
    std::deque<Req *> pending;               // taken from the queue, waiting for admission
    std::vector<Req *> active;
    int rr = 0;
    std::atomic<bool> stop{false};
    std::thread worker;
};

namespace {

// The batch of one path: kind SV_PROPS or SV_T_FROM_H, and the precision
// (SV_PREC_SERVER: the surrogate, or the FP32 PR path without one, for the
// properties; the configured precision for T from h).
pr_status record_batch(sv_server *s, int path, int nslots_bucket, cudaStream_t st, const SvSlot *d_tab)
{
    const int kind = path / kNumPrec, prec = path % kNumPrec;
    const int C = s->cfg.chunk;
    const int64_t rows = (int64_t)nslots_bucket * C, L = s->st_rows;
    const int blocks = (int)std::min<int64_t>((rows + 255) / 256, 4096);
    pr_status e = PR_OK;
    if (prec == SV_PREC_FP64) {
        gather_kernel<double><<<blocks, 256, 0, st>>>(d_tab, nslots_bucket, C, kind, s->sdT, s->sdp, s->sdY, s->sdh, L);
        PR_CUDA_TRY(cudaGetLastError());
        if (kind == SV_PROPS)
            e = pr_props(s->ctx, PR_FP64, rows, s->sdT, s->sdp, s->sdY, L, s->sdout, s->sdout + L, s->sdout + 2 * L,
                         s->sdout + 3 * L, s->sdout + 4 * L, s->sdout + 5 * L, nullptr, st);
        else
            e = pr_T_from_h(s->ctx, PR_FP64, rows, s->sdh, s->sdp, s->sdY, L, s->sdT, s->sdout, s->stst, s->stit, 60,
                            kRtolFp64, st);
        if (e) return e;
        scatter_kernel<double><<<blocks, 256, 0, st>>>(d_tab, nslots_bucket, C, kind, s->sdout, s->stst, L);
        PR_CUDA_TRY(cudaGetLastError());
        return PR_OK;
    }
    gather_kernel<float><<<blocks, 256, 0, st>>>(d_tab, nslots_bucket, C, kind, s->stT, s->stp, s->stY, s->sth, L);
    PR_CUDA_TRY(cudaGetLastError());
    if (kind == SV_PROPS) {
        if (prec == SV_PREC_SERVER && s->model)
            e = surrogate_infer(s->model, rows, s->stT, s->stp, s->stY, L, s->stout, L, nullptr, st);
        else
            e = pr_props(s->ctx, prec == SV_PREC_MIXED ? PR_MIXED : PR_FP32, rows, s->stT, s->stp, s->stY, L,
                         s->stout, s->stout + L, s->stout + 2 * L, s->stout + 3 * L, s->stout + 4 * L, s->stout + 5 * L,
                         nullptr, st);
    } else {
        const pr_precision pp = (prec == SV_PREC_SERVER) ? (pr_precision)s->cfg.newton_precision
                                : (prec == SV_PREC_MIXED) ? PR_MIXED : PR_FP32;
        e = pr_T_from_h(s->ctx, pp, rows, s->sth, s->stp, s->stY, L, s->stT, s->stout, s->stst, s->stit, 60, kRtolFp32,
                        st);
    }
    if (e) return e;
    scatter_kernel<float><<<blocks, 256, 0, st>>>(d_tab, nslots_bucket, C, kind, s->stout, s->stst, L);
    PR_CUDA_TRY(cudaGetLastError());
    return PR_OK;
}

// Capture one graph per (path, table, bucket): H2D of the descriptor table
// followed by the batch's kernels.
pr_status build_graphs(sv_server *s)
{
    for (int kind = 0; kind < kNumPaths; ++kind) {
        for (int t = 0; t < 2; ++t) {
            for (int b : s->buckets) {
                // warm-up run (sets kernel attributes, loads modules) before capturing
                for (int k = 0; k < b; ++k) s->h_tab[t][k] = SvSlot{};
                PR_CUDA_TRY(cudaMemcpyAsync(s->d_tab[t], s->h_tab[t], b * sizeof(SvSlot), cudaMemcpyHostToDevice,
                                            s->s_compute));
                pr_status e = record_batch(s, kind, b, s->s_compute, s->d_tab[t]);
                if (e) return e;
                PR_CUDA_TRY(cudaStreamSynchronize(s->s_compute));
                cudaGraph_t g;
                PR_CUDA_TRY(cudaStreamBeginCapture(s->s_compute, cudaStreamCaptureModeThreadLocal));
                cudaError_t ce = cudaMemcpyAsync(s->d_tab[t], s->h_tab[t], b * sizeof(SvSlot), cudaMemcpyHostToDevice,
                                                 s->s_compute);
                e = (ce == cudaSuccess) ? record_batch(s, kind, b, s->s_compute, s->d_tab[t]) : PR_ECUDA;
                cudaError_t ee = cudaStreamEndCapture(s->s_compute, &g);
                if (e) return e;
                PR_CUDA_TRY(ee);
                cudaGraphExec_t ex;
                PR_CUDA_TRY(cudaGraphInstantiate(&ex, g, 0));
                cudaGraphDestroy(g);
                s->graphs[kind][t].push_back(ex);
            }
        }
    }
    return PR_OK;
}

// Arena space back; the completion itself is published by publish().
void retire(sv_server *s, Req *q, pr_status st, std::vector<std::pair<Req *, pr_status>> &done)
{
    if (q->bytes) s->arena->release(q->off, q->bytes);
    q->bytes = 0;
    done.emplace_back(q, st);
}

// Admit pending requests (arrival order) while they fit in the arena.
void admit(sv_server *s, std::vector<std::pair<Req *, pr_status>> &done)
{
    while (!s->pending.empty()) {
        Req *q = s->pending.front();
        size_t off;
        if (!s->arena->alloc(q->bytes, &off)) {
            if (q->bytes > s->cfg.hbm_budget_bytes) {   // can never fit
                s->pending.pop_front();
                q->bytes = 0;                            // nothing was allocated
                retire(s, q, PR_ENOMEM, done);
                continue;
            }
            break;
        }
        s->pending.pop_front();
        q->off = off;
        const size_t n = (size_t)q->r.n;
        auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
        char *b = s->arena_base + off;
        q->dT = (float *)b; b += al(4 * n);
        q->dp = (float *)b; b += al(4 * n);
        q->dY = (float *)b; b += al(4 * n * NSP);
        if (q->r.kind == SV_PROPS) {
            q->dout = (float *)b;
        } else {
            q->dh = (float *)b; b += al(4 * n);
            q->dout = (float *)b; b += al(4 * n);
            q->dst = (int32_t *)b;
        }
        cudaMemcpyAsync(q->dT, q->r.T, 4 * n, cudaMemcpyHostToDevice, s->s_copy);
        cudaMemcpyAsync(q->dp, q->r.p, 4 * n, cudaMemcpyHostToDevice, s->s_copy);
        cudaMemcpyAsync(q->dY, q->r.Y, 4 * n * NSP, cudaMemcpyHostToDevice, s->s_copy);
        if (q->r.kind == SV_T_FROM_H) cudaMemcpyAsync(q->dh, q->r.h, 4 * n, cudaMemcpyHostToDevice, s->s_copy);
        cudaEventCreateWithFlags(&q->ev_in, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&q->ev_done, cudaEventDisableTiming);
        cudaEventRecord(q->ev_in, s->s_copy);
        q->state.store(kAdmitted);
        s->active.push_back(q);
    }
}

inline int path_of(const Req *q) { return q->r.kind * kNumPrec + q->r.precision; }

// Fill and launch one batch of `path` from the admitted requests; returns
// the slots used (0 when no chunk was ready) and the slots launched.
int launch_batch(sv_server *s, int path, int *launched_slots)
{
    const int C = s->cfg.chunk, S = s->cfg.max_slots;
    const int kind = path / kNumPrec;
    const int t = s->tab_next;
    // the table buffer must not be overwritten before its previous batch read it
    if (cudaEventQuery(s->tab_free[t]) != cudaSuccess) return 0;
    SvSlot *tab = s->h_tab[t];
    std::vector<Req *> used;
    int n = 0;
    const int na = (int)s->active.size();
    // round-robin at chunk granularity: each pass gives every ready request one
    // more chunk, so concurrent requests share the batch
    bool progress = true;
    while (n < S && progress) {
        progress = false;
        for (int k = 0; k < na && n < S; ++k) {
            Req *q = s->active[(s->rr + k) % na];
            if (q->state.load() != kAdmitted || path_of(q) != path || q->next >= q->r.n) continue;
            if (cudaEventQuery(q->ev_in) != cudaSuccess) continue;
            const int cnt = (int)std::min<int64_t>(C, q->r.n - q->next);
            tab[n++] = SvSlot{q->dT, q->dp, q->dY, q->dh, q->dout, q->dst, q->r.n, q->next, cnt, kind};
            q->next += cnt;
            if (std::find(used.begin(), used.end(), q) == used.end()) used.push_back(q);
            progress = true;
        }
    }
    if (n == 0) return 0;
    s->rr = (s->rr + 1) % std::max(1, na);
    size_t bi = 0;
    while (s->buckets[bi] < n) ++bi;
    for (int k = n; k < s->buckets[bi]; ++k) tab[k] = SvSlot{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 1, 0, 0, kind};
    cudaGraphLaunch(s->graphs[path][t][bi], s->s_compute);
    cudaEventRecord(s->tab_free[t], s->s_compute);
    s->tab_next ^= 1;
    *launched_slots = s->buckets[bi];
    cudaEventRecord(s->ev_batch, s->s_compute);
    for (Req *q : used) {
        if (q->next >= q->r.n) {
            // all chunks launched: results back to the host after this batch
            cudaStreamWaitEvent(s->s_copy, s->ev_batch, 0);
            const size_t nn = (size_t)q->r.n;
            if (kind == SV_PROPS) {
                cudaMemcpyAsync(q->r.out, q->dout, 4 * nn * 6, cudaMemcpyDeviceToHost, s->s_copy);
            } else {
                cudaMemcpyAsync(q->r.out, q->dout, 4 * nn, cudaMemcpyDeviceToHost, s->s_copy);
                if (q->r.status) cudaMemcpyAsync(q->r.status, q->dst, 4 * nn, cudaMemcpyDeviceToHost, s->s_copy);
            }
            cudaEventRecord(q->ev_done, s->s_copy);
            q->state.store(kDraining);
        }
    }
    return n;
}

void reap(sv_server *s, std::vector<std::pair<Req *, pr_status>> &done)
{
    for (auto it = s->active.begin(); it != s->active.end();) {
        Req *q = *it;
        if (q->state.load() == kDraining && cudaEventQuery(q->ev_done) == cudaSuccess) {
            cudaEventDestroy(q->ev_in);
            cudaEventDestroy(q->ev_done);
            q->ev_in = q->ev_done = nullptr;
            retire(s, q, PR_OK, done);
            it = s->active.erase(it);
        } else {
            ++it;
        }
    }
}

void worker_main(sv_server *s)
{
    cudaSetDevice(s->ctx->device);
    std::vector<std::pair<Req *, pr_status>> done;
    while (!s->stop.load()) {
        {   // take the new submissions
            std::lock_guard<std::mutex> lk(s->mu);
            while (!s->queue.empty()) {
                s->pending.push_back(s->queue.front());
                s->queue.pop_front();
            }
        }
        done.clear();
        admit(s, done);
        int batches = 0, used = 0, launched_slots = 0;
        for (int path = 0; path < kNumPaths; ++path) {
            int ls = 0;
            const int n = launch_batch(s, path, &ls);
            if (n) {
                ++batches;
                used += n;
                launched_slots += ls;
            }
        }
        reap(s, done);
        {   // publish completions and counters
            std::lock_guard<std::mutex> lk(s->mu);
            const double t = now_ms();
            for (auto &d : done) {
                Req *q = d.first;
                q->result = d.second;
                q->t_done = t;
                q->state.store(kDone);
                s->stats.completed += 1;
                if (d.second == PR_OK) s->stats.cells += q->r.n;
            }
            s->stats.batches += batches;
            s->stats.slots_used += used;
            s->stats.slots_launched += launched_slots;
            s->stats.bytes_in_use = s->arena->used();
            s->stats.peak_bytes_in_use = s->arena->peak();
            s->stats.active = s->active.size() + s->pending.size();
        }
        if (!done.empty()) s->cv_done.notify_all();
        if (!batches) {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->queue.empty() && s->pending.empty() && s->active.empty())
                s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            else {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(50));
            }
        }
    }
}

}  // namespace

extern "C" {

pr_status serve_create(pr_ctx *ctx, sg_model *model, const sv_config *cfg, sv_server **out)
{
    PR_CHECK_ARG(ctx && cfg && out, "serve_create: null argument");
    *out = nullptr;
    PR_CHECK_ARG(ctx->n_species == NSP, "serve_create: the server takes 9-species contexts");
    PR_CHECK_ARG(cfg->chunk >= 128 && cfg->chunk % 128 == 0 && cfg->chunk <= (1 << 22),
                 "serve_create: chunk must be a multiple of 128 in [128, 4194304]");
    PR_CHECK_ARG(cfg->max_slots >= 1 && cfg->max_slots <= 256, "serve_create: max_slots in 1..256");
    PR_CHECK_ARG(cfg->newton_precision == PR_MIXED || cfg->newton_precision == PR_FP32 ||
                     cfg->newton_precision == PR_FP64,
                 "serve_create: newton_precision must be PR_FP64, PR_MIXED or PR_FP32");
    PR_CHECK_ARG(cfg->hbm_budget_bytes >= (size_t)1 << 20, "serve_create: budget below 1 MiB");
    PR_CHECK_ARG(!model || sg_mode_of(model) == SG_MODE_FORWARD, "serve_create: the server takes a forward model");
    sv_server *s = new (std::nothrow) sv_server();
    if (!s) { prgb::set_error("serve_create: host allocation failed"); return PR_ENOMEM; }
    s->ctx = ctx;
    s->model = model;
    s->cfg = *cfg;
    memset(&s->stats, 0, sizeof(s->stats));
    for (int b = 1; b < cfg->max_slots; b *= 2) s->buckets.push_back(b);
    s->buckets.push_back(cfg->max_slots);
    const int64_t rows = (int64_t)cfg->max_slots * cfg->chunk;
    s->st_rows = rows;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->arena_base, cfg->hbm_budget_bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->stT, rows * 4 * (4 + NSP + 6));
    if (e == cudaSuccess) {
        s->stp = s->stT + rows;
        s->sth = s->stp + rows;
        s->stY = s->sth + rows;
        s->stout = s->stY + rows * NSP;
    }
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->sdT, rows * 8 * (4 + NSP + 6));
    if (e == cudaSuccess) {
        s->sdp = s->sdT + rows;
        s->sdh = s->sdp + rows;
        s->sdY = s->sdh + rows;
        s->sdout = s->sdY + rows * NSP;
    }
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->stst, rows * 4 * 2);
    if (e == cudaSuccess) s->stit = s->stst + rows;
    for (int t = 0; t < 2 && e == cudaSuccess; ++t) {
        e = cudaHostAlloc((void **)&s->h_tab[t], cfg->max_slots * sizeof(SvSlot), cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc((void **)&s->d_tab[t], cfg->max_slots * sizeof(SvSlot));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->tab_free[t], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_batch, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_compute, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_copy, cudaStreamNonBlocking);
    pr_status st = PR_OK;
    if (e != cudaSuccess) {
        prgb::set_error("serve_create: %s", cudaGetErrorString(e));
        st = (e == cudaErrorMemoryAllocation) ? PR_ENOMEM : PR_ECUDA;
    }
    if (!st) st = build_graphs(s);
    if (!st) {
        e = cudaStreamSynchronize(s->s_compute);
        if (e != cudaSuccess) { prgb::set_error("serve_create: %s", cudaGetErrorString(e)); st = PR_ECUDA; }
    }
    if (st) {
        serve_destroy(s);
        return st;
    }
    s->arena = new Arena(cfg->hbm_budget_bytes);
    s->worker = std::thread(worker_main, s);
    *out = s;
    return PR_OK;
}

pr_status serve_submit(sv_server *s, const sv_request *req, uint64_t *ticket)
{
    PR_CHECK_ARG(s && req && ticket, "serve_submit: null argument");
    PR_CHECK_ARG(req->kind == SV_PROPS || req->kind == SV_T_FROM_H, "serve_submit: bad kind %d", req->kind);
    PR_CHECK_ARG(req->n >= 1 && req->n <= ((int64_t)1 << 31) - 1, "serve_submit: n out of range");
    PR_CHECK_ARG(req->T && req->p && req->Y && req->out, "serve_submit: null array");
    PR_CHECK_ARG(req->kind == SV_PROPS || req->h, "serve_submit: T-from-h needs h");
    PR_CHECK_ARG(req->precision >= SV_PREC_SERVER && req->precision <= SV_PREC_FP32,
                 "serve_submit: bad precision %d", req->precision);
    Req *q = new (std::nothrow) Req();
    if (!q) { prgb::set_error("serve_submit: host allocation failed"); return PR_ENOMEM; }
    q->r = *req;
    q->bytes = req_bytes(*req);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        q->ticket = s->next_ticket++;
        q->t_submit = now_ms();
        s->queue.push_back(q);
        s->all[q->ticket] = q;
        s->stats.submitted += 1;
        s->stats.queued = s->queue.size();
    }
    s->cv_work.notify_one();
    *ticket = q->ticket;
    return PR_OK;
}

pr_status serve_poll(sv_server *s, uint64_t ticket, int *done, pr_status *result, double *latency_ms)
{
    PR_CHECK_ARG(s && done, "serve_poll: null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    PR_CHECK_ARG(it != s->all.end(), "serve_poll: unknown ticket %llu", (unsigned long long)ticket);
    Req *q = it->second;
    *done = q->state.load() == kDone;
    if (*done) {
        if (result) *result = q->result;
        if (latency_ms) *latency_ms = q->t_done - q->t_submit;
    }
    return PR_OK;
}

pr_status serve_wait(sv_server *s, uint64_t ticket, double timeout_ms, pr_status *result, double *latency_ms)
{
    PR_CHECK_ARG(s, "serve_wait: null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    PR_CHECK_ARG(it != s->all.end(), "serve_wait: unknown ticket %llu", (unsigned long long)ticket);
    Req *q = it->second;
    const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms),
                                        [&] { return q->state.load() == kDone; });
    if (!ok) {
        prgb::set_error("serve_wait: ticket %llu not done after %.1f ms", (unsigned long long)ticket, timeout_ms);
        return PR_ETIMEOUT;
    }
    if (result) *result = q->result;
    if (latency_ms) *latency_ms = q->t_done - q->t_submit;
    return PR_OK;
}

pr_status serve_stats(sv_server *s, sv_stats *out)
{
    PR_CHECK_ARG(s && out, "serve_stats: null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;   // the worker's counters as of its last publication
    out->queued = s->queue.size();
    return PR_OK;
}

void serve_destroy(sv_server *s)
{
    if (!s) return;
    s->stop.store(true);
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    if (s->s_compute) cudaStreamSynchronize(s->s_compute);
    if (s->s_copy) cudaStreamSynchronize(s->s_copy);
    for (auto &kv : s->all) {
        Req *q = kv.second;
        if (q->ev_in) cudaEventDestroy(q->ev_in);
        if (q->ev_done) cudaEventDestroy(q->ev_done);
        delete q;
    }
    for (int k = 0; k < kNumPaths; ++k)
        for (int t = 0; t < 2; ++t)
            for (cudaGraphExec_t g : s->graphs[k][t]) cudaGraphExecDestroy(g);
    for (int t = 0; t < 2; ++t) {
        if (s->h_tab[t]) cudaFreeHost(s->h_tab[t]);
        if (s->d_tab[t]) cudaFree(s->d_tab[t]);
        if (s->tab_free[t]) cudaEventDestroy(s->tab_free[t]);
    }
    if (s->ev_batch) cudaEventDestroy(s->ev_batch);
    if (s->stT) cudaFree(s->stT);
    if (s->sdT) cudaFree(s->sdT);
    if (s->stst) cudaFree(s->stst);
    if (s->arena_base) cudaFree(s->arena_base);
    if (s->s_compute) cudaStreamDestroy(s->s_compute);
    if (s->s_copy) cudaStreamDestroy(s->s_copy);
    delete s->arena;
    delete s;
}

}  // extern "C"
