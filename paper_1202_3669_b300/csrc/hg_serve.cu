// Request server with continuous batching (Sec. 3.2.3, CrystalGPU's job
// management: jobs are submitted to an outstanding queue, a manager thread per
// GPU runs them and notifies completion, buffers are preallocated and reused,
// and transfers overlap computation).
//
// One progress thread owns the GPU side:
//   admission  -- outstanding requests are admitted in arrival order while
//                 their input fits in the device arena (one allocation made
//                 at start, the device budget) and the wave limits allow;
//   staging    -- admitted inputs go host -> device on a copy stream: inputs
//                 in mapped pinned memory up to kGatherMax bytes are pulled by
//                 one gather kernel per wave (a copy call costs ~6 us whatever
//                 its size: the serving mix's inputs up to 512 KiB ran at
//                 26 GB/s as one copy each, 50 GB/s gathered, against 55.7
//                 GB/s for one large copy), larger or unmapped ones by one
//                 copy call each;
//                 the wave's compute waits on the staging in-stream;
//   waves      -- the requests admitted together (until the wave's input
//                 reaches wave_target_bytes) run as one wave: one batched
//                 chunking job (hg_job.cu) for the chunking requests plus the
//                 fixed-block kernels for the block requests, then one copy
//                 of the wave's outputs to pinned host memory;
//   overlap    -- up to max_inflight_waves waves are on the GPU at once, so the
//                 next wave's copies and admission proceed while one computes;
//   completion -- finished waves release their arena ranges and wake pollers.
// Requests arriving while waves run are admitted as soon as memory and a wave
// slot free up: that is the continuous batching.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hg_internal.h"

using namespace hg;

namespace {

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// First-fit range allocator over [0, size) with coalescing, 256-byte granules.
class RangeAlloc {
  public:
    void init(uint64_t size) { free_.clear(); if (size) free_[0] = size; total_ = size; }
    bool alloc(uint64_t bytes, uint64_t *off) {
        bytes = a256(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const uint64_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t bytes) {
        bytes = a256(bytes ? bytes : 1);
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
    uint64_t used() const { return used_; }
    uint64_t total() const { return total_; }

  private:
    std::map<uint64_t, uint64_t> free_;
    uint64_t used_ = 0, total_ = 0;
};

enum State { kQueued, kAdmitted, kDone };

// Inputs up to kGatherMax bytes in mapped pinned host memory are gathered by
// kernel, in pieces of kGatherPiece bytes (one CTA each) so that a large input
// does not leave one CTA streaming it alone; larger or unmapped inputs take
// one copy call each. A copy call costs ~6 us on top of the copy engine's
// 55.7 GB/s, the gather runs at ~50 GB/s with no per-input cost: the two
// break even near 3 MB. Served ceiling on the serving mix with the gather up
// to 0.5 / 2 / 4 / 16 MiB: 50.4 / 51.7 / 51.4 / 46.4 GB/s.
constexpr uint64_t kGatherMax = 2ull << 20;
constexpr uint64_t kGatherPiece = 256ull << 10;

// One input to gather: n bytes from host memory (device-visible address src)
// to the arena (dst, 256-byte aligned, room for n rounded up to 256 bytes).
struct GatherEnt {
    const uint8_t *src;
    uint8_t *dst;
    uint64_t n;
};

// One CTA per input. Each warp covers 32 destination granules of 16 bytes
// (512 bytes) per step: lanes load 32 consecutive aligned 16-byte source
// granules (one coalesced read of host memory over the link) plus the granule
// after them (lane 31), and shift each granule with the next lane's into place,
// so the source may start at any byte. Only aligned granules holding request
// bytes are read (they lie in the pages that hold the request, so they are
// mapped); the last destination granule may carry bytes past n (the arena range
// is rounded up to 256 bytes). Four steps are loaded before they are stored.
// On the serving mix's inputs up to 512 KiB (2368 inputs, 420 MB, any source
// alignment) this runs at 50.2 GB/s against 32.7 GB/s with 4-byte words, 26 GB/s
// with a copy call per input and 55.7 GB/s for one copy of as many bytes.
__global__ void __launch_bounds__(256) k_gather(const GatherEnt *__restrict__ ents) {
    const GatherEnt e = ents[blockIdx.x];
    const uintptr_t s0 = reinterpret_cast<uintptr_t>(e.src);
    const uint32_t sh = (uint32_t)(s0 & 15), q = sh >> 2, r8 = (sh & 3) * 8;
    const uint4 *sg = reinterpret_cast<const uint4 *>(s0 & ~(uintptr_t)15);
    const uint64_t nsg = (s0 + e.n + 15) / 16 - s0 / 16;      // source granules with request bytes
    const uint64_t ndg = (e.n + 15) / 16;                      // destination granules
    uint4 *dg = reinterpret_cast<uint4 *>(e.dst);
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    constexpr int U = 4;
    for (uint64_t base = (uint64_t)warp * 32 * U; base < ndg; base += (uint64_t)nwarps * 32 * U) {
        uint4 v[U], x[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint64_t k = base + (uint64_t)u * 32 + lane;
            v[u] = k < nsg ? sg[k] : make_uint4(0, 0, 0, 0);
            const uint64_t k2 = base + (uint64_t)u * 32 + 32;
            x[u] = (lane == 31 && k2 < nsg) ? sg[k2] : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            uint4 nx;
            nx.x = __shfl_down_sync(0xffffffffu, v[u].x, 1);
            nx.y = __shfl_down_sync(0xffffffffu, v[u].y, 1);
            nx.z = __shfl_down_sync(0xffffffffu, v[u].z, 1);
            nx.w = __shfl_down_sync(0xffffffffu, v[u].w, 1);
            if (lane == 31) nx = x[u];
            // destination words i = source words q + i .. q + i + 1 shifted by r8 bits
            const uint32_t w[8] = {v[u].x, v[u].y, v[u].z, v[u].w, nx.x, nx.y, nx.z, nx.w};
            uint32_t o[5];
#pragma unroll
            for (int i = 0; i < 5; i++)
                o[i] = (q & 2) ? ((q & 1) ? w[i + 3] : w[i + 2]) : ((q & 1) ? w[i + 1] : w[i]);
            const uint64_t k = base + (uint64_t)u * 32 + lane;
            if (k < ndg)
                dg[k] = make_uint4(__funnelshift_r(o[0], o[1], r8), __funnelshift_r(o[1], o[2], r8),
                                   __funnelshift_r(o[2], o[3], r8), __funnelshift_r(o[3], o[4], r8));
        }
    }
}

struct Req {
    uint64_t ticket = 0;
    hg_request rq{};
    State state = kQueued;
    int status = HG_OK;
    uint64_t arena_off = 0, arena_bytes = 0;
    const uint8_t *d_src = nullptr;   // device-visible address of the input (mapped pinned), or null
    uint64_t t_submit = 0, t_admit = 0, t_done = 0;
    // results (host)
    std::vector<uint64_t> ends;
    std::vector<uint8_t> digests;
    uint8_t root[20] = {};
    uint64_t count = 0;
    // placement inside its wave
    uint32_t file = 0;          // CDC: file index in the wave's job
    uint64_t out_off = 0;       // BLOCKS: byte offset of its digests in the wave's block area
};

struct Wave {
    int slot = -1;
    std::vector<std::shared_ptr<Req>> reqs;
    cudaEvent_t done = nullptr;
    JobHost host;
    uint32_t ncdc = 0;
};

// Device + pinned resources of one in-flight wave.
struct WaveSlot {
    char *dmem = nullptr;      // scratch + job arrays + outputs (device)
    char *hmem = nullptr;      // pinned: job arrays in, outputs back
    size_t dbytes = 0, hbytes = 0;
    JobScratch sc{};
    // device arrays
    const uint8_t **d_ptr = nullptr;
    uint64_t *d_len = nullptr, *d_ts = nullptr, *d_so = nullptr;
    uint32_t *d_small = nullptr, *d_big = nullptr;
    uint64_t *d_ends = nullptr, *d_counts = nullptr;
    uint8_t *d_dig = nullptr, *d_blk = nullptr;
    // pinned mirrors (same layout as the contiguous device block from d_ptr on)
    char *h_arrays = nullptr;
    size_t arrays_bytes = 0, out_bytes = 0;
    char *d_arrays = nullptr, *d_out = nullptr, *h_out = nullptr;
    BlkReq *d_blkreq = nullptr, *h_blkreq = nullptr;
    GatherEnt *h_gather = nullptr, *d_gather = nullptr;   // mapped pinned gather list
    cudaStream_t s_cdc = nullptr, s_blk = nullptr;   // this slot's compute streams
    cudaEvent_t ev_staged = nullptr, ev_blk = nullptr;
    bool busy = false;
};

}  // namespace

struct hg_server {
    hg_ctx *ctx = nullptr;
    hg_server_config cfg{};
    char *arena = nullptr;
    RangeAlloc alloc;
    std::vector<WaveSlot> slots;
    uint64_t max_slots_per_wave = 0, max_tiles_per_wave = 0, max_blk_bytes = 0;
    cudaStream_t copy_s = nullptr, comp_s = nullptr;
    JobTuning tune{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Req>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Req>> reqs;
    std::deque<Wave> inflight;
    std::thread th;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::deque<uint64_t> completed;       // tickets finished since the last wait_any
    hg_server_stats stats{};
    int fatal = HG_OK;
};

static uint64_t req_out_bytes(const hg_request &r, uint64_t min_chunk) {
    const int dl = r.algo == HG_MD5 ? 16 : 20;
    if (r.kind == HG_REQ_CDC) return (r.n ? r.n / min_chunk + 1 : 0) * (8 + dl);
    return ((r.n + r.block - 1) / r.block) * dl + 32;
}

static void progress(hg_server *S);

extern "C" {

void hg_server_default_config(hg_server_config *c) {
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    c->device_budget = 32ull << 30;
    c->max_wave_bytes = 1ull << 30;
    c->max_wave_requests = 4096;
    c->max_inflight_waves = 3;
    hg_cdc_default_params(&c->cdc);
    c->wave_target_bytes = 256ull << 20;
}

int hg_server_create(hg_ctx *ctx, const hg_server_config *cfg, hg_server **out) {
    if (!ctx || !cfg || !out) return HG_EINVAL;
    *out = nullptr;
    const hg_cdc_params &p = cfg->cdc;
    if ((p.window_hash != HG_WIN_MD5 && p.window_hash != HG_WIN_RABIN) || p.window < 1 ||
        p.window > (p.window_hash == HG_WIN_RABIN ? 64u : 55u) || p.mask_bits < 1 ||
        p.mask_bits > 32 ||
        (p.mask_bits < 32 && (p.magic >> p.mask_bits)) || p.min_chunk < 1 || p.min_chunk > p.max_chunk ||
        cfg->max_wave_bytes == 0 || cfg->max_wave_requests == 0 || cfg->max_inflight_waves == 0 ||
        cfg->max_inflight_waves > 8 || cfg->device_budget < cfg->max_wave_bytes)
        return HG_EINVAL;
    hg_server *S = new (std::nothrow) hg_server();
    if (!S) return HG_ENOMEM;
    S->ctx = ctx;
    S->cfg = *cfg;
    const uint64_t W = cfg->max_wave_bytes, R = cfg->max_wave_requests;
    S->max_tiles_per_wave = W / kWinTile + R;
    S->max_slots_per_wave = W / p.min_chunk + R;
    S->max_blk_bytes = W / 2 + R * 32;              // block digests of one wave
    const uint64_t cand_cap = cand_capacity(W) + R;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    int rc = HG_OK;
    S->slots.resize(cfg->max_inflight_waves);
    size_t slot_dev_total = 0;
    for (auto &ws : S->slots) {
        ws.arrays_bytes = a256(R * 8) * 2 + a256((R + 1) * 8) * 2 + a256(R * 4 + 4) * 2 +
                          a256(R * sizeof(BlkReq));
        ws.out_bytes = a256(S->max_slots_per_wave * 8) + a256(R * 8) +
                       a256(S->max_slots_per_wave * 36) + a256(S->max_blk_bytes);
        const size_t scratch = job_scratch_bytes(S->max_tiles_per_wave, cand_cap, S->max_slots_per_wave);
        ws.dbytes = scratch + ws.arrays_bytes + ws.out_bytes;
        ws.hbytes = ws.arrays_bytes + ws.out_bytes;
        slot_dev_total += ws.dbytes;
    }
    if (cfg->device_budget <= slot_dev_total + W) rc = HG_ENOMEM;
    const uint64_t arena_bytes = rc == HG_OK ? cfg->device_budget - slot_dev_total : 0;
    if (rc == HG_OK && ctx->held + cfg->device_budget > ctx->budget) rc = HG_ENOMEM;
    if (rc == HG_OK && cudaMalloc(&S->arena, arena_bytes) != cudaSuccess) { cudaGetLastError(); rc = HG_ENOMEM; }
    for (auto &ws : S->slots) {
        if (rc != HG_OK) break;
        if (cudaMalloc(&ws.dmem, ws.dbytes) != cudaSuccess ||
            cudaHostAlloc(&ws.hmem, ws.hbytes, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc(&ws.h_gather, (R + W / kGatherPiece + 1) * sizeof(GatherEnt),
                          cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer((void **)&ws.d_gather, ws.h_gather, 0) != cudaSuccess) {
            cudaGetLastError();
            rc = HG_ENOMEM;
            break;
        }
        job_scratch_carve(ws.dmem, S->max_tiles_per_wave, cand_cap, S->max_slots_per_wave, &ws.sc);
        const size_t scratch = job_scratch_bytes(S->max_tiles_per_wave, cand_cap, S->max_slots_per_wave);
        ws.d_arrays = ws.dmem + scratch;
        ws.d_out = ws.d_arrays + ws.arrays_bytes;
        ws.h_arrays = ws.hmem;
        ws.h_out = ws.hmem + ws.arrays_bytes;
        char *m = ws.d_arrays;
        ws.d_ptr = (const uint8_t **)m;  m += a256(R * 8);
        ws.d_len = (uint64_t *)m;        m += a256(R * 8);
        ws.d_ts = (uint64_t *)m;         m += a256((R + 1) * 8);
        ws.d_so = (uint64_t *)m;         m += a256((R + 1) * 8);
        ws.d_small = (uint32_t *)m;      m += a256(R * 4 + 4);
        ws.d_big = (uint32_t *)m;        m += a256(R * 4 + 4);
        ws.d_blkreq = (BlkReq *)m;
        ws.h_blkreq = (BlkReq *)(ws.h_arrays + (m - ws.d_arrays));
        m = ws.d_out;
        ws.d_ends = (uint64_t *)m;       m += a256(S->max_slots_per_wave * 8);
        ws.d_counts = (uint64_t *)m;     m += a256(R * 8);
        ws.d_dig = (uint8_t *)m;         m += a256(S->max_slots_per_wave * 36);
        ws.d_blk = (uint8_t *)m;
        if (cudaMemset(ws.sc.err, 0, 4) != cudaSuccess ||
            cudaStreamCreateWithFlags(&ws.s_cdc, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&ws.s_blk, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ws.ev_staged, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ws.ev_blk, cudaEventDisableTiming) != cudaSuccess)
            rc = HG_ECUDA;
    }
    if (rc == HG_OK && (cudaStreamCreateWithFlags(&S->copy_s, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaStreamCreateWithFlags(&S->comp_s, cudaStreamNonBlocking) != cudaSuccess))
        rc = HG_ECUDA;
    if (rc == HG_OK) {
        S->alloc.init(arena_bytes);
        ctx->held += cfg->device_budget;
        S->tune = JobTuning{0, 32, 8, 16384};       // one-warp window span CTAs
        S->th = std::thread(progress, S);
    }
    cudaSetDevice(prev);
    if (rc != HG_OK) {
        for (auto &ws : S->slots) {
            if (ws.dmem) cudaFree(ws.dmem);
            if (ws.hmem) cudaFreeHost(ws.hmem);
            if (ws.h_gather) cudaFreeHost(ws.h_gather);
            if (ws.s_cdc) cudaStreamDestroy(ws.s_cdc);
            if (ws.s_blk) cudaStreamDestroy(ws.s_blk);
            if (ws.ev_staged) cudaEventDestroy(ws.ev_staged);
            if (ws.ev_blk) cudaEventDestroy(ws.ev_blk);
        }
        if (S->arena) cudaFree(S->arena);
        if (S->copy_s) cudaStreamDestroy(S->copy_s);
        if (S->comp_s) cudaStreamDestroy(S->comp_s);
        delete S;
        return rc;
    }
    *out = S;
    return HG_OK;
}

int hg_server_destroy(hg_server *S) {
    if (!S) return HG_EINVAL;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->ctx->device);
    cudaDeviceSynchronize();
    for (auto &w : S->inflight)
        if (w.done) cudaEventDestroy(w.done);
    for (auto &ws : S->slots) {
        if (ws.dmem) cudaFree(ws.dmem);
        if (ws.hmem) cudaFreeHost(ws.hmem);
        if (ws.h_gather) cudaFreeHost(ws.h_gather);
        if (ws.s_cdc) cudaStreamDestroy(ws.s_cdc);
        if (ws.s_blk) cudaStreamDestroy(ws.s_blk);
        if (ws.ev_staged) cudaEventDestroy(ws.ev_staged);
        if (ws.ev_blk) cudaEventDestroy(ws.ev_blk);
    }
    if (S->arena) cudaFree(S->arena);
    cudaStreamDestroy(S->copy_s);
    cudaStreamDestroy(S->comp_s);
    S->ctx->held -= S->cfg.device_budget;
    cudaSetDevice(prev);
    delete S;
    return HG_OK;
}

int hg_submit(hg_server *S, const hg_request *r, uint64_t *ticket) {
    if (!S || !r || !ticket) return HG_EINVAL;
    if ((r->kind != HG_REQ_CDC && r->kind != HG_REQ_BLOCKS) || (r->algo != HG_MD5 && r->algo != HG_SHA1) ||
        (r->n && !r->h_data) || (r->kind == HG_REQ_BLOCKS && r->block == 0))
        return HG_EINVAL;
    // a request must fit one wave and the arena on its own
    if (r->n > S->cfg.max_wave_bytes || a256(r->n) > S->alloc.total() ||
        req_out_bytes(*r, S->cfg.cdc.min_chunk) > (r->kind == HG_REQ_CDC ? S->max_slots_per_wave * 28 : S->max_blk_bytes))
        return HG_ENOMEM;
    auto q = std::make_shared<Req>();
    q->rq = *r;
    q->t_submit = now_ns();
    if (r->n && r->n <= kGatherMax) {
        // gather by kernel only from pinned host memory the server's device has mapped
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, r->h_data) == cudaSuccess && a.type == cudaMemoryTypeHost &&
            a.devicePointer && a.device == S->ctx->device)
            q->d_src = static_cast<const uint8_t *>(a.devicePointer);
        else
            cudaGetLastError();
    }
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->fatal) return S->fatal;
        q->ticket = S->next_ticket++;
        S->queue.push_back(q);
        S->reqs[q->ticket] = q;
        S->stats.submitted++;
    }
    S->cv_work.notify_one();
    *ticket = q->ticket;
    return HG_OK;
}

int hg_cancel(hg_server *S, uint64_t ticket) {
    if (!S) return HG_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return HG_EINVAL;
    auto &q = it->second;
    if (q->state != kQueued) return HG_EAGAIN;                  // already admitted or done
    for (auto qi = S->queue.begin(); qi != S->queue.end(); ++qi)
        if ((*qi)->ticket == ticket) { S->queue.erase(qi); break; }
    q->state = kDone;
    q->status = HG_ECANCELED;
    q->t_done = now_ns();
    S->stats.cancelled++;
    S->completed.push_back(ticket);
    S->cv_done.notify_all();
    return HG_OK;
}

int hg_poll(hg_server *S, uint64_t ticket, hg_result *res, int64_t timeout_us) {
    if (!S || !res) return HG_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return HG_EINVAL;
    std::shared_ptr<Req> q = it->second;
    auto ready = [&] { return q->state == kDone || S->fatal; };
    if (!ready()) {
        if (timeout_us < 0) S->cv_done.wait(lk, ready);
        else if (timeout_us > 0) S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    }
    if (q->state != kDone) return S->fatal ? S->fatal : HG_EAGAIN;
    std::memset(res, 0, sizeof *res);
    res->status = q->status;
    res->algo = q->rq.algo;
    res->count = q->count;
    res->ends = q->ends.empty() ? nullptr : q->ends.data();
    res->digests = q->digests.empty() ? nullptr : q->digests.data();
    std::memcpy(res->root, q->root, 20);
    res->t_submit_ns = q->t_submit;
    res->t_admit_ns = q->t_admit;
    res->t_done_ns = q->t_done;
    return HG_OK;
}

int hg_release(hg_server *S, uint64_t ticket) {
    if (!S) return HG_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return HG_EINVAL;
    if (it->second->state != kDone) return HG_EAGAIN;
    S->reqs.erase(it);
    return HG_OK;
}

int hg_server_wait_any(hg_server *S, uint64_t *tickets, uint32_t max, int64_t timeout_us,
                       uint32_t *n_out) {
    if (!S || !n_out || (max && !tickets)) return HG_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto ready = [&] { return !S->completed.empty() || S->fatal; };
    if (!ready()) {
        if (timeout_us < 0) S->cv_done.wait(lk, ready);
        else if (timeout_us > 0) S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    }
    uint32_t n = 0;
    while (n < max && !S->completed.empty()) {
        tickets[n++] = S->completed.front();
        S->completed.pop_front();
    }
    *n_out = n;
    return S->fatal ? S->fatal : HG_OK;
}

int hg_server_get_stats(hg_server *S, hg_server_stats *st) {
    if (!S || !st) return HG_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    *st = S->stats;
    st->arena_used = S->alloc.used();
    st->arena_bytes = S->alloc.total();
    st->queued = S->queue.size();
    return HG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- progress thread ----------
static int launch_wave(hg_server *S, Wave &w) {
    WaveSlot &ws = S->slots[w.slot];
    const hg_cdc_params &p = S->cfg.cdc;
    // inputs: small mapped ones gathered by one kernel, the others one copy each,
    // all on the copy stream
    uint32_t ng = 0;
    for (auto &q : w.reqs)
        if (q->rq.n && q->d_src)
            for (uint64_t o = 0; o < q->rq.n; o += kGatherPiece)
                ws.h_gather[ng++] = GatherEnt{q->d_src + o, (uint8_t *)S->arena + q->arena_off + o,
                                              std::min(kGatherPiece, q->rq.n - o)};
    if (ng) {
        k_gather<<<ng, 256, 0, S->copy_s>>>(ws.d_gather);
        if (cudaGetLastError() != cudaSuccess) return HG_ECUDA;
    }
    for (auto &q : w.reqs)
        if (q->rq.n && !q->d_src &&
            cudaMemcpyAsync(S->arena + q->arena_off, q->rq.h_data, q->rq.n, cudaMemcpyHostToDevice,
                            S->copy_s) != cudaSuccess)
            return HG_ECUDA;
    cudaStream_t cs = ws.s_cdc, bs = ws.s_blk;
    cudaEventRecord(ws.ev_staged, S->copy_s);
    cudaStreamWaitEvent(cs, ws.ev_staged, 0);
    cudaStreamWaitEvent(bs, ws.ev_staged, 0);
    // chunking requests -> one job
    std::vector<uint64_t> lens;
    std::vector<const uint8_t *> ptrs;
    uint64_t blk_off = 0, nblk_total = 0;
    uint32_t nblkreq = 0;
    for (auto &q : w.reqs) {
        if (q->rq.kind == HG_REQ_CDC) {
            q->file = (uint32_t)lens.size();
            lens.push_back(q->rq.n);
            ptrs.push_back((const uint8_t *)S->arena + q->arena_off);
        } else {
            q->out_off = blk_off;
            const uint64_t nb = (q->rq.n + q->rq.block - 1) / q->rq.block;
            ws.h_blkreq[nblkreq++] = BlkReq{(const uint8_t *)S->arena + q->arena_off, q->rq.n,
                                             q->rq.block, nblk_total, (uint8_t *)ws.d_blk + blk_off,
                                             q->rq.algo, q->rq.want_root};
            nblk_total += nb;
            blk_off += a256(req_out_bytes(q->rq, p.min_chunk));
        }
    }
    w.ncdc = (uint32_t)lens.size();
    int rc = HG_OK;
    if (w.ncdc) {
        job_plan(lens.data(), w.ncdc, p.min_chunk, &w.host);
        const uint32_t nf = w.ncdc;
        char *h = ws.h_arrays;
        const size_t R = S->cfg.max_wave_requests;
        std::memcpy(h, ptrs.data(), nf * 8);
        std::memcpy(h + a256(R * 8), lens.data(), nf * 8);
        std::memcpy(h + a256(R * 8) * 2, w.host.tile_start.data(), (nf + 1) * 8);
        std::memcpy(h + a256(R * 8) * 2 + a256((R + 1) * 8), w.host.slot_off.data(), (nf + 1) * 8);
        char *hs = h + a256(R * 8) * 2 + a256((R + 1) * 8) * 2;
        if (!w.host.small.empty()) std::memcpy(hs, w.host.small.data(), w.host.small.size() * 4);
        if (!w.host.big.empty()) std::memcpy(hs + a256(R * 4 + 4), w.host.big.data(), w.host.big.size() * 4);
        if (cudaMemcpyAsync(ws.d_arrays, ws.h_arrays, (char *)ws.d_blkreq - ws.d_arrays,
                            cudaMemcpyHostToDevice, cs) != cudaSuccess)
            return HG_ECUDA;
        JobDev j{nullptr, nullptr, ws.d_ptr, ws.d_len, ws.d_ts, ws.d_so, ws.d_small, ws.d_big, nf,
                 (uint32_t)w.host.small.size(), (uint32_t)w.host.big.size(), (uint32_t)w.host.ntiles};
        // one job per digest algorithm present in the wave
        bool has[2] = {false, false};
        for (auto &q : w.reqs)
            if (q->rq.kind == HG_REQ_CDC) has[q->rq.algo] = true;
        for (int algo = 0; algo < 2 && rc == HG_OK; algo++) {
            if (!has[algo]) continue;
            // the first job computes boundaries for all files; a second algorithm
            // recomputes them (same result) and only its digests are used
            rc = enqueue_cdc_job(j, ws.sc, p, algo, S->tune, S->ctx->num_sms, ws.d_ends,
                                 ws.d_counts, algo == HG_MD5 ? ws.d_dig : ws.d_dig + S->max_slots_per_wave * 16,
                                 cs);
        }
        if (rc) return rc;
    }
    if (nblkreq) {
        // all block requests of the wave in one launch (plus one for their roots),
        // on the slot's second stream so they overlap the chunking job
        if (cudaMemcpyAsync(ws.d_blkreq, ws.h_blkreq, nblkreq * sizeof(BlkReq),
                            cudaMemcpyHostToDevice, bs) != cudaSuccess)
            return HG_ECUDA;
        if ((rc = launch_multi_blocks(ws.d_blkreq, nblkreq, nblk_total, bs))) return rc;
    }
    cudaEventRecord(ws.ev_blk, bs);
    cudaStreamWaitEvent(cs, ws.ev_blk, 0);
    // outputs back: only the used part of each region
    const uint64_t MS = S->max_slots_per_wave, R = S->cfg.max_wave_requests;
    const size_t o_counts = a256(MS * 8), o_dig = o_counts + a256(R * 8), o_blk = o_dig + a256(MS * 36);
    auto back = [&](size_t off, size_t bytes) {
        return bytes == 0 || cudaMemcpyAsync(ws.h_out + off, ws.d_out + off, bytes,
                                             cudaMemcpyDeviceToHost, cs) == cudaSuccess;
    };
    bool ok = true;
    if (w.ncdc) {
        const uint64_t ts = w.host.total_slots;
        bool has[2] = {false, false};
        for (auto &q : w.reqs)
            if (q->rq.kind == HG_REQ_CDC) has[q->rq.algo] = true;
        ok = back(0, ts * 8) && back(o_counts, (size_t)w.ncdc * 8) &&
             (!has[HG_MD5] || back(o_dig, ts * 16)) && (!has[HG_SHA1] || back(o_dig + MS * 16, ts * 20));
    }
    if (ok && blk_off) ok = back(o_blk, blk_off);
    if (!ok) return HG_ECUDA;
    if (cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming) != cudaSuccess) return HG_ECUDA;
    return cuda_status(cudaEventRecord(w.done, cs));
}

static void finish_wave(hg_server *S, Wave &w) {
    WaveSlot &ws = S->slots[w.slot];
    const uint64_t t = now_ns();
    const char *ho = ws.h_out;
    const uint64_t MS = S->max_slots_per_wave;
    const uint64_t *h_ends = (const uint64_t *)ho;
    const uint64_t *h_counts = (const uint64_t *)(ho + a256(MS * 8));
    const uint8_t *h_dig = (const uint8_t *)(ho + a256(MS * 8) + a256(S->cfg.max_wave_requests * 8));
    const uint8_t *h_blk = h_dig + a256(MS * 36);
    std::lock_guard<std::mutex> g(S->mu);
    for (auto &q : w.reqs) {
        const int dl = q->rq.algo == HG_MD5 ? 16 : 20;
        if (q->rq.kind == HG_REQ_CDC) {
            const uint64_t so = w.host.slot_off[q->file];
            const uint64_t cap = w.host.slot_off[q->file + 1] - so;
            const uint64_t k = std::min(h_counts[q->file], cap);
            q->count = k;
            q->ends.assign(h_ends + so, h_ends + so + k);
            const uint8_t *d = q->rq.algo == HG_MD5 ? h_dig : h_dig + MS * 16;
            q->digests.assign(d + so * dl, d + (so + k) * dl);
        } else {
            const uint64_t nblk = (q->rq.n + q->rq.block - 1) / q->rq.block;
            const uint8_t *d = h_blk + q->out_off;
            q->count = nblk;
            q->digests.assign(d, d + nblk * dl);
            if (q->rq.want_root) std::memcpy(q->root, d + nblk * dl, dl);
        }
        S->alloc.release(q->arena_off, q->arena_bytes);
        q->state = kDone;
        q->status = HG_OK;
        q->t_done = t;
        S->completed.push_back(q->ticket);
        S->stats.completed++;
        S->stats.bytes_done += q->rq.n;
    }
    S->stats.waves++;
    ws.busy = false;
    cudaEventDestroy(w.done);
    w.done = nullptr;
}

static void progress(hg_server *S) {
    cudaSetDevice(S->ctx->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        // completions (waves on different slots may finish in any order)
        bool progressed = false;
        for (size_t i = 0; i < S->inflight.size();) {
            Wave &w = S->inflight[i];
            const cudaError_t e = cudaEventQuery(w.done);
            if (e == cudaErrorNotReady) { i++; continue; }
            if (e != cudaSuccess) { S->fatal = HG_ECUDA; break; }
            lk.unlock();
            int err = 0;
            cudaMemcpy(&err, S->slots[w.slot].sc.err, sizeof(int), cudaMemcpyDeviceToHost);
            lk.lock();
            if (err) S->fatal = err;
            lk.unlock();
            finish_wave(S, w);
            lk.lock();
            S->inflight.erase(S->inflight.begin() + i);
            progressed = true;
        }
        if (progressed) S->cv_done.notify_all();
        if (S->fatal) {
            S->cv_done.notify_all();
            break;
        }
        if (S->stop) {
            // stopping: cancel what never got admitted, finish what is on the GPU
            for (auto &q : S->queue) {
                q->state = kDone;
                q->status = HG_ECANCELED;
                q->t_done = now_ns();
                S->completed.push_back(q->ticket);
                S->stats.cancelled++;
            }
            S->queue.clear();
            S->cv_done.notify_all();
            if (S->inflight.empty()) break;
        }
        // admission into a free wave slot
        int slot = -1;
        for (int i = 0; i < (int)S->slots.size(); i++)
            if (!S->slots[i].busy) { slot = i; break; }
        if (slot >= 0 && !S->queue.empty()) {
            Wave w;
            w.slot = slot;
            uint64_t bytes = 0, blk = 0, slots_used = 0;
            const hg_cdc_params &p = S->cfg.cdc;
            const uint64_t wave_target = S->cfg.wave_target_bytes ? S->cfg.wave_target_bytes
                                                                  : S->cfg.max_wave_bytes;
            while (!S->queue.empty() && w.reqs.size() < S->cfg.max_wave_requests) {
                auto &q = S->queue.front();
                const uint64_t ob = req_out_bytes(q->rq, p.min_chunk);
                const bool cdc = q->rq.kind == HG_REQ_CDC;
                const uint64_t ns = cdc ? (q->rq.n ? q->rq.n / p.min_chunk + 1 : 0) : 0;
                if (bytes + q->rq.n > S->cfg.max_wave_bytes) break;
                if (!w.reqs.empty() && bytes + q->rq.n > wave_target) break;
                if (!cdc && blk + a256(ob) > S->max_blk_bytes) break;
                if (cdc && slots_used + ns > S->max_slots_per_wave) break;
                uint64_t off;
                if (!S->alloc.alloc(q->rq.n, &off)) break;              // wait for memory
                q->arena_off = off;
                q->arena_bytes = q->rq.n;
                q->state = kAdmitted;
                q->t_admit = now_ns();
                bytes += q->rq.n;
                if (cdc) slots_used += ns; else blk += a256(ob);
                w.reqs.push_back(q);
                S->queue.pop_front();
            }
            if (!w.reqs.empty()) {
                S->slots[slot].busy = true;
                lk.unlock();
                const int rc = launch_wave(S, w);
                lk.lock();
                if (rc) { S->fatal = rc; continue; }
                S->inflight.push_back(std::move(w));
                continue;
            }
        }
        // nothing to launch: wait briefly for an arrival or a completion
        S->cv_work.wait_for(lk, std::chrono::microseconds(S->inflight.empty() ? 200 : 20));
    }
}

// ---------------------------------------------------------------- trace replay -------------
extern "C" int hg_server_replay(hg_server *S, const hg_request *reqs, const uint64_t *arrival_ns,
                                uint32_t nreq, uint64_t *latency_ns, uint64_t *span_ns) {
    if (!S || (nreq && (!reqs || !arrival_ns || !latency_ns))) return HG_EINVAL;
    std::vector<uint64_t> tickets(nreq, 0);
    std::unordered_map<uint64_t, uint32_t> index;
    index.reserve(nreq * 2 + 1);
    const uint64_t t0 = now_ns();
    uint32_t next = 0, done = 0;
    std::vector<uint64_t> got(1024);
    int rc = HG_OK;
    while (done < nreq && rc == HG_OK) {
        const uint64_t t = now_ns() - t0;
        while (next < nreq && arrival_ns[next] <= t) {
            uint64_t tk = 0;
            if ((rc = hg_submit(S, &reqs[next], &tk))) break;
            tickets[next] = tk;
            index[tk] = next;
            next++;
        }
        if (rc) break;
        const int64_t wait_us = next < nreq ? (int64_t)std::min<uint64_t>(
                                                  200, (arrival_ns[next] > t ? arrival_ns[next] - t : 0) / 1000)
                                            : 1000;
        uint32_t n = 0;
        if ((rc = hg_server_wait_any(S, got.data(), (uint32_t)got.size(), wait_us, &n))) break;
        for (uint32_t k = 0; k < n; k++) {
            auto it = index.find(got[k]);
            if (it == index.end()) continue;
            hg_result r;
            if (hg_poll(S, got[k], &r, 0) == HG_OK) {
                latency_ns[it->second] = r.t_done_ns - (t0 + arrival_ns[it->second]);
                if (r.status) rc = r.status;
            }
            hg_release(S, got[k]);
            done++;
        }
    }
    if (span_ns) *span_ns = now_ns() - t0;
    return rc;
}
