// C ABI of libhashgpu.so: argument checks, scratch management and launches.
// Every computation is done by the kernels in hg_direct.cu and hg_cdc.cu.
#include <algorithm>
#include <mutex>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "hg_internal.h"

namespace hg {

static int check_params(const hg_cdc_params *p) {
    if (!p || (p->window_hash != HG_WIN_MD5 && p->window_hash != HG_WIN_RABIN)) return HG_EINVAL;
    if (p->window < 1 || p->window > (p->window_hash == HG_WIN_RABIN ? 64u : 55u))
        return HG_EUNSUPPORTED;
    if (p->mask_bits < 1 || p->mask_bits > 32) return HG_EINVAL;
    if (p->mask_bits < 32 && (p->magic >> p->mask_bits) != 0) return HG_EINVAL;
    if (p->min_chunk < 1 || p->min_chunk > p->max_chunk) return HG_EINVAL;
    return HG_OK;
}

int ensure(hg_ctx *ctx, void **p, uint64_t *cap, uint64_t count, size_t elem) {
    if (count <= *cap && *p) return HG_OK;
    uint64_t want = count + count / 4 + 1024;            // grow with headroom
    const size_t old_bytes = (size_t)(*cap) * elem;
    const size_t new_bytes = (size_t)want * elem;
    if (ctx->held - old_bytes + new_bytes > ctx->budget) {
        want = count;
        if (ctx->held - old_bytes + (size_t)want * elem > ctx->budget) return HG_ENOMEM;
    }
    if (*p) {
        cudaError_t e = cudaDeviceSynchronize();         // scratch may be in use by queued work
        if (e != cudaSuccess) return HG_ECUDA;
        cudaFree(*p);
        ctx->held -= old_bytes;
        *p = nullptr;
        *cap = 0;
    }
    void *q = nullptr;
    if (cudaMalloc(&q, (size_t)want * elem) != cudaSuccess) {
        cudaGetLastError();
        return HG_ENOMEM;
    }
    *p = q;
    *cap = want;
    ctx->held += (size_t)want * elem;
    ctx->scratch_gen++;
    return HG_OK;
}

// Scratch for chunking an n-byte input.
static int ensure_cdc(hg_ctx *ctx, uint64_t n) {
    const uint64_t words = (n + 31) / 32, tiles = (n + kWinTile - 1) / kWinTile;
    int r;
    if ((r = ensure(ctx, (void **)&ctx->d_bitmap, &ctx->bitmap_words, words ? words : 1, 4))) return r;
    if ((r = ensure(ctx, (void **)&ctx->d_tile_cnt, &ctx->tile_cap, tiles ? tiles : 1, 4))) return r;
    if ((r = ensure(ctx, (void **)&ctx->d_tile_off, &ctx->tile_off_cap, tiles ? tiles : 1, 8))) return r;
    if ((r = ensure(ctx, (void **)&ctx->d_cands, &ctx->cand_cap, cand_capacity(n), 8))) return r;
    return HG_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace hg

using namespace hg;

extern "C" {

void hg_cdc_default_params(hg_cdc_params *p) {
    if (!p) return;
    p->window = 20;
    p->mask_bits = 13;
    p->magic = 0x0F0F;
    p->window_hash = HG_WIN_MD5;
    p->min_chunk = 2048;
    p->max_chunk = 65536;
}

const char *hg_strerror(int s) {
    switch (s) {
        case HG_OK: return "ok";
        case HG_EINVAL: return "invalid argument";
        case HG_ENOMEM: return "device budget or allocation exhausted";
        case HG_ECAPACITY: return "output capacity too small";
        case HG_ETIMEDOUT: return "bounded device wait timed out";
        case HG_ECUDA: return "CUDA runtime error";
        case HG_EAGAIN: return "not ready";
        case HG_ECANCELED: return "cancelled";
        case HG_EUNSUPPORTED: return "unsupported parameters";
        case HG_EBOUNDS: return "debug bounds check failed";
        default: return "unknown status";
    }
}

int hg_digest_len(int algo) { return algo == HG_MD5 ? 16 : algo == HG_SHA1 ? 20 : HG_EINVAL; }

int hg_host_digest(int algo, const uint8_t *msg, uint64_t n, uint8_t *out) {
    if (hg_digest_len(algo) < 0 || !out || (n && !msg)) return HG_EINVAL;
    host_digest(algo, msg, n, out);
    return HG_OK;
}

int hg_init(hg_ctx **out, int device, size_t budget) {
    if (!out) return HG_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return HG_ECUDA;
    }
    hg_ctx *c = new (std::nothrow) hg_ctx();
    if (!c) return HG_ENOMEM;
    c->device = device;
    c->budget = budget ? budget : ((size_t)32 << 30);
    DeviceGuard g(device);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (rabin_prepare() != HG_OK || cudaMalloc(&c->d_err, 64) != cudaSuccess ||
        cudaMemset(c->d_err, 0, 64) != cudaSuccess) {
        cudaGetLastError();
        if (c->d_err) cudaFree(c->d_err);
        delete c;
        return HG_ECUDA;
    }
    c->d_ncand = reinterpret_cast<uint64_t *>(reinterpret_cast<char *>(c->d_err) + 8);
    c->held = 64;
    *out = c;
    return HG_OK;
}

int hg_destroy(hg_ctx *c) {
    if (!c) return HG_EINVAL;
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    cudaFree(c->d_bitmap);
    cudaFree(c->d_tile_cnt);
    cudaFree(c->d_tile_off);
    cudaFree(c->d_cands);
    cudaFree(c->d_segdig);
    cudaFree(c->d_tasks);
    cudaFree(c->d_err);
    pinned_destroy(c);
    if (c->root_stage) cudaFreeHost(c->root_stage);
    if (c->pipe_ready) {
        if (c->p_exec) cudaGraphExecDestroy(c->p_exec);
        cudaStreamDestroy(c->p_cap);
        cudaFree(c->d_pipe);
        cudaStreamDestroy(c->p_win);
        cudaStreamDestroy(c->p_sel);
        cudaEventDestroy(c->p_fork);
        cudaEventDestroy(c->p_done_sel);
        for (int i = 0; i < kMaxSeg; i++) {
            cudaStreamDestroy(c->p_hash[i]);
            cudaEventDestroy(c->p_join[i]);
            cudaEventDestroy(c->p_ev_win[i]);
            cudaEventDestroy(c->p_ev_copy[i]);
            cudaEventDestroy(c->p_ev_sel[i]);
        }
    }
    delete c;
    return HG_OK;
}

int hg_reserve(hg_ctx *c, uint64_t max_bytes) {
    if (!c) return HG_EINVAL;
    DeviceGuard g(c->device);
    return ensure_cdc(c, max_bytes);
}

uint64_t hg_scratch_bytes(const hg_ctx *c) { return c ? c->held : 0; }

int hg_sync(hg_ctx *c, void *stream) {
    if (!c) return HG_EINVAL;
    DeviceGuard g(c->device);
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return HG_ECUDA;
    }
    int err = 0;
    if (cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return HG_ECUDA;
    if (err) cudaMemset(c->d_err, 0, sizeof(int));
    return err;
}

int hg_hash_blocks(hg_ctx *c, int algo, const uint8_t *d_in, uint64_t n, uint64_t block,
                   uint8_t *d_digests, uint8_t *d_root, void *stream) {
    if (!c || block == 0 || hg_digest_len(algo) < 0) return HG_EINVAL;
    const uint64_t nblk = (n + block - 1) / block;
    if ((n && !d_in) || (nblk && !d_digests)) return HG_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_digests) & 3) || (reinterpret_cast<uintptr_t>(d_root) & 3))
        return HG_EINVAL;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    int r = launch_hash_blocks(algo, d_in, n, block, d_digests, s, c->d_err);
    if (r || !d_root) return r;
    // The hash-of-hashes is one serial chain: on a host core (Sec. 3.2.2 computes
    // it on the CPU) unless the list is tiny or the stream is being captured.
    const uint64_t nbytes = nblk * (uint64_t)hg_digest_len(algo);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusActive;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;
    }
    if (nbytes >= host_root_min_bytes(algo) && cs == cudaStreamCaptureStatusNone)
        return enqueue_host_root(c, algo, d_digests, nbytes, d_root, s);
    return launch_root(algo, d_digests, nbytes, d_root, s);
}

int hg_hash_blocks_pmd(hg_ctx *c, int algo, const uint8_t *d_in, uint64_t n, uint64_t block,
                       uint64_t segment, uint8_t *d_seg_digests, uint8_t *d_ids, void *stream) {
    const int dl = hg_digest_len(algo);
    if (!c || dl < 0 || segment == 0 || block == 0 || block % segment) return HG_EINVAL;
    const uint64_t nblk = (n + block - 1) / block, nseg = (n + segment - 1) / segment;
    if (nblk == 0) return HG_OK;
    if (!d_in || !d_ids || (reinterpret_cast<uintptr_t>(d_ids) & 3) ||
        (reinterpret_cast<uintptr_t>(d_seg_digests) & 15))
        return HG_EINVAL;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    int r;
    uint8_t *seg = d_seg_digests;
    if (!seg) {
        if ((r = ensure(c, (void **)&c->d_segdig, &c->segdig_cap, nseg * (uint64_t)dl, 1))) return r;
        seg = c->d_segdig;
    }
    // level 1: every segment of the input (blocks are whole numbers of
    // segments, so the segment grid of the input is that of every block)
    if ((r = launch_hash_blocks(algo, d_in, n, segment, seg, s, c->d_err))) return r;
    // level 2: block i's identifier digests its (block/segment) segment
    // digests, which sit contiguously; the last block may have fewer
    return launch_hash_blocks(algo, seg, nseg * (uint64_t)dl, (block / segment) * (uint64_t)dl, d_ids,
                              s, c->d_err);
}

int hg_window_bitmap(hg_ctx *c, const uint8_t *d_in, uint64_t n, const hg_cdc_params *p,
                     uint32_t *d_bitmap, void *stream) {
    if (!c) return HG_EINVAL;
    int r = check_params(p);
    if (r) return r;
    if (n == 0) return HG_OK;
    if (!d_in || !d_bitmap || (reinterpret_cast<uintptr_t>(d_bitmap) & 3)) return HG_EINVAL;
    DeviceGuard g(c->device);
    const uint64_t tiles = (n + kWinTile - 1) / kWinTile;
    if ((r = ensure(c, (void **)&c->d_tile_cnt, &c->tile_cap, tiles, 4))) return r;
    return launch_window_bitmap(d_in, n, *p, d_bitmap, c->d_tile_cnt, (cudaStream_t)stream, c->d_err);
}

int hg_cdc_candidates(hg_ctx *c, const uint8_t *d_in, uint64_t n, const hg_cdc_params *p,
                      uint64_t *d_cands, uint64_t cap, uint64_t *d_count, void *stream) {
    if (!c || !d_count || (cap && !d_cands)) return HG_EINVAL;
    int r = check_params(p);
    if (r) return r;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return cuda_status(cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s));
    if (!d_in) return HG_EINVAL;
    if ((r = ensure_cdc(c, n))) return r;
    if ((r = launch_window_bitmap(d_in, n, *p, c->d_bitmap, c->d_tile_cnt, s, c->d_err))) return r;
    const uint64_t tiles = (n + kWinTile - 1) / kWinTile;
    return launch_compact(c->d_bitmap, n, c->d_tile_cnt, c->d_tile_off, tiles, d_cands, cap,
                          d_count, s);
}

int hg_cdc_boundaries(hg_ctx *c, const uint8_t *d_in, uint64_t n, const hg_cdc_params *p,
                      uint64_t *d_ends, uint64_t cap, uint64_t *d_count, void *stream) {
    if (!c || !d_count || (cap && !d_ends)) return HG_EINVAL;
    int r = check_params(p);
    if (r) return r;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return cuda_status(cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s));
    if (!d_in) return HG_EINVAL;
    if ((r = ensure_cdc(c, n))) return r;
    if ((r = launch_window_bitmap(d_in, n, *p, c->d_bitmap, c->d_tile_cnt, s, c->d_err))) return r;
    const uint64_t tiles = (n + kWinTile - 1) / kWinTile;
    if ((r = launch_compact(c->d_bitmap, n, c->d_tile_cnt, c->d_tile_off, tiles, c->d_cands,
                            c->cand_cap, c->d_ncand, s)))
        return r;
    return launch_select(c->d_cands, c->d_ncand, c->cand_cap, c->d_bitmap, n, *p, d_ends, cap,
                         d_count, s);
}

}  // extern "C"

namespace hg {

// One host -> device copy stream per device for the whole process: copies of
// several contexts then queue back to back instead of interleaving (two
// interleaved 64 MiB copies measured 44 GB/s together, one at a time 55 GB/s).
static cudaStream_t shared_copy_stream(int dev) {
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> g(mu);
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        streams[dev] = nullptr;
    }
    return streams[dev];
}

static int pipe_setup(hg_ctx *c) {
    if (c->pipe_ready) return HG_OK;
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    bool ok = cudaStreamCreateWithPriority(&c->p_win, cudaStreamNonBlocking, least) == cudaSuccess &&
              cudaStreamCreateWithFlags(&c->p_cap, cudaStreamNonBlocking) == cudaSuccess &&
              (c->p_copy = shared_copy_stream(c->device)) != nullptr &&
              cudaStreamCreateWithPriority(&c->p_sel, cudaStreamNonBlocking, greatest) == cudaSuccess &&
              cudaEventCreateWithFlags(&c->p_fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&c->p_done_sel, cudaEventDisableTiming) == cudaSuccess &&
              cudaMalloc(&c->d_pipe, sizeof(PipeState) + kLongListBytes) == cudaSuccess;
    for (int i = 0; ok && i < kMaxSeg; i++)   // one digest stream per segment: they never wait on each other
        ok = cudaStreamCreateWithPriority(&c->p_hash[i], cudaStreamNonBlocking, greatest) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->p_join[i], cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; ok && i < kMaxSeg; i++)
        ok = cudaEventCreateWithFlags(&c->p_ev_copy[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->p_ev_win[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->p_ev_sel[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return HG_ECUDA;
    }
    c->held += sizeof(PipeState) + kLongListBytes;
    c->pipe_ready = true;
    return HG_OK;
}

// Segment bounds for chunking n bytes: one segment up to 64 MiB; above that,
// segments of at least 32 MiB (at most 64 of them), each decided and digested
// while the next is window-hashed. Inner bounds are tile multiples.
static std::vector<uint64_t> pipe_bounds(uint64_t n) {
    std::vector<uint64_t> b{0};
    if (n > (64ull << 20)) {
        const uint64_t seg = std::max<uint64_t>(32ull << 20, ((n / 60 + kWinTile - 1) / kWinTile) * kWinTile);
        for (uint64_t x = seg; x + seg / 2 < n; x += seg) b.push_back(x);
    }
    b.push_back(n);
    return b;
}

// Segments when the input still has to cross the host link: 8 MiB pieces
// (at most 60), so window hashing starts after the first piece lands.
static std::vector<uint64_t> pipe_bounds_h2d(uint64_t n) {
    std::vector<uint64_t> b{0};
    const uint64_t seg = std::max<uint64_t>(8ull << 20, ((n / 60 + kWinTile - 1) / kWinTile) * kWinTile);
    for (uint64_t x = seg; x + seg / 4 < n; x += seg) b.push_back(x);
    b.push_back(n);
    return b;
}

}  // namespace hg

extern "C" {

uint32_t hg_cdc_hash_plan(uint64_t n, uint64_t *bounds, uint32_t max) {
    if (n == 0) return 0;
    const std::vector<uint64_t> b = pipe_bounds(n);
    if (bounds)
        for (uint32_t i = 0; i < b.size() && i < max; i++) bounds[i] = b[i];
    return (uint32_t)(b.size() - 1);
}

}  // extern "C"

namespace hg {

// Enqueue the whole pipeline, forked from and joined back into stream s.
static int enqueue_cdc_hash(hg_ctx *c, int algo, const uint8_t *d_in, uint64_t n,
                            const hg_cdc_params *p, uint64_t *d_ends, uint64_t cap,
                            uint64_t *d_count, uint8_t *d_digests, cudaStream_t s,
                            const uint8_t *h_in) {
    const std::vector<uint64_t> b = h_in ? pipe_bounds_h2d(n) : pipe_bounds(n);
    const int nseg = (int)b.size() - 1;
    if (nseg > kMaxSeg) return HG_EUNSUPPORTED;
    PipeBufs pb{c->d_bitmap, c->d_tile_cnt, c->d_tile_off, c->d_cands, c->cand_cap,
                d_ends, cap, d_digests, (PipeState *)c->d_pipe, c->d_err,
                reinterpret_cast<uint32_t *>(static_cast<char *>(c->d_pipe) + sizeof(PipeState)),
                long_chains(c->num_sms), c->d_tasks};
    // Device input in several segments: digests after the last selection, in
    // one length-sorted launch. Per-segment digest launches shared the SMs with
    // the later segments' window kernels (1 GiB: 14.6 ms against 10.8 ms of
    // windows). Host input keeps per-segment digests, which overlap the copies.
    const bool defer = !h_in && nseg > 1;
    int r;
    cudaEventRecord(c->p_fork, s);
    cudaStreamWaitEvent(c->p_win, c->p_fork, 0);
    cudaStreamWaitEvent(c->p_sel, c->p_fork, 0);
    for (int i = 0; i < nseg; i++) cudaStreamWaitEvent(c->p_hash[i], c->p_fork, 0);
    if (cudaMemsetAsync(c->d_pipe, 0, sizeof(PipeState), c->p_sel) != cudaSuccess) return HG_ECUDA;
    if (h_in) {
        // the input crosses the host link in segment pieces, in order, on the copy stream
        cudaStreamWaitEvent(c->p_copy, c->p_fork, 0);
        for (int k = 0; k < nseg; k++) {
            if (cudaMemcpyAsync(const_cast<uint8_t *>(d_in) + b[k], h_in + b[k], b[k + 1] - b[k],
                                cudaMemcpyHostToDevice, c->p_copy) != cudaSuccess)
                return HG_ECUDA;
            cudaEventRecord(c->p_ev_copy[k], c->p_copy);
        }
    }
    for (int k = 0; k < nseg; k++) {
        const uint64_t lo = b[k], hi = b[k + 1];
        const uint32_t t0 = (uint32_t)(lo / kWinTile);
        const uint32_t nt = (uint32_t)((hi + kWinTile - 1) / kWinTile - t0);
        const uint64_t L = (k == nseg - 1) ? n : hi;
        const uint64_t max_chunks = (hi - lo + p->max_chunk) / p->min_chunk + 2;
        if ((r = launch_pipe_segment(d_in, n, n, *p, algo, t0, nt, L, k, max_chunks, pb, c->p_win,
                                     c->p_sel, c->p_hash[k], c->p_ev_win[k], c->p_ev_sel[k],
                                     h_in ? c->p_ev_copy[k] : nullptr, !defer)))
            return r;
    }
    if (defer && (r = launch_hash_sorted(d_in, n, n / p->min_chunk + 2, *p, algo, pb, c->p_sel)))
        return r;
    cudaEventRecord(c->p_done_sel, c->p_sel);
    cudaStreamWaitEvent(s, c->p_done_sel, 0);
    cudaEventRecord(c->p_done_sel, c->p_win);
    cudaStreamWaitEvent(s, c->p_done_sel, 0);
    if (h_in) {
        cudaEventRecord(c->p_done_sel, c->p_copy);
        cudaStreamWaitEvent(s, c->p_done_sel, 0);
    }
    for (int i = 0; i < nseg; i++) {
        cudaEventRecord(c->p_join[i], c->p_hash[i]);
        cudaStreamWaitEvent(s, c->p_join[i], 0);
    }
    return cuda_status(cudaMemcpyAsync(d_count, &((PipeState *)c->d_pipe)->count, sizeof(uint64_t),
                                       cudaMemcpyDeviceToDevice, s));
}

}  // namespace hg

extern "C" {

}  // extern "C"

namespace hg {

static int run_cdc_hash(hg_ctx *c, int algo, const uint8_t *h_in, const uint8_t *d_in, uint64_t n,
                        const hg_cdc_params *p, uint64_t *d_ends, uint64_t cap, uint64_t *d_count,
                        uint8_t *d_digests, void *stream) {
    if (!c || !d_count || hg_digest_len(algo) < 0) return HG_EINVAL;
    int r = check_params(p);
    if (r) return r;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return cuda_status(cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s));
    if (!d_in || !d_ends || !d_digests || (reinterpret_cast<uintptr_t>(d_digests) & 3))
        return HG_EINVAL;
    if (cap < n / p->min_chunk + 1) return HG_ECAPACITY;
    if ((r = ensure_cdc(c, n)) || (r = pipe_setup(c)) ||
        (r = ensure(c, (void **)&c->d_tasks, &c->tasks_cap, n / p->min_chunk + 2, 4)))
        return r;
    // With host input the launches go straight onto the context streams, so the
    // segment copies use the process-wide copy stream and several calls' copies
    // queue instead of interleaving (a replayed graph would pick its own
    // streams). Their host cost hides behind the copies.
    if (h_in) return enqueue_cdc_hash(c, algo, d_in, n, p, d_ends, cap, d_count, d_digests, s, h_in);
    // On device input the pipeline (about five launches per segment) is
    // captured once into a CUDA graph and replayed while its arguments and the
    // scratch stay the same.
    const uint64_t key[16] = {(uint64_t)(uintptr_t)d_in, n, p->window, p->mask_bits, p->magic,
                              p->min_chunk, p->max_chunk, (uint64_t)algo,
                              (uint64_t)(uintptr_t)d_ends, cap, (uint64_t)(uintptr_t)d_count,
                              (uint64_t)(uintptr_t)d_digests, c->scratch_gen,
                              (uint64_t)(uintptr_t)h_in, 1, p->window_hash};
    if (!c->p_exec || std::memcmp(key, c->p_key, sizeof key)) {
        if (c->p_exec) {
            cudaStreamSynchronize(s);
            cudaGraphExecDestroy(c->p_exec);
            c->p_exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(c->p_cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return HG_ECUDA;
        r = enqueue_cdc_hash(c, algo, d_in, n, p, d_ends, cap, d_count, d_digests, c->p_cap, h_in);
        const cudaError_t e = cudaStreamEndCapture(c->p_cap, &graph);
        if (r || e != cudaSuccess) {
            cudaGetLastError();
            if (graph) cudaGraphDestroy(graph);
            return r ? r : HG_ECUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&c->p_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            cudaGetLastError();
            c->p_exec = nullptr;
            return HG_ECUDA;
        }
        std::memcpy(c->p_key, key, sizeof key);
    }
    return cuda_status(cudaGraphLaunch(c->p_exec, s));
}

}  // namespace hg

extern "C" {

int hg_cdc_hash(hg_ctx *c, int algo, const uint8_t *d_in, uint64_t n, const hg_cdc_params *p,
                uint64_t *d_ends, uint64_t cap, uint64_t *d_count, uint8_t *d_digests,
                void *stream) {
    return run_cdc_hash(c, algo, nullptr, d_in, n, p, d_ends, cap, d_count, d_digests, stream);
}

int hg_cdc_hash_h2d(hg_ctx *c, int algo, const uint8_t *h_in, uint8_t *d_in, uint64_t n,
                    const hg_cdc_params *p, uint64_t *d_ends, uint64_t cap, uint64_t *d_count,
                    uint8_t *d_digests, void *stream) {
    if (n && !h_in) return HG_EINVAL;
    return run_cdc_hash(c, algo, h_in, d_in, n, p, d_ends, cap, d_count, d_digests, stream);
}

int hg_hash_chunks(hg_ctx *c, int algo, const uint8_t *d_in, uint64_t n, const uint64_t *d_ends,
                   uint64_t nchunk, const uint64_t *d_count, uint8_t *d_digests, void *stream) {
    if (!c || hg_digest_len(algo) < 0) return HG_EINVAL;
    if (nchunk == 0) return HG_OK;
    if ((n && !d_in) || !d_ends || !d_digests || (reinterpret_cast<uintptr_t>(d_digests) & 3))
        return HG_EINVAL;
    DeviceGuard g(c->device);
    return launch_hash_chunks(algo, d_in, n, d_ends, nchunk, d_count, d_digests,
                              (cudaStream_t)stream, c->d_err);
}

}  // extern "C"
