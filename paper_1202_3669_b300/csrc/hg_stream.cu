// Streaming content-defined chunking: a stream fed in buffers of any size.
//
// Sec. 3.2.4 ("Content-based Chunking Integration"): written data is
// buffered, each full buffer is chunked on the GPU, its new chunks are
// digested, and when chunk boundaries do not line up with the buffer the
// leftover bytes go to the first chunk of the next buffer. Here each feed is
// appended to the bytes carried from the previous feed (the still-open chunk
// plus the window - 1 bytes before it) in a working buffer; the segment
// pipeline of hg_cdc_hash runs on it with the end of the stream unknown, so it
// finalises only the cuts the data seen so far decides; those chunks are
// digested at once, and a kernel moves the new open chunk to the other working
// buffer. The results equal chunking the concatenated stream in one call.
#include <cstring>
#include <new>

#include "hg_internal.h"

using namespace hg;

struct hg_cdc_stream {
    hg_ctx *ctx = nullptr;
    int algo = HG_MD5;
    hg_cdc_params p{};
    uint64_t max_feed = 0, buf_cap = 0, end_cap = 0, cand_cap = 0, ntiles_cap = 0;
    char *mem = nullptr;
    size_t mem_bytes = 0;
    uint8_t *buf[2] = {};
    int cur = 0;
    uint64_t carry_len = 0;   // bytes at the start of buf[cur] carried from the previous feed
    uint64_t start0 = 0;      // where the open chunk starts in buf[cur]
    uint64_t base = 0;        // stream offset of buf[cur][0]
    uint64_t fed = 0;         // bytes fed so far
    PipeBufs pb{};
    uint64_t *h_info = nullptr;    // pinned: {carry, halo, bytes carried, count} of the last feed
    uint64_t *d_info = nullptr;
    cudaEvent_t done = nullptr, ev_a = nullptr, ev_b = nullptr;
    bool pending = false, closed = false;
    uint64_t last_wl = 0;
};

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Absorb the previous feed's carry: after it completes, the open chunk (and
// its halo) sit at the start of the other working buffer.
static int settle(hg_cdc_stream *st) {
    if (!st->pending) return HG_OK;
    if (cudaEventSynchronize(st->done) != cudaSuccess) return HG_ECUDA;
    const uint64_t carry = st->h_info[0], h = st->h_info[1], moved = st->h_info[2];
    st->base += carry - h;
    st->cur ^= 1;
    st->carry_len = moved;
    st->start0 = h;
    st->pending = false;
    return HG_OK;
}

static int run_feed(hg_cdc_stream *st, uint64_t wl, bool final, uint64_t *d_ends, uint64_t cap,
                    uint64_t *d_count, uint8_t *d_digests, cudaStream_t s) {
    const hg_cdc_params &p = st->p;
    int r;
    if ((r = launch_stream_init(st->pb.st, st->start0, s))) return r;
    const uint64_t ntiles = (wl + kWinTile - 1) / kWinTile;
    PipeBufs pb = st->pb;
    pb.digests = d_digests;
    const uint64_t max_chunks = wl / p.min_chunk + 2;
    if (wl > st->start0) {
        if ((r = launch_pipe_segment(st->buf[st->cur], wl, final ? wl : ~0ull, p, st->algo, 0,
                                     (uint32_t)ntiles, wl, 0, max_chunks, pb, s, s, s, st->ev_a,
                                     st->ev_b, nullptr)))
            return r;
    }
    if ((r = launch_stream_out(pb.ends, pb.st, st->base, d_ends, cap, d_count, s))) return r;
    if (!final) {
        if ((r = launch_stream_carry(st->buf[st->cur], wl, pb.st, p.window - 1, st->buf[st->cur ^ 1],
                                     st->d_info, s)))
            return r;
        if (cudaMemcpyAsync(st->h_info, st->d_info, 4 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaEventRecord(st->done, s) != cudaSuccess)
            return HG_ECUDA;
        st->pending = true;
    }
    return HG_OK;
}

extern "C" {

int hg_stream_open(hg_ctx *ctx, int algo, const hg_cdc_params *p, uint64_t max_feed_bytes,
                   hg_cdc_stream **out) {
    if (!ctx || !p || !out || (algo != HG_MD5 && algo != HG_SHA1) || max_feed_bytes == 0)
        return HG_EINVAL;
    *out = nullptr;
    if ((p->window_hash != HG_WIN_MD5 && p->window_hash != HG_WIN_RABIN) || p->window < 1 ||
        p->window > (p->window_hash == HG_WIN_RABIN ? 64u : 55u) || p->mask_bits < 1 || p->mask_bits > 32 ||
        (p->mask_bits < 32 && (p->magic >> p->mask_bits)) || p->min_chunk < 1 ||
        p->min_chunk > p->max_chunk)
        return HG_EINVAL;
    hg_cdc_stream *st = new (std::nothrow) hg_cdc_stream();
    if (!st) return HG_ENOMEM;
    st->ctx = ctx;
    st->algo = algo;
    st->p = *p;
    st->max_feed = max_feed_bytes;
    // carried bytes stay below max_chunk + window; round the buffer to tiles
    st->buf_cap = ((max_feed_bytes + p->max_chunk + p->window + 2 * kWinTile) / kWinTile) * kWinTile;
    st->ntiles_cap = st->buf_cap / kWinTile;
    st->cand_cap = cand_capacity(st->buf_cap);
    st->end_cap = st->buf_cap / p->min_chunk + 2;
    const size_t sizes[] = {st->buf_cap, st->buf_cap, st->ntiles_cap * kWinThreads * 4,
                            st->ntiles_cap * 4, (st->ntiles_cap + 1) * 8, st->cand_cap * 8,
                            st->end_cap * 8, sizeof(PipeState), 64, 64, kLongListBytes};
    size_t total = 0;
    for (size_t z : sizes) total += a256(z);
    st->mem_bytes = total;
    if (ctx->held + total > ctx->budget) { delete st; return HG_ENOMEM; }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    int rc = HG_OK;
    if (cudaMalloc(&st->mem, total) != cudaSuccess ||
        cudaHostAlloc(&st->h_info, 64, cudaHostAllocDefault) != cudaSuccess ||
        cudaEventCreateWithFlags(&st->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&st->ev_a, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&st->ev_b, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        rc = HG_ENOMEM;
    }
    if (rc == HG_OK) {
        ctx->held += total;
        char *m = st->mem;
        auto take = [&](size_t z) { char *q = m; m += a256(z); return q; };
        st->buf[0] = (uint8_t *)take(sizes[0]);
        st->buf[1] = (uint8_t *)take(sizes[1]);
        st->pb.bitmap = (uint32_t *)take(sizes[2]);
        st->pb.tile_cnt = (uint32_t *)take(sizes[3]);
        st->pb.tile_off = (uint64_t *)take(sizes[4]);
        st->pb.cands = (uint64_t *)take(sizes[5]);
        st->pb.cand_cap = st->cand_cap;
        st->pb.ends = (uint64_t *)take(sizes[6]);
        st->pb.cap = st->end_cap;
        st->pb.st = (PipeState *)take(sizes[7]);
        st->pb.err = (int *)take(sizes[8]);
        st->d_info = (uint64_t *)take(sizes[9]);
        st->pb.long_idx = (uint32_t *)take(sizes[10]);
        st->pb.klong = long_chains(ctx->num_sms);
        if (cudaMemset(st->pb.err, 0, 4) != cudaSuccess) rc = HG_ECUDA;
    }
    cudaSetDevice(prev);
    if (rc != HG_OK) {
        if (st->mem) { cudaFree(st->mem); ctx->held -= total; }
        if (st->h_info) cudaFreeHost(st->h_info);
        if (st->done) cudaEventDestroy(st->done);
        if (st->ev_a) cudaEventDestroy(st->ev_a);
        if (st->ev_b) cudaEventDestroy(st->ev_b);
        delete st;
        return rc;
    }
    *out = st;
    return HG_OK;
}

int hg_stream_feed(hg_cdc_stream *st, const uint8_t *d_data, uint64_t len, uint64_t *d_ends,
                   uint64_t cap, uint64_t *d_count, uint8_t *d_digests, void *stream) {
    if (!st || st->closed || !d_count || (len && !d_data) || !d_ends || !d_digests ||
        (reinterpret_cast<uintptr_t>(d_digests) & 3))
        return HG_EINVAL;
    if (len > st->max_feed) return HG_ECAPACITY;
    if (cap < (st->carry_len + len) / st->p.min_chunk + 1 && cap < st->end_cap) return HG_ECAPACITY;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(st->ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    int r = settle(st);
    if (r == HG_OK && len &&
        cudaMemcpyAsync(st->buf[st->cur] + st->carry_len, d_data, len, cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
        r = HG_ECUDA;
    if (r == HG_OK) {
        const uint64_t wl = st->carry_len + len;
        st->fed += len;
        r = run_feed(st, wl, false, d_ends, cap, d_count, d_digests, s);
    }
    cudaSetDevice(prev);
    return r;
}

int hg_stream_close(hg_cdc_stream *st, uint64_t *d_ends, uint64_t cap, uint64_t *d_count,
                    uint8_t *d_digests, void *stream) {
    if (!st || st->closed || !d_count || !d_ends || !d_digests ||
        (reinterpret_cast<uintptr_t>(d_digests) & 3))
        return HG_EINVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(st->ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    int r = settle(st);
    if (r == HG_OK) r = run_feed(st, st->carry_len, true, d_ends, cap, d_count, d_digests, s);
    if (r == HG_OK) st->closed = true;
    cudaSetDevice(prev);
    return r;
}

int hg_stream_destroy(hg_cdc_stream *st) {
    if (!st) return HG_EINVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(st->ctx->device);
    cudaDeviceSynchronize();
    cudaFree(st->mem);
    st->ctx->held -= st->mem_bytes;
    cudaFreeHost(st->h_info);
    cudaEventDestroy(st->done);
    cudaEventDestroy(st->ev_a);
    cudaEventDestroy(st->ev_b);
    cudaSetDevice(prev);
    delete st;
    return HG_OK;
}

}  // extern "C"
