// Batched content-defined chunking and chunk digests for many files in one pass.
//
// The paper gets its large speed-ups only when many hashing jobs are batched
// (Sec. 3.2.3: a stream of hashing computations; Sec. 4.1: gains need a batch
// of at least three jobs) and it buffers writes so each GPU job covers many
// chunks (Sec. 3.2.4). Here a whole set of files, stored back to back in one
// device buffer, is chunked and hashed by a fixed sequence of launches with no
// host round trip, which is captured once into a CUDA graph:
//   1. a persistent window kernel pulls 8 KiB tiles of the concatenated
//      buffer from an atomic tile counter (the device work queue), prefetching
//      the next tile by bulk async copy while it hashes the current one, and
//      clears the windows that would straddle a file start;
//   2. the candidate bitmap is compacted into one sorted list (all files);
//   3. every file selects its boundaries from its slice of that list: files
//      below a size threshold with one thread each, the others with one CTA
//      each running the parallel exact selection;
//   4. the chunks become a task list with long chunks first;
//   5. a persistent kernel hashes the tasks, warps pulling 32 at a time.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "hg_device.cuh"
#include "hg_internal.h"
#include "hg_select.cuh"
#include "hg_window.cuh"

namespace hg {
namespace {

constexpr uint64_t kBigFileBytes = 1ull << 20;   // files from 1 MiB up get a CTA for selection

// counters in d_words
enum { kNcand = 0, kTotal = 1, kFront = 2, kBack = 3, kTaskCtr = 4, kTileCtr = 5, kNumWords = 8 };

__device__ __forceinline__ uint32_t upper_index(const uint64_t *__restrict__ a, uint32_t lo,
                                                uint32_t hi, uint64_t v) {
    // first i in [lo, hi) with a[i] > v (hi if none); a sorted
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (__ldg(a + mid) > v) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// Persistent window kernel over the concatenation of nfile files.
template <int W>
__global__ void __launch_bounds__(kWinThreads) k_batch_window(
    const uint8_t *__restrict__ in, uint64_t N, const uint64_t *__restrict__ file_off,
    uint32_t nfile, uint32_t wrt, uint32_t mask, uint32_t magic, uint32_t *__restrict__ bitmap,
    uint32_t *__restrict__ tile_cnt, uint32_t ntiles, unsigned long long *tile_ctr, int *err) {
    const uint32_t wlen = W ? (uint32_t)W : wrt;
    __shared__ __align__(128) uint8_t sbuf[2][kSmemBytes];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t s_tile[2];
    __shared__ uint32_t s_frange[2];
    __shared__ uint32_t warp_cnt[kWinThreads / 32];
    const int t = threadIdx.x;
    const bool aligned = (reinterpret_cast<uintptr_t>(in) & 15) == 0;
    auto fast = [&](uint32_t tl) {
        const uint64_t b = (uint64_t)tl * kWinTile;
        return aligned && b >= (uint64_t)kHalo && b + kWinTile <= N;
    };
    if (t == 0) {
        mbar_init(smem_u32(&mbar[0]));
        mbar_init(smem_u32(&mbar[1]));
    }
    __syncthreads();
    if (t == 0) {
        const uint32_t c = (uint32_t)atomicAdd(tile_ctr, 1ull);
        s_tile[0] = c;
        if (c < ntiles && fast(c))
            bulk_load(smem_u32(sbuf[0]), in + (uint64_t)c * kWinTile - kHalo,
                      (uint32_t)(kHalo + kWinTile), smem_u32(&mbar[0]));
    }
    __syncthreads();
    int b = 0;
    uint32_t phase[2] = {0, 0};
    while (true) {
        const uint32_t cur = s_tile[b];
        if (cur >= ntiles) break;
        const uint64_t tile = (uint64_t)cur * kWinTile;
        if (t == 0) {
            const uint32_t nx = (uint32_t)atomicAdd(tile_ctr, 1ull);
            s_tile[b ^ 1] = nx;
            if (nx < ntiles && fast(nx))
                bulk_load(smem_u32(sbuf[b ^ 1]), in + (uint64_t)nx * kWinTile - kHalo,
                          (uint32_t)(kHalo + kWinTile), smem_u32(&mbar[b ^ 1]));
            // files f >= 1 whose start can clear a window end of this tile:
            // starts in [tile + 2 - wlen, tile + kWinTile - 1]
            const uint64_t lo = tile + 2 >= wlen ? tile + 2 - wlen : 0;
            s_frange[0] = lo ? upper_index(file_off, 1, nfile, lo - 1) : 1;
            s_frange[1] = upper_index(file_off, 1, nfile, tile + kWinTile - 1);
        }
        bool timed_out = false;
        if (fast(cur)) {
            timed_out = !mbar_wait(smem_u32(&mbar[b]), phase[b]);
            if (timed_out) atomicCAS(err, 0, (int)HG_ETIMEDOUT);
            phase[b] ^= 1;
        } else {
            for (int i = t; i < kHalo + (int)kWinTile; i += kWinThreads) {
                const int64_t g = (int64_t)tile - kHalo + i;
                sbuf[b][i] = (g >= 0 && (uint64_t)g < N) ? in[g] : (uint8_t)0;
            }
        }
        if (t < 4) reinterpret_cast<uint32_t *>(sbuf[b] + kHalo + kWinTile)[t] = 0;
        if (__syncthreads_or(timed_out)) {
            // bounded drain of the other buffer's copy, then leave
            if (t == 0 && s_tile[b ^ 1] < ntiles && fast(s_tile[b ^ 1]))
                mbar_wait(smem_u32(&mbar[b ^ 1]), phase[b ^ 1]);
            return;
        }
        const uint64_t p0 = tile + 32u * (uint64_t)t;
        uint32_t bits = clip_bits(window_bits32<W>(sbuf[b], t, wlen, mask, magic), p0, wlen, N);
        // a window must lie inside one file: clear ends p in [start, start + wlen - 2]
        for (uint32_t f = s_frange[0]; f < s_frange[1]; f++) {
            const uint64_t st = __ldg(file_off + f);
            const uint64_t a = max(st, p0), e = min(st + wlen - 2, p0 + 31);
            if (wlen >= 2 && a <= e) {
                const uint32_t nb = (uint32_t)(e - a + 1);
                const uint32_t m = (nb >= 32 ? 0xffffffffu : ((1u << nb) - 1u)) << (a - p0);
                bits &= ~m;
            }
        }
        const uint64_t widx = tile / 32 + t;
        if (widx < (N + 31) / 32) bitmap[widx] = bits;
        const uint32_t c = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(bits));
        if ((t & 31) == 0) warp_cnt[t >> 5] = c;
        __syncthreads();
        if (t == 0) {
            uint32_t s = 0;
#pragma unroll
            for (int w = 0; w < kWinThreads / 32; w++) s += warp_cnt[w];
            tile_cnt[cur] = s;
        }
        b ^= 1;
    }
}

// Candidate slice of file f: indices [k0, k1) of cuts in (start, end].
__device__ __forceinline__ void file_slice(const uint64_t *__restrict__ C, uint32_t m,
                                           uint64_t start, uint64_t end, uint32_t &k0,
                                           uint32_t &k1) {
    k0 = upper_index(C, 0, m, start);
    k1 = upper_index(C, k0, m, end);
}

__global__ void k_batch_select_small(const uint32_t *__restrict__ files, uint32_t nsmall,
                                     const uint64_t *__restrict__ file_off,
                                     const uint64_t *__restrict__ slot_off,
                                     const uint64_t *__restrict__ cands, uint64_t cand_cap,
                                     const uint32_t *__restrict__ bitmap, uint64_t mn, uint64_t mx,
                                     uint64_t *__restrict__ ends, uint64_t *__restrict__ counts,
                                     unsigned long long *words) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nsmall) return;
    const uint32_t f = files[i];
    const uint64_t s0 = file_off[f], n = file_off[f + 1];
    const uint64_t so = slot_off[f], cap = slot_off[f + 1] - so;
    const uint64_t ncand = words[kNcand];
    uint64_t idx = 0;
    if (ncand <= cand_cap && ncand < 0xffffffffull) {
        uint32_t k0, k1;
        file_slice(cands, (uint32_t)ncand, s0, n, k0, k1);
        select_thread(cands + k0, k1 - k0, s0, n, mn, mx, WriteEmit{ends + so, cap, &idx, s0});
    } else {
        select_thread_bitmap(bitmap, s0, n, mn, mx, WriteEmit{ends + so, cap, &idx, s0});
    }
    counts[f] = idx;
    atomicAdd(&words[kTotal], (unsigned long long)min(idx, cap));
}

__global__ void __launch_bounds__(kSelThreads) k_batch_select_big(
    const uint32_t *__restrict__ files, const uint64_t *__restrict__ file_off,
    const uint64_t *__restrict__ slot_off, const uint64_t *__restrict__ cands, uint64_t cand_cap,
    const uint32_t *__restrict__ bitmap, uint64_t mn, uint64_t mx, uint64_t *__restrict__ ends,
    uint64_t *__restrict__ counts, unsigned long long *words) {
    __shared__ uint32_t s_k[2];
    const uint32_t f = files[blockIdx.x];
    const uint64_t s0 = file_off[f], n = file_off[f + 1];
    const uint64_t so = slot_off[f], cap = slot_off[f + 1] - so;
    const uint64_t ncand = words[kNcand];
    if (ncand > cand_cap || ncand >= 0xffffffffull) {
        if (threadIdx.x == 0) {
            uint64_t idx = 0;
            select_thread_bitmap(bitmap, s0, n, mn, mx, WriteEmit{ends + so, cap, &idx, s0});
            counts[f] = idx;
            atomicAdd(&words[kTotal], (unsigned long long)min(idx, cap));
        }
        return;
    }
    if (threadIdx.x == 0) {
        uint32_t k0, k1;
        file_slice(cands, (uint32_t)ncand, s0, n, k0, k1);
        s_k[0] = k0;
        s_k[1] = k1;
    }
    __syncthreads();
    const uint32_t k0 = s_k[0], k1 = s_k[1];
    select_block(cands + k0, k1 - k0, s0, n, mn, mx, ends + so, cap, counts + f);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(&words[kTotal], (unsigned long long)min(counts[f], cap));
}

// Task list: long chunks from the front, the rest from the back.
__global__ void k_batch_tasks(const uint64_t *__restrict__ slot_off,
                              const uint64_t *__restrict__ ends, const uint64_t *__restrict__ counts,
                              uint64_t long_bytes, unsigned long long *words,
                              uint64_t *__restrict__ tasks) {
    const uint32_t f = blockIdx.x;
    const uint64_t so = slot_off[f];
    const uint64_t cnt = min(counts[f], slot_off[f + 1] - so);
    const uint64_t total = words[kTotal];
    const int lane = threadIdx.x & 31;
    for (uint64_t r = 0; r < cnt; r += blockDim.x) {
        const uint64_t i = r + threadIdx.x;
        const bool act = i < cnt;
        uint64_t len = 0;
        if (act) len = ends[so + i] - (i ? ends[so + i - 1] : 0);
        const bool lng = act && len >= long_bytes;
        const uint32_t ml = __ballot_sync(0xffffffffu, lng);
        const uint32_t ms = __ballot_sync(0xffffffffu, act && !lng);
        unsigned long long bl = 0, bs = 0;
        if (lane == 0) {
            if (ml) bl = atomicAdd(&words[kFront], (unsigned long long)__popc(ml));
            if (ms) bs = atomicAdd(&words[kBack], (unsigned long long)__popc(ms));
        }
        bl = __shfl_sync(0xffffffffu, bl, 0);
        bs = __shfl_sync(0xffffffffu, bs, 0);
        const uint32_t below = (1u << lane) - 1u;
        if (lng) tasks[bl + __popc(ml & below)] = ((uint64_t)f << 32) | (uint32_t)i;
        else if (act) tasks[total - 1 - (bs + __popc(ms & below))] = ((uint64_t)f << 32) | (uint32_t)i;
    }
}

template <class H>
__global__ void k_batch_hash(const uint8_t *__restrict__ data, const uint64_t *__restrict__ file_off,
                             const uint64_t *__restrict__ slot_off,
                             const uint64_t *__restrict__ ends, const uint64_t *__restrict__ tasks,
                             unsigned long long *words, uint8_t *__restrict__ digests) {
    const int lane = threadIdx.x & 31;
    const uint64_t total = words[kTotal];
    while (true) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&words[kTaskCtr], 32ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= total) break;
        const uint64_t k = base + lane;
        if (k < total) {
            const uint64_t tk = tasks[k];
            const uint32_t f = (uint32_t)(tk >> 32), i = (uint32_t)tk;
            const uint64_t so = slot_off[f];
            const uint64_t lo = i ? ends[so + i - 1] : 0, hi = ends[so + i];
            H hs;
            hash_range(data + file_off[f] + lo, hi - lo, hs);
            store_digest(hs, digests + (so + i) * H::kDigest);
        }
    }
}

template <int W>
void launch_batch_window_t(int grid, const uint8_t *d, uint64_t N, const uint64_t *fo, uint32_t nfile,
                           uint32_t w, uint32_t mask, uint32_t magic, uint32_t *bm, uint32_t *tc,
                           uint32_t ntiles, unsigned long long *ctr, int *err, cudaStream_t s) {
    k_batch_window<W><<<grid, kWinThreads, 0, s>>>(d, N, fo, nfile, w, mask, magic, bm, tc, ntiles,
                                                   ctr, err);
}

int window_occupancy(uint32_t w) {
    int nb = 0;
    switch (w) {
        case 16: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_window<16>, kWinThreads, 0); break;
        case 20: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_window<20>, kWinThreads, 0); break;
        case 24: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_window<24>, kWinThreads, 0); break;
        case 32: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_window<32>, kWinThreads, 0); break;
        case 48: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_window<48>, kWinThreads, 0); break;
        default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_window<0>, kWinThreads, 0);
    }
    return nb > 0 ? nb : 1;
}

}  // namespace
}  // namespace hg

using namespace hg;

struct hg_batch {
    hg_ctx *ctx = nullptr;
    uint32_t nfile = 0;
    uint64_t total = 0, total_slots = 0, ntiles = 0, cand_cap = 0;
    hg_cdc_params p{};
    std::vector<uint64_t> h_file_off, h_slot_off;
    uint32_t nsmall = 0, nbig = 0;
    char *mem = nullptr;
    size_t mem_bytes = 0;
    uint64_t *d_file_off = nullptr, *d_slot_off = nullptr, *d_tile_off = nullptr,
             *d_cands = nullptr, *d_tasks = nullptr;
    uint32_t *d_small = nullptr, *d_big = nullptr, *d_bitmap = nullptr, *d_tile_cnt = nullptr;
    unsigned long long *d_words = nullptr;
    int *d_err = nullptr;
    hg_batch_tuning tune{};
    int win_max_per_sm = 8;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void *g_key[5] = {};
    hg_batch_tuning g_tune{};
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" {

int hg_batch_create(hg_ctx *ctx, const uint64_t *h_file_off, uint32_t nfile,
                    const hg_cdc_params *p, hg_batch **out) {
    if (!ctx || !h_file_off || !p || !out || nfile == 0 || nfile >= (1u << 31)) return HG_EINVAL;
    *out = nullptr;
    if (p->reserved || p->window < 1 || p->window > 55 || p->mask_bits < 1 || p->mask_bits > 32 ||
        (p->mask_bits < 32 && (p->magic >> p->mask_bits)) || p->min_chunk < 1 ||
        p->min_chunk > p->max_chunk)
        return HG_EINVAL;
    if (h_file_off[0] != 0) return HG_EINVAL;
    for (uint32_t f = 0; f < nfile; f++)
        if (h_file_off[f + 1] < h_file_off[f]) return HG_EINVAL;
    hg_batch *b = new (std::nothrow) hg_batch();
    if (!b) return HG_ENOMEM;
    b->ctx = ctx;
    b->nfile = nfile;
    b->p = *p;
    b->total = h_file_off[nfile];
    b->h_file_off.assign(h_file_off, h_file_off + nfile + 1);
    b->h_slot_off.resize(nfile + 1);
    std::vector<uint32_t> small, big;
    uint64_t so = 0;
    for (uint32_t f = 0; f < nfile; f++) {
        const uint64_t sz = h_file_off[f + 1] - h_file_off[f];
        b->h_slot_off[f] = so;
        so += sz ? sz / p->min_chunk + 1 : 0;              // >= chunks the rule can make
        (sz >= kBigFileBytes ? big : small).push_back(f);
    }
    b->h_slot_off[nfile] = so;
    b->total_slots = so;
    b->nsmall = (uint32_t)small.size();
    b->nbig = (uint32_t)big.size();
    b->ntiles = (b->total + kWinTile - 1) / kWinTile;
    b->cand_cap = cand_capacity(b->total);
    if (b->ntiles >= (1ull << 32)) { delete b; return HG_EUNSUPPORTED; }
    // one device allocation, carved
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    const size_t o_fo = take((nfile + 1) * 8), o_so = take((nfile + 1) * 8);
    const size_t o_small = take((size_t)b->nsmall * 4 + 4), o_big = take((size_t)b->nbig * 4 + 4);
    const size_t o_bm = take(((b->total + 31) / 32 + 1) * 4);
    const size_t o_tc = take((b->ntiles + 1) * 4), o_to = take((b->ntiles + 1) * 8);
    const size_t o_c = take(b->cand_cap * 8), o_t = take((b->total_slots + 1) * 8);
    const size_t o_w = take(kNumWords * 8 + 64);
    b->mem_bytes = off;
    if (ctx->held + off > ctx->budget) { delete b; return HG_ENOMEM; }
    int dev = ctx->device, prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(dev);
    int rc = HG_OK;
    if (cudaMalloc(&b->mem, off) != cudaSuccess) { cudaGetLastError(); rc = HG_ENOMEM; }
    if (rc == HG_OK) {
        ctx->held += off;
        b->d_file_off = (uint64_t *)(b->mem + o_fo);
        b->d_slot_off = (uint64_t *)(b->mem + o_so);
        b->d_small = (uint32_t *)(b->mem + o_small);
        b->d_big = (uint32_t *)(b->mem + o_big);
        b->d_bitmap = (uint32_t *)(b->mem + o_bm);
        b->d_tile_cnt = (uint32_t *)(b->mem + o_tc);
        b->d_tile_off = (uint64_t *)(b->mem + o_to);
        b->d_cands = (uint64_t *)(b->mem + o_c);
        b->d_tasks = (uint64_t *)(b->mem + o_t);
        b->d_words = (unsigned long long *)(b->mem + o_w);
        b->d_err = (int *)(b->mem + o_w + kNumWords * 8);
        if (cudaMemcpy(b->d_file_off, h_file_off, (nfile + 1) * 8, cudaMemcpyHostToDevice) ||
            cudaMemcpy(b->d_slot_off, b->h_slot_off.data(), (nfile + 1) * 8, cudaMemcpyHostToDevice) ||
            (b->nsmall && cudaMemcpy(b->d_small, small.data(), b->nsmall * 4, cudaMemcpyHostToDevice)) ||
            (b->nbig && cudaMemcpy(b->d_big, big.data(), b->nbig * 4, cudaMemcpyHostToDevice)) ||
            cudaMemset(b->d_err, 0, 4) ||
            cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking))
            rc = HG_ECUDA;
    }
    if (rc == HG_OK) {
        b->win_max_per_sm = window_occupancy(p->window);
        b->tune.window_ctas_per_sm = b->win_max_per_sm;
        b->tune.hash_threads = 128;
        b->tune.hash_ctas_per_sm = 8;
        b->tune.long_chunk_bytes = 16384;
    }
    cudaSetDevice(prev);
    if (rc != HG_OK) {
        if (b->mem) { cudaFree(b->mem); ctx->held -= off; }
        delete b;
        return rc;
    }
    *out = b;
    return HG_OK;
}

int hg_batch_destroy(hg_batch *b) {
    if (!b) return HG_EINVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->ctx->device);
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->mem) { cudaFree(b->mem); b->ctx->held -= b->mem_bytes; }
    cudaSetDevice(prev);
    delete b;
    return HG_OK;
}

uint64_t hg_batch_slots(const hg_batch *b, uint64_t *h_slot_off) {
    if (!b) return 0;
    if (h_slot_off) std::memcpy(h_slot_off, b->h_slot_off.data(), (b->nfile + 1) * 8);
    return b->total_slots;
}

int hg_batch_get_tuning(const hg_batch *b, hg_batch_tuning *t) {
    if (!b || !t) return HG_EINVAL;
    *t = b->tune;
    return HG_OK;
}

int hg_batch_set_tuning(hg_batch *b, const hg_batch_tuning *t) {
    if (!b || !t || t->window_ctas_per_sm < 1 || t->hash_ctas_per_sm < 1 ||
        (t->hash_threads != 32 && t->hash_threads != 64 && t->hash_threads != 128 &&
         t->hash_threads != 256 && t->hash_threads != 512) || t->long_chunk_bytes == 0)
        return HG_EINVAL;
    b->tune = *t;
    if (b->tune.window_ctas_per_sm > b->win_max_per_sm) b->tune.window_ctas_per_sm = b->win_max_per_sm;
    return HG_OK;
}

int hg_batch_cdc_hash(hg_batch *b, int algo, const uint8_t *d_data, uint64_t *d_ends,
                      uint64_t *d_counts, uint8_t *d_digests, void *stream) {
    if (!b || (algo != HG_MD5 && algo != HG_SHA1)) return HG_EINVAL;
    if ((b->total && !d_data) || !d_counts || (b->total_slots && (!d_ends || !d_digests)) ||
        (reinterpret_cast<uintptr_t>(d_digests) & 3))
        return HG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const hg_cdc_params &p = b->p;
    int sms = b->ctx->num_sms;
    if (cudaMemsetAsync(b->d_words, 0, kNumWords * 8, s) != cudaSuccess ||
        cudaMemsetAsync(d_counts, 0, (size_t)b->nfile * 8, s) != cudaSuccess)
        return HG_ECUDA;
    if (b->ntiles) {
        const uint32_t mask = p.mask_bits >= 32 ? 0xffffffffu : ((1u << p.mask_bits) - 1u);
        const int grid = (int)std::min<uint64_t>(b->ntiles, (uint64_t)sms * b->tune.window_ctas_per_sm);
        unsigned long long *ctr = b->d_words + kTileCtr;
        switch (p.window) {
#define HG_BW(w)                                                                                  \
    case w:                                                                                       \
        launch_batch_window_t<w>(grid, d_data, b->total, b->d_file_off, b->nfile, w, mask, p.magic, \
                                 b->d_bitmap, b->d_tile_cnt, (uint32_t)b->ntiles, ctr, b->d_err, s); \
        break;
            HG_BW(16) HG_BW(20) HG_BW(24) HG_BW(32) HG_BW(48)
#undef HG_BW
            default:
                launch_batch_window_t<0>(grid, d_data, b->total, b->d_file_off, b->nfile, p.window,
                                         mask, p.magic, b->d_bitmap, b->d_tile_cnt,
                                         (uint32_t)b->ntiles, ctr, b->d_err, s);
        }
        int r = launch_compact(b->d_bitmap, b->total, b->d_tile_cnt, b->d_tile_off, b->ntiles,
                               b->d_cands, b->cand_cap, (uint64_t *)(b->d_words + kNcand), s);
        if (r) return r;
    }
    if (b->nsmall)
        k_batch_select_small<<<(b->nsmall + 127) / 128, 128, 0, s>>>(
            b->d_small, b->nsmall, b->d_file_off, b->d_slot_off, b->d_cands, b->cand_cap,
            b->d_bitmap, p.min_chunk, p.max_chunk, d_ends, d_counts, b->d_words);
    if (b->nbig)
        k_batch_select_big<<<b->nbig, kSelThreads, 0, s>>>(
            b->d_big, b->d_file_off, b->d_slot_off, b->d_cands, b->cand_cap, b->d_bitmap,
            p.min_chunk, p.max_chunk, d_ends, d_counts, b->d_words);
    k_batch_tasks<<<b->nfile, 128, 0, s>>>(b->d_slot_off, d_ends, d_counts,
                                           b->tune.long_chunk_bytes, b->d_words, b->d_tasks);
    const int hgrid = sms * b->tune.hash_ctas_per_sm;
    if (algo == HG_MD5)
        k_batch_hash<Md5><<<hgrid, b->tune.hash_threads, 0, s>>>(
            d_data, b->d_file_off, b->d_slot_off, d_ends, b->d_tasks, b->d_words, d_digests);
    else
        k_batch_hash<Sha1><<<hgrid, b->tune.hash_threads, 0, s>>>(
            d_data, b->d_file_off, b->d_slot_off, d_ends, b->d_tasks, b->d_words, d_digests);
    return cuda_status(cudaGetLastError());
}

int hg_batch_cdc_hash_graph(hg_batch *b, int algo, const uint8_t *d_data, uint64_t *d_ends,
                            uint64_t *d_counts, uint8_t *d_digests, void *stream) {
    if (!b) return HG_EINVAL;
    const void *key[5] = {d_data, d_ends, d_counts, d_digests, (const void *)(uintptr_t)(algo + 1)};
    const bool same = b->exec && !std::memcmp(key, b->g_key, sizeof key) &&
                      !std::memcmp(&b->tune, &b->g_tune, sizeof b->tune);
    if (!same) {
        if (b->exec) {
            cudaStreamSynchronize((cudaStream_t)stream);
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return HG_ECUDA;
        int r = hg_batch_cdc_hash(b, algo, d_data, d_ends, d_counts, d_digests, b->cap_stream);
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
        if (r) { if (g) cudaGraphDestroy(g); return r; }
        if (e != cudaSuccess) { cudaGetLastError(); return HG_ECUDA; }
        e = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { cudaGetLastError(); b->exec = nullptr; return HG_ECUDA; }
        std::memcpy(b->g_key, key, sizeof key);
        b->g_tune = b->tune;
    }
    return cuda_status(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
}

int hg_batch_sync(hg_batch *b, void *stream) {
    if (!b) return HG_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return HG_ECUDA;
    }
    int err = 0;
    if (cudaMemcpy(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return HG_ECUDA;
    if (err) cudaMemset(b->d_err, 0, sizeof(int));
    return err;
}

int hg_batch_autotune(hg_batch *b, int algo, const uint8_t *d_data, uint64_t *d_ends,
                      uint64_t *d_counts, uint8_t *d_digests, void *stream, hg_batch_tuning *best) {
    if (!b) return HG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) || cudaEventCreate(&e1)) return HG_ECUDA;
    auto time_it = [&](float *ms) -> int {
        int r = hg_batch_cdc_hash(b, algo, d_data, d_ends, d_counts, d_digests, stream);  // warm
        if (r) return r;
        float acc = 0;
        for (int k = 0; k < 2; k++) {
            cudaEventRecord(e0, s);
            if ((r = hg_batch_cdc_hash(b, algo, d_data, d_ends, d_counts, d_digests, stream))) return r;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) return HG_ECUDA;
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            acc += t;
        }
        *ms = acc / 2;
        return HG_OK;
    };
    hg_batch_tuning cur = b->tune, top = cur;
    float best_ms = 1e30f;
    int rc = HG_OK;
    // window persistence first (the dominant kernel), then the chunk-hash shape
    for (int w : {b->win_max_per_sm, std::max(1, b->win_max_per_sm * 3 / 4), std::max(1, b->win_max_per_sm / 2)}) {
        cur = top;
        cur.window_ctas_per_sm = w;
        b->tune = cur;
        float ms;
        if ((rc = time_it(&ms))) break;
        if (ms < best_ms) { best_ms = ms; top = cur; }
    }
    if (rc == HG_OK) {
        for (int ht : {64, 128, 256})
            for (int hc : {4, 8, 16})
                for (uint64_t lb : {8192ull, 32768ull}) {
                    cur = top;
                    cur.hash_threads = ht;
                    cur.hash_ctas_per_sm = hc;
                    cur.long_chunk_bytes = lb;
                    b->tune = cur;
                    float ms;
                    if ((rc = time_it(&ms))) break;
                    if (ms < best_ms) { best_ms = ms; top = cur; }
                }
    }
    b->tune = top;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best) *best = top;
    return rc;
}

}  // extern "C"
