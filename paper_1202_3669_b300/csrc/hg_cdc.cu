// Content-defined chunking kernels: compaction, selection, segment digests.
//
// Sec. 2.1 ("Content-based chunking") and Sec. 3.2.2: a small window is hashed
// with MD5 at every byte offset, independently per window, and a boundary is
// declared where the hash matches a predefined value. The paper leaves the
// boundary scan to the CPU because it could not synchronise all GPU threads;
// here the scan is done on the device by compaction and a selection kernel.
#include "hg_device.cuh"
#include "hg_internal.h"
#include "hg_select.cuh"

namespace hg {
namespace {

// Exclusive scan of the per-tile candidate counts, one CTA.
__global__ void __launch_bounds__(1024) k_scan_tiles(const uint32_t *__restrict__ cnt,
                                                     uint64_t ntiles, uint64_t *__restrict__ off,
                                                     uint64_t *__restrict__ total) {
    __shared__ uint64_t warp_sum[32];
    const int t = threadIdx.x;
    const uint64_t per = (ntiles + 1023) / 1024;
    const uint64_t a = min(ntiles, per * t), b = min(ntiles, per * (t + 1));
    uint64_t s = 0;
    for (uint64_t i = a; i < b; i++) s += cnt[i];
    // block-wide exclusive scan of s
    uint64_t x = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, d);
        if ((t & 31) >= d) x += y;
    }
    if ((t & 31) == 31) warp_sum[t >> 5] = x;
    __syncthreads();
    if (t < 32) {
        uint64_t w = warp_sum[t];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, w, d);
            if (t >= d) w += y;
        }
        warp_sum[t] = w;                                 // inclusive over warps
    }
    __syncthreads();
    uint64_t run = x - s + ((t >> 5) ? warp_sum[(t >> 5) - 1] : 0);
    for (uint64_t i = a; i < b; i++) {
        off[i] = run;
        run += cnt[i];
    }
    if (t == 1023) *total = run;
}

// Exclusive scan of the counts of tiles [0, ntiles) of a segment, added to the
// running candidate count *total (read first, updated at the end), one CTA.
__global__ void __launch_bounds__(1024) k_scan_tiles_base(const uint32_t *__restrict__ cnt,
                                                          uint64_t ntiles, uint64_t *__restrict__ off,
                                                          uint64_t *total) {
    __shared__ uint64_t warp_sum[32];
    __shared__ uint64_t s_base;
    const int t = threadIdx.x;
    if (t == 0) s_base = *total;
    const uint64_t per = (ntiles + 1023) / 1024;
    const uint64_t a = min(ntiles, per * t), b = min(ntiles, per * (t + 1));
    uint64_t s = 0;
    for (uint64_t i = a; i < b; i++) s += cnt[i];
    uint64_t x = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, d);
        if ((t & 31) >= d) x += y;
    }
    if ((t & 31) == 31) warp_sum[t >> 5] = x;
    __syncthreads();
    if (t < 32) {
        uint64_t w = warp_sum[t];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, w, d);
            if (t >= d) w += y;
        }
        warp_sum[t] = w;
    }
    __syncthreads();
    uint64_t run = s_base + x - s + ((t >> 5) ? warp_sum[(t >> 5) - 1] : 0);
    for (uint64_t i = a; i < b; i++) {
        off[i] = run;
        run += cnt[i];
    }
    if (t == 1023) *total = run;
}

// Bitmap -> increasing cut positions. One CTA per window tile; tiles without
// candidates leave at once.
__global__ void __launch_bounds__(kWinThreads) k_compact(const uint32_t *__restrict__ bitmap,
                                                         uint64_t nwords,
                                                         const uint32_t *__restrict__ tile_cnt,
                                                         const uint64_t *__restrict__ tile_off,
                                                         uint64_t *__restrict__ cands,
                                                         uint64_t cap, uint32_t tile0) {
    __shared__ uint32_t warp_sum[kWinThreads / 32];
    const uint32_t tix = blockIdx.x + tile0;
    if (tile_cnt[tix] == 0) return;
    const int t = threadIdx.x;
    const uint64_t widx = (uint64_t)tix * kWinThreads + t;
    uint32_t w = widx < nwords ? bitmap[widx] : 0u;
    const uint32_t c = __popc(w);
    uint32_t x = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if ((t & 31) >= d) x += y;
    }
    if ((t & 31) == 31) warp_sum[t >> 5] = x;
    __syncthreads();
    uint32_t before = x - c;
    for (int k = 0; k < (t >> 5); k++) before += warp_sum[k];
    uint64_t idx = tile_off[tix] + before;
    const uint64_t pos0 = widx * 32;
    while (w) {
        const int b = __ffs(w) - 1;
        w &= w - 1;
        if (idx < cap && HG_DOK(pos0 + b < nwords * 32, nullptr))
            cands[idx] = pos0 + b + 1;                  // cut after the window's last byte
        idx++;
    }
}

// First candidate cut c with lo <= c <= hi (and c <= n), from the bitmap:
// window end p = c - 1. One warp; returns UINT64_MAX when there is none.
__device__ uint64_t first_cut_bitmap(const uint32_t *__restrict__ bitmap, uint64_t n, uint64_t lo,
                                     uint64_t hi) {
    const int lane = threadIdx.x & 31;
    if (hi > n) hi = n;
    if (lo < 1) lo = 1;
    if (lo > hi) return UINT64_MAX;
    const uint64_t plo = lo - 1, phi = hi - 1;        // window ends, inclusive
    for (uint64_t wb = plo / 32; wb <= phi / 32; wb += 32) {
        const uint64_t wi = wb + lane;
        uint32_t w = 0;
        if (wi <= phi / 32) {
            w = bitmap[wi];
            if (wi == plo / 32) w &= ~0u << (plo % 32);
            if (wi == phi / 32 && (phi % 32) != 31) w &= (1u << (phi % 32 + 1)) - 1u;
        }
        const uint32_t any = __ballot_sync(0xffffffffu, w != 0);
        if (any) {
            const int src = __ffs(any) - 1;
            const uint32_t ws = __shfl_sync(0xffffffffu, w, src);
            return (wb + src) * 32 + (__ffs(ws) - 1) + 1;
        }
    }
    return UINT64_MAX;
}

// Greedy min/max selection by one warp, walking the chain chunk by chunk. It
// reads the sorted candidate list 32 at a time, or scans the bitmap when the
// list overflowed its capacity. Serial: used only for that overflow case.
__device__ void select_serial(const uint64_t *__restrict__ cands, uint64_t ncand, bool use_list,
                              const uint32_t *__restrict__ bitmap, uint64_t n, uint64_t mn,
                              uint64_t mx, uint64_t *__restrict__ ends, uint64_t cap,
                              uint64_t *__restrict__ d_count) {
    const int lane = threadIdx.x & 31;
    uint64_t base = 0;
    uint64_t mine = (use_list && lane < ncand) ? cands[lane] : UINT64_MAX;
    uint64_t s = 0, count = 0;
    while (s < n) {
        const uint64_t lo = s + mn, hi = s + mx;
        uint64_t c = UINT64_MAX;
        if (use_list) {
            while (true) {
                const uint32_t ge = __ballot_sync(0xffffffffu, mine >= lo);
                if (ge) {
                    c = __shfl_sync(0xffffffffu, mine, __ffs(ge) - 1);
                    break;
                }
                if (base + 32 >= ncand) break;            // list exhausted
                base += 32;
                mine = (base + lane < ncand) ? cands[base + lane] : UINT64_MAX;
            }
            if (c > hi || c > n) c = UINT64_MAX;
        } else {
            c = first_cut_bitmap(bitmap, n, lo, hi);
        }
        uint64_t cut;
        if (c != UINT64_MAX) cut = c;
        else if (hi < n) cut = hi;
        else cut = n;
        if (lane == 0 && count < cap) ends[count] = cut;
        count++;
        s = cut;
    }
    if (lane == 0) *d_count = count;
}

// Selection for one segment of a pipelined chunking: candidates are known up to
// L (the segment's end; L = n for the last one). Starts from the carried chunk
// start, appends every cut the known candidates decide, and carries the start
// of the still-open chunk to the next segment.
__global__ void __launch_bounds__(kSelThreads) k_select_seg(
    const uint64_t *__restrict__ cands, uint64_t cand_cap, const uint32_t *__restrict__ bitmap,
    uint64_t n, uint64_t L, uint64_t mn, uint64_t mx, uint64_t *__restrict__ ends, uint64_t cap,
    PipeState *st, int seg, uint32_t *__restrict__ long_idx, uint32_t klong) {
    __shared__ uint64_t s_carry, s_count, s_ncand, s_new, s_thr;
    __shared__ uint32_t s_k0, s_nlong;
    __shared__ uint32_t hist[128];
    const int t = threadIdx.x;
    if (t == 0) {
        s_carry = st->carry;
        s_count = st->count;
        s_ncand = st->ncand;
        uint32_t k0 = 0;
        if (s_ncand <= cand_cap && s_ncand < 0xffffffffull) {
            uint32_t hi = (uint32_t)s_ncand;                  // first candidate > carry
            while (k0 < hi) {
                const uint32_t mid = k0 + (hi - k0) / 2;
                if (cands[mid] > s_carry) hi = mid; else k0 = mid + 1;
            }
        }
        s_k0 = k0;
        s_new = 0;
        s_nlong = 0;
    }
    if (t < 128) hist[t] = 0;
    __syncthreads();
    const uint64_t count = s_count, carry = s_carry;
    const uint64_t room = cap > count ? cap - count : 0;
    if (s_ncand > cand_cap || s_ncand >= 0xffffffffull) {
        if (t == 0) {
            uint64_t idx = 0;
            const uint64_t last = select_thread_bitmap(bitmap, carry, n, mn, mx,
                                                       WriteEmit{ends + count, room, &idx, 0}, L);
            s_new = idx;
            st->carry = last;
        }
    } else {
        select_block(cands + s_k0, (uint32_t)(s_ncand - s_k0), carry, n, mn, mx, ends + count, room,
                     &s_new, L, 0);
    }
    __syncthreads();
    const uint64_t nw = s_new;
    if (t == 0) {
        st->count = count + nw;
        if (!(s_ncand > cand_cap || s_ncand >= 0xffffffffull)) st->carry = nw ? ends[count + nw - 1] : carry;
        st->seg_cnt[seg + 1] = count + nw;
    }
    // The segment's longest chunks (at most klong) get lone lanes in
    // k_hash_seg: histogram of sizes in 128 bands of (max+1)/128 bytes, the
    // lowest band from which the bands above hold at most klong chunks.
    const uint64_t hi = min(count + nw, cap);
    const uint64_t start0 = st->start0;
    for (uint64_t i = count + t; i < hi; i += kSelThreads) {
        const uint64_t a = i ? ends[i - 1] : start0;
        const uint64_t q = (ends[i] - a) * 128 / (mx + 1);
        const uint32_t band = q < 127 ? (uint32_t)q : 127u;
        atomicAdd(&hist[band], 1u);
    }
    __syncthreads();
    if (t == 0) {
        uint32_t cum = 0;
        int b = 128;
        while (b > 0 && cum + hist[b - 1] <= klong) cum += hist[--b];
        s_thr = b == 128 ? ~0ull : (b * (mx + 1) + 127) / 128;
    }
    __syncthreads();
    const uint64_t thr = s_thr;
    for (uint64_t i = count + t; i < hi; i += kSelThreads) {
        const uint64_t a = i ? ends[i - 1] : start0;
        if (ends[i] - a >= thr) {
            const uint32_t k = atomicAdd(&s_nlong, 1u);
            if (k < klong) long_idx[(size_t)seg * kLongMax + k] = (uint32_t)(i - count);
        }
    }
    __syncthreads();
    if (t == 0) {
        st->thr[seg] = thr;
        st->nlong[seg] = min(s_nlong, klong);
    }
}

// Digests of the chunks one segment's selection finalized. The first
// ceil(klong/4) CTAs give each of the segment's listed longest chunks a warp
// of its own (lane 0); the other CTAs take one chunk per thread and skip
// those.
template <class H>
__global__ void __launch_bounds__(128) k_hash_seg(const uint8_t *__restrict__ in,
                                                  const uint64_t *__restrict__ ends,
                                                  const PipeState *st, int seg,
                                                  const uint32_t *__restrict__ long_idx,
                                                  uint32_t klong, uint8_t *__restrict__ out,
                                                  uint64_t n, int *err) {
    const uint64_t lo = st->seg_cnt[seg], hi = st->seg_cnt[seg + 1];
    const uint32_t long_ctas = (klong + 3) / 4;
    uint64_t i;
    if (blockIdx.x < long_ctas) {
        const uint32_t w = blockIdx.x * 4 + threadIdx.x / 32;
        if ((threadIdx.x & 31) != 0 || w >= st->nlong[seg]) return;
        i = lo + long_idx[(size_t)seg * kLongMax + w];
    } else {
        i = lo + (uint64_t)(blockIdx.x - long_ctas) * blockDim.x + threadIdx.x;
        if (i >= hi) return;
        const uint64_t a0 = i ? ends[i - 1] : st->start0;
        if (ends[i] - a0 >= st->thr[seg]) return;          // on a lone lane
    }
    const uint64_t a = i ? ends[i - 1] : st->start0, b = ends[i];
    if (!HG_DOK(a <= b && b <= n, err)) return;
    H hs;
    hash_range_staged(in + a, b - a, hs, stage_ring_dyn());
    store_digest(hs, out + i * H::kDigest);
}

// Deferred digests (launch_hash_sorted): length bands of (max+1)/128 bytes,
// numbered longest first.
__device__ __forceinline__ uint32_t len_band(uint64_t len, uint64_t mx) {
    const uint64_t q = len * 128 / (mx + 1);
    return 127u - (q < 127 ? (uint32_t)q : 127u);
}

__global__ void __launch_bounds__(256) k_len_hist(const uint64_t *__restrict__ ends, PipeState *st,
                                                  uint64_t mx) {
    __shared__ uint32_t h[128];
    if (threadIdx.x < 128) h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t cnt = st->count, s0 = st->start0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t a = i ? ends[i - 1] : s0;
        atomicAdd(&h[len_band(ends[i] - a, mx)], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 128 && h[threadIdx.x]) atomicAdd(&st->band_cnt[threadIdx.x], h[threadIdx.x]);
}

// One warp: exclusive scan of the 128 band counts into the bands' first slots.
__global__ void k_len_scan(PipeState *st) {
    const int lane = threadIdx.x;
    uint32_t v[4], sum = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) { v[k] = st->band_cnt[4 * lane + k]; sum += v[k]; }
    uint32_t x = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    uint32_t run = x - sum;
#pragma unroll
    for (int k = 0; k < 4; k++) { st->band_cur[4 * lane + k] = run; run += v[k]; }
}

__global__ void __launch_bounds__(256) k_len_scatter(const uint64_t *__restrict__ ends, PipeState *st,
                                                     uint64_t mx, uint32_t *__restrict__ tasks) {
    const uint64_t cnt = st->count, s0 = st->start0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t a = i ? ends[i - 1] : s0;
        const uint32_t at = atomicAdd(&st->band_cur[len_band(ends[i] - a, mx)], 1u);
        tasks[at] = (uint32_t)i;
    }
}

// The first ceil(klong/4) CTAs give the klong longest chunks a warp each
// (lane 0); the other CTAs are persistent bulk warps that take the rest 32 at
// a time, longest first, from a counter. Few bulk warps per SM leave issue
// slots to the long chains, which set the launch's duration: with every
// chunk's warp resident at once (1 GiB: 3.3K warps) the long chains crawled.
// Measured on 1 GiB (105K chunks): one bulk CTA of 4 warps per SM 12.42 ms
// for the whole call, two 12.65, four 13.05, one warp per chunk 12.66.
template <class H>
__global__ void __launch_bounds__(128) k_hash_sorted(const uint8_t *__restrict__ in,
                                                     const uint64_t *__restrict__ ends,
                                                     PipeState *st,
                                                     const uint32_t *__restrict__ tasks,
                                                     uint32_t klong, uint8_t *__restrict__ out,
                                                     uint64_t n, int *err) {
    const uint64_t cnt = st->count, s0 = st->start0;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t long_ctas = (klong + 3) / 4;
    if (blockIdx.x < long_ctas) {
        const uint64_t k = (uint64_t)blockIdx.x * 4 + threadIdx.x / 32;
        if (lane || k >= klong || k >= cnt) return;
        const uint64_t i = tasks[k];
        const uint64_t a = i ? ends[i - 1] : s0;
        if (!HG_DOK(i < cnt && a <= ends[i] && ends[i] <= n, err)) return;
        H hs;
        hash_range_staged(in + a, ends[i] - a, hs, stage_ring_dyn());
        store_digest(hs, out + i * H::kDigest);
        return;
    }
    while (true) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&st->task_ctr, 32ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (klong + base >= cnt) return;
        const uint64_t k = klong + base + lane;
        if (k < cnt) {
            const uint64_t i = tasks[k];
            const uint64_t a = i ? ends[i - 1] : s0;
            if (HG_DOK(i < cnt && a <= ends[i] && ends[i] <= n, err)) {
                H hs;
                hash_range_staged(in + a, ends[i] - a, hs, stage_ring_dyn());
                store_digest(hs, out + i * H::kDigest);
            }
        }
    }
}

// Streaming: start a feed whose first chunk starts at start0 of the buffer.
__global__ void k_stream_init(PipeState *st, uint64_t start0) {
    if (threadIdx.x == 0) {
        st->carry = start0;
        st->start0 = start0;
        st->count = 0;
        st->ncand = 0;
        st->seg_cnt[0] = 0;
    }
}

// Streaming: the feed's chunk ends, shifted to stream offsets, and its count.
__global__ void k_stream_out(const uint64_t *__restrict__ ends, const PipeState *st, uint64_t base,
                             uint64_t *__restrict__ out, uint64_t cap, uint64_t *count_out) {
    const uint64_t cnt = st->count;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt && i < cap;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = ends[i] + base;
    if (blockIdx.x == 0 && threadIdx.x == 0) *count_out = cnt;
}

// Streaming: copy the open chunk and the halo before it, [carry - h, wl), to the
// start of the next working buffer; info = {carry, h, bytes copied, count}.
__global__ void k_stream_carry(const uint8_t *__restrict__ src, uint64_t wl, const PipeState *st,
                               uint32_t halo, uint8_t *__restrict__ dst, uint64_t *info) {
    const uint64_t carry = st->carry;
    const uint64_t h = carry < halo ? carry : halo;
    const uint64_t from = carry - h, len = wl > from ? wl - from : 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = src[from + i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        info[0] = carry;
        info[1] = h;
        info[2] = len;
        info[3] = st->count;
    }
}

// Selection of the whole stream by one CTA (parallel, exact); when the
// candidate list overflowed, warp 0 walks the bitmap instead.
__global__ void __launch_bounds__(kSelThreads) k_select_par(
    const uint64_t *__restrict__ cands, const uint64_t *__restrict__ d_ncand, uint64_t cand_cap,
    const uint32_t *__restrict__ bitmap, uint64_t n, uint64_t mn, uint64_t mx,
    uint64_t *__restrict__ ends, uint64_t cap, uint64_t *__restrict__ d_count) {
    const uint64_t ncand = *d_ncand;
    if (ncand > cand_cap || ncand >= 0xffffffffull) {
        if (threadIdx.x < 32) select_serial(cands, ncand, false, bitmap, n, mn, mx, ends, cap, d_count);
        return;
    }
    select_block(cands, (uint32_t)ncand, 0, n, mn, mx, ends, cap, d_count);
}


}  // namespace


int launch_compact(const uint32_t *d_bitmap, uint64_t n, const uint32_t *d_tile_cnt,
                   uint64_t *d_tile_off, uint64_t ntiles, uint64_t *d_cands, uint64_t cap,
                   uint64_t *d_count, cudaStream_t s) {
    if (ntiles == 0) return cuda_status(cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s));
    k_scan_tiles<<<1, 1024, 0, s>>>(d_tile_cnt, ntiles, d_tile_off, d_count);
    k_compact<<<(unsigned)ntiles, kWinThreads, 0, s>>>(d_bitmap, (n + 31) / 32, d_tile_cnt,
                                                       d_tile_off, d_cands, cap, 0);
    return cuda_status(cudaGetLastError());
}

int launch_stream_init(PipeState *st, uint64_t start0, cudaStream_t s) {
    k_stream_init<<<1, 32, 0, s>>>(st, start0);
    return cuda_status(cudaGetLastError());
}

int launch_stream_out(const uint64_t *ends, const PipeState *st, uint64_t base, uint64_t *d_ends_out,
                      uint64_t cap, uint64_t *d_count_out, cudaStream_t s) {
    k_stream_out<<<64, 256, 0, s>>>(ends, st, base, d_ends_out, cap, d_count_out);
    return cuda_status(cudaGetLastError());
}

int launch_stream_carry(const uint8_t *src, uint64_t wl, const PipeState *st, uint32_t halo,
                        uint8_t *dst, uint64_t *info, cudaStream_t s) {
    k_stream_carry<<<64, 256, 0, s>>>(src, wl, st, halo, dst, info);
    return cuda_status(cudaGetLastError());
}

int launch_pipe_segment(const uint8_t *d_in, uint64_t n, uint64_t n_sel, const hg_cdc_params &p,
                        int algo, uint32_t tile0, uint32_t ntiles, uint64_t L, int seg,
                        uint64_t max_chunks, const PipeBufs &b, cudaStream_t s_win,
                        cudaStream_t s_sel, cudaStream_t s_hash, cudaEvent_t ev_win,
                        cudaEvent_t ev_sel, cudaEvent_t ev_input, bool digests) {
    if (ev_input) cudaStreamWaitEvent(s_win, ev_input, 0);    // this segment's bytes are in place
    // windows run back to back on s_win; the small serial steps (scan, compaction,
    // selection) of segment k run on s_sel, in segment order, once its windows are done
    int r;
    if ((r = launch_window_range(d_in, n, p, b.bitmap, b.tile_cnt, tile0, ntiles, s_win, b.err)))
        return r;
    cudaEventRecord(ev_win, s_win);
    cudaStreamWaitEvent(s_sel, ev_win, 0);
    k_scan_tiles_base<<<1, 1024, 0, s_sel>>>(b.tile_cnt + tile0, ntiles, b.tile_off + tile0,
                                             &b.st->ncand);
    k_compact<<<ntiles, kWinThreads, 0, s_sel>>>(b.bitmap, (n + 31) / 32, b.tile_cnt, b.tile_off,
                                                 b.cands, b.cand_cap, tile0);
    k_select_seg<<<1, kSelThreads, 0, s_sel>>>(b.cands, b.cand_cap, b.bitmap, n_sel, L, p.min_chunk,
                                               p.max_chunk, b.ends, b.cap, b.st, seg, b.long_idx,
                                               b.klong);
    cudaEventRecord(ev_sel, s_sel);
    if (!digests) return cuda_status(cudaGetLastError());
    cudaStreamWaitEvent(s_hash, ev_sel, 0);
    const unsigned grid = (unsigned)((max_chunks + 127) / 128 + (b.klong + 3) / 4);
    const size_t smem = stage_bytes(128);
    if (algo == HG_MD5) {
        if (allow_dyn_smem((const void *)k_hash_seg<Md5Chain>, smem) != cudaSuccess) return HG_ECUDA;
        k_hash_seg<Md5Chain><<<grid, 128, smem, s_hash>>>(d_in, b.ends, b.st, seg, b.long_idx, b.klong,
                                                          b.digests, n, b.err);
    } else {
        if (allow_dyn_smem((const void *)k_hash_seg<Sha1>, smem) != cudaSuccess) return HG_ECUDA;
        k_hash_seg<Sha1><<<grid, 128, smem, s_hash>>>(d_in, b.ends, b.st, seg, b.long_idx, b.klong,
                                                      b.digests, n, b.err);
    }
    return cuda_status(cudaGetLastError());
}

constexpr uint64_t kBulkCtasPerSm = 1;

int launch_hash_sorted(const uint8_t *d_in, uint64_t n, uint64_t max_chunks, const hg_cdc_params &p,
                       int algo, const PipeBufs &b, cudaStream_t s) {
    const unsigned sgrid = 4 * 148;
    k_len_hist<<<sgrid, 256, 0, s>>>(b.ends, b.st, p.max_chunk);
    k_len_scan<<<1, 32, 0, s>>>(b.st);
    k_len_scatter<<<sgrid, 256, 0, s>>>(b.ends, b.st, p.max_chunk, b.tasks);
    // bulk: kBulkCtasPerSm CTAs of 4 warps per SM (the lone-warp count is one per SM)
    const uint64_t bulk_ctas = (uint64_t)b.klong * kBulkCtasPerSm;
    const uint64_t need = ((max_chunks + 31) / 32 + 3) / 4;
    const unsigned grid = (unsigned)((b.klong + 3) / 4 + (need < bulk_ctas ? need : bulk_ctas));
    const size_t smem = stage_bytes(128);
    if (algo == HG_MD5) {
        if (allow_dyn_smem((const void *)k_hash_sorted<Md5Chain>, smem) != cudaSuccess) return HG_ECUDA;
        k_hash_sorted<Md5Chain><<<grid, 128, smem, s>>>(d_in, b.ends, b.st, b.tasks, b.klong,
                                                        b.digests, n, b.err);
    } else {
        if (allow_dyn_smem((const void *)k_hash_sorted<Sha1>, smem) != cudaSuccess) return HG_ECUDA;
        k_hash_sorted<Sha1><<<grid, 128, smem, s>>>(d_in, b.ends, b.st, b.tasks, b.klong, b.digests,
                                                    n, b.err);
    }
    return cuda_status(cudaGetLastError());
}

int launch_scan_tiles(const uint32_t *d_tile_cnt, uint64_t ntiles, uint64_t *d_tile_off,
                      uint64_t *d_total, cudaStream_t s) {
    if (ntiles == 0) return cuda_status(cudaMemsetAsync(d_total, 0, sizeof(uint64_t), s));
    k_scan_tiles<<<1, 1024, 0, s>>>(d_tile_cnt, ntiles, d_tile_off, d_total);
    return cuda_status(cudaGetLastError());
}

int launch_select(const uint64_t *d_cands, const uint64_t *d_ncand, uint64_t cand_cap,
                  const uint32_t *d_bitmap, uint64_t n, const hg_cdc_params &p, uint64_t *d_ends,
                  uint64_t cap, uint64_t *d_count, cudaStream_t s) {
    k_select_par<<<1, kSelThreads, 0, s>>>(d_cands, d_ncand, cand_cap, d_bitmap, n, p.min_chunk,
                                           p.max_chunk, d_ends, cap, d_count);
    return cuda_status(cudaGetLastError());
}

}  // namespace hg
