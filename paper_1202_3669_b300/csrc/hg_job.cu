// One batched chunking job over many files: the kernels shared by the batch
// API (files back to back in one buffer) and the request server (one device
// staging buffer per request).
//
// The paper gets its speed-ups only when hashing jobs are batched (Sec. 3.2.3:
// a stream of hashing computations; Sec. 4.1: gains need batches) and it
// buffers writes so each GPU job covers many chunks (Sec. 3.2.4). A job here
// is a fixed sequence of launches with no host round trip:
//   1. a persistent window kernel pulls 8 KiB tiles from an atomic tile counter
//      (the device work queue); tiles never span files, each file's tiles are
//      consecutive; the next tile is prefetched by bulk async copy while the
//      current one is hashed;
//   2. the per-tile counts are scanned and every tile writes its candidates
//      (cut positions local to its file), so each file's candidates form one
//      sorted slice of the list;
//   3. every file selects its boundaries from its slice: small files with one
//      thread each, the others with one CTA each running the parallel exact
//      selection;
//   4. the chunks become a task list with long chunks first;
//   5. a persistent kernel hashes the tasks, each warp pulling 32 at a time.
#include <algorithm>

#include "hg_device.cuh"
#include "hg_internal.h"
#include "hg_rabin.cuh"
#include "hg_select.cuh"
#include "hg_window.cuh"

namespace hg {
namespace {

__device__ __forceinline__ uint32_t upper_index(const uint64_t *__restrict__ a, uint32_t lo,
                                                uint32_t hi, uint64_t v) {
    // first i in [lo, hi) with a[i] > v (hi if none); a sorted
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (__ldg(a + mid) > v) hi = mid; else lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ const uint8_t *jptr(const JobDev &j, uint32_t f) {
    return j.base ? j.base + j.file_off[f] : j.file_ptr[f];
}
__device__ __forceinline__ uint64_t jlen(const JobDev &j, uint32_t f) {
    return j.base ? j.file_off[f + 1] - j.file_off[f] : j.file_len[f];
}
// file owning global tile t (the last f with tile_start[f] <= t)
__device__ __forceinline__ uint32_t tile_file(const JobDev &j, uint32_t t) {
    return upper_index(j.tile_start, 0, j.nfile + 1, t) - 1;
}

struct TileRef {
    const uint8_t *ptr;   // file bytes
    uint64_t len;         // file length
    uint64_t lo;          // local offset of the tile's first window end
    bool fast;            // interior tile of a 16-byte aligned file: one bulk copy
};

__device__ __forceinline__ TileRef tile_ref(const JobDev &j, uint32_t t) {
    const uint32_t f = tile_file(j, t);
    TileRef r;
    r.ptr = jptr(j, f);
    r.len = jlen(j, f);
    r.lo = (uint64_t)(t - j.tile_start[f]) * kWinTile;
    r.fast = ((reinterpret_cast<uintptr_t>(r.ptr) & 15) == 0) && r.lo >= (uint64_t)kHalo &&
             r.lo + kWinTile <= r.len;
    return r;
}

// Pipe policy: the constant-word steps' adds on the FMA pipe, the data-word
// steps' on the ALU (at this kernel's 32 registers and 8-warp CTAs moving the
// data-word adds as well measured slower: 0.657 vs 0.651 ms per 64 MiB).
template <int W>
__global__ void __launch_bounds__(kWinThreads) k_job_window(JobDev j, uint32_t wrt, uint32_t mask,
                                                            uint32_t magic,
                                                            uint32_t *__restrict__ bitmap,
                                                            uint32_t *__restrict__ tile_cnt,
                                                            unsigned long long *tile_ctr, int *err,
                                                            uint32_t one) {
    const uint32_t wlen = W ? (uint32_t)W : wrt;
    __shared__ __align__(128) uint8_t sbuf[2][kSmemBytes];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t s_tile[2];
    __shared__ TileRef s_ref[2];
    __shared__ uint32_t warp_cnt[kWinThreads / 32];
    const int t = threadIdx.x;
    const uint32_t ntiles = j.ntiles;
    auto claim = [&](int buf) {            // thread 0: next tile into buffer buf
        const uint32_t c = (uint32_t)atomicAdd(tile_ctr, 1ull);
        s_tile[buf] = c;
        if (c < ntiles) {
            const TileRef r = tile_ref(j, c);
            s_ref[buf] = r;
            if (r.fast)
                bulk_load(smem_u32(sbuf[buf]), r.ptr + r.lo - kHalo, (uint32_t)(kHalo + kWinTile),
                          smem_u32(&mbar[buf]));
        }
    };
    if (t == 0) {
        mbar_init(smem_u32(&mbar[0]));
        mbar_init(smem_u32(&mbar[1]));
    }
    __syncthreads();
    if (t == 0) claim(0);
    __syncthreads();
    int b = 0;
    uint32_t phase[2] = {0, 0};
    while (true) {
        const uint32_t cur = s_tile[b];
        if (cur >= ntiles) break;
        const TileRef r = s_ref[b];
        if (t == 0) claim(b ^ 1);
        bool timed_out = false;
        if (r.fast) {
            timed_out = !mbar_wait(smem_u32(&mbar[b]), phase[b]);
            if (timed_out) atomicCAS(err, 0, (int)HG_ETIMEDOUT);
            phase[b] ^= 1;
        } else {
            for (int i = t; i < kHalo + (int)kWinTile; i += kWinThreads) {
                const int64_t g = (int64_t)r.lo - kHalo + i;
                sbuf[b][i] = (g >= 0 && (uint64_t)g < r.len) ? r.ptr[g] : (uint8_t)0;
            }
        }
        if (t < 4) reinterpret_cast<uint32_t *>(sbuf[b] + kHalo + kWinTile)[t] = 0;
        if (__syncthreads_or(timed_out)) {
            // bounded drain of the copy into the other buffer, then leave
            if (t == 0 && s_tile[b ^ 1] < ntiles && s_ref[b ^ 1].fast)
                mbar_wait(smem_u32(&mbar[b ^ 1]), phase[b ^ 1]);
            return;
        }
        const uint64_t p0 = r.lo + 32u * (uint64_t)t;
        const uint32_t bits =
            clip_bits(window_bits32<W, kPolAll2, kPolAllPlain>(sbuf[b], t, wlen, mask, magic, one),
                      p0, wlen, r.len);
        bitmap[(uint64_t)cur * kWinThreads + t] = bits;
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

// The same window test in one-warp CTAs (the form of the single-buffer window
// kernel): CTA b takes span b % 8 (1024 window ends) of global tile b / 8, of
// whichever file owns the tile; spans past the file's end write zero words.
// Counts are added to the tile's count (zeroed before the launch). Selected by
// the tuning's window_ctas_per_sm = 0.
//
// Files of a batch start at any byte. An interior span whose bytes do not
// start on a 16-byte boundary is still staged by one bulk copy: the copy takes
// the 16-byte granules that cover the span (its extra bytes lie in granules
// that hold span bytes, so in the same mapped memory) into a second buffer,
// and the warp shifts the words into place (9 funnel shifts a lane). The 4096-
// file batch stored back to back took 43.79 ms with such spans staged by byte
// loads, 42.24 ms with every file moved to a 16-byte aligned slot.
template <int W>
__global__ void __launch_bounds__(32, 32) k_job_window_span(JobDev j, uint32_t wrt, uint32_t mask,
                                                            uint32_t magic,
                                                            uint32_t *__restrict__ bitmap,
                                                            uint32_t *__restrict__ tile_cnt, int *err,
                                                            uint32_t one) {
    const uint32_t wlen = W ? (uint32_t)W : wrt;
    constexpr int kSub = (int)(kWinTile / kWinSpan);
    constexpr int kSpanBytes = kHalo + kWinSpan;              // a multiple of 16
    __shared__ __align__(128) uint8_t sbuf[kSpanBytes + 16];
    __shared__ __align__(128) uint8_t sraw[kSpanBytes + 16];  // granules of an unaligned span
    __shared__ __align__(8) uint64_t mbar;
    const int t = threadIdx.x;
    const uint32_t tile = blockIdx.x / kSub, sub = blockIdx.x % kSub;
    if (!HG_DOK(tile < j.ntiles, err)) return;
    const TileRef r = tile_ref(j, tile);
    const uint64_t lo = r.lo + (uint64_t)sub * kWinSpan;
    uint32_t bits = 0;
    if (lo < r.len) {
        const bool fast = lo >= (uint64_t)kHalo && lo + kWinSpan <= r.len;
        if (t < 4) reinterpret_cast<uint32_t *>(sbuf + kSpanBytes)[t] = 0;
        bool timed_out = false;
        if (fast) {
            const uint8_t *src = r.ptr + lo - kHalo;
            const uint32_t a = (uint32_t)(reinterpret_cast<uintptr_t>(src) & 15);
            const uint32_t mb = smem_u32(&mbar);
            if (t == 0) mbar_init(mb);
            __syncwarp();
            if (t == 0) {
                if (a == 0) bulk_load(smem_u32(sbuf), src, (uint32_t)kSpanBytes, mb);
                else bulk_load(smem_u32(sraw), src - a, (uint32_t)(kSpanBytes + 16), mb);
            }
            timed_out = !mbar_wait(mb, 0);
            if (timed_out) {
                atomicCAS(err, 0, (int)HG_ETIMEDOUT);
                mbar_wait(mb, 0);
            }
            if (a != 0 && !timed_out) {
                // span word i = bytes a + 4i .. a + 4i + 3 of the granules
                const uint32_t *rw = reinterpret_cast<const uint32_t *>(sraw);
                uint32_t *sw = reinterpret_cast<uint32_t *>(sbuf);
                const uint32_t q = a >> 2, r8 = (a & 3) * 8;
                for (int i = t; i < kSpanBytes / 4; i += 32)
                    sw[i] = __funnelshift_r(rw[i + q], rw[i + q + 1], r8);
            }
        } else {
            for (int i = t; i < kHalo + kWinSpan; i += 32) {
                const int64_t g = (int64_t)lo - kHalo + i;
                sbuf[i] = (g >= 0 && (uint64_t)g < r.len) ? r.ptr[g] : (uint8_t)0;
            }
        }
        if (__any_sync(0xffffffffu, timed_out)) return;
        __syncwarp();
        bits = clip_bits(window_bits32<W>(sbuf, t, wlen, mask, magic, one), lo + 32u * (uint64_t)t,
                         wlen, r.len);
    }
    bitmap[(uint64_t)tile * kWinThreads + sub * 32 + t] = bits;
    const uint32_t c = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(bits));
    if (t == 0 && c) atomicAdd(&tile_cnt[tile], c);
}

// Tile bitmap -> candidate cuts local to the tile's file, at the tile's scanned offset.
__global__ void __launch_bounds__(kWinThreads) k_job_compact(JobDev j,
                                                             const uint32_t *__restrict__ bitmap,
                                                             const uint32_t *__restrict__ tile_cnt,
                                                             const uint64_t *__restrict__ tile_off,
                                                             uint64_t *__restrict__ cands,
                                                             uint64_t cap) {
    __shared__ uint32_t warp_sum[kWinThreads / 32];
    __shared__ uint64_t s_lo;
    const uint32_t tile = blockIdx.x;
    if (tile_cnt[tile] == 0) return;
    const int t = threadIdx.x;
    if (t == 0) {
        const uint32_t f = tile_file(j, tile);
        s_lo = (uint64_t)(tile - j.tile_start[f]) * kWinTile;
    }
    uint32_t w = bitmap[(uint64_t)tile * kWinThreads + t];
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
    uint64_t idx = tile_off[tile] + before;
    const uint64_t pos0 = s_lo + 32u * (uint64_t)t;
    while (w) {
        const int bit = __ffs(w) - 1;
        w &= w - 1;
        if (idx < cap) cands[idx] = pos0 + bit + 1;
        idx++;
    }
}

__device__ __forceinline__ void file_cands(const JobDev &j, const uint64_t *__restrict__ tile_off,
                                           uint32_t f, uint64_t &k0, uint64_t &k1) {
    k0 = tile_off[j.tile_start[f]];
    k1 = tile_off[j.tile_start[f + 1]];
}

__global__ void k_job_select_small(JobDev j, const uint64_t *__restrict__ tile_off,
                                   const uint64_t *__restrict__ cands, uint64_t cand_cap,
                                   const uint32_t *__restrict__ bitmap, uint64_t mn, uint64_t mx,
                                   uint64_t *__restrict__ ends, uint64_t *__restrict__ counts,
                                   unsigned long long *words) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= j.nsmall) return;
    const uint32_t f = j.small[i];
    const uint64_t n = jlen(j, f);
    const uint64_t so = j.slot_off[f], cap = j.slot_off[f + 1] - so;
    const uint64_t ncand = tile_off[j.ntiles];
    uint64_t idx = 0;
    if (ncand <= cand_cap && ncand < 0xffffffffull) {
        uint64_t k0, k1;
        file_cands(j, tile_off, f, k0, k1);
        select_thread(cands + k0, (uint32_t)(k1 - k0), 0, n, mn, mx, WriteEmit{ends + so, cap, &idx, 0});
    } else {
        select_thread_bitmap(bitmap + (uint64_t)j.tile_start[f] * kWinThreads, 0, n, mn, mx,
                             WriteEmit{ends + so, cap, &idx, 0});
    }
    counts[f] = idx;
    atomicAdd(&words[kJobTotal], (unsigned long long)min(idx, cap));
}

__global__ void __launch_bounds__(kSelThreads) k_job_select_big(
    JobDev j, const uint64_t *__restrict__ tile_off, const uint64_t *__restrict__ cands,
    uint64_t cand_cap, const uint32_t *__restrict__ bitmap, uint64_t mn, uint64_t mx,
    uint64_t *__restrict__ ends, uint64_t *__restrict__ counts, unsigned long long *words) {
    const uint32_t f = j.big[blockIdx.x];
    const uint64_t n = jlen(j, f);
    const uint64_t so = j.slot_off[f], cap = j.slot_off[f + 1] - so;
    const uint64_t ncand = tile_off[j.ntiles];
    if (ncand > cand_cap || ncand >= 0xffffffffull) {
        if (threadIdx.x == 0) {
            uint64_t idx = 0;
            select_thread_bitmap(bitmap + (uint64_t)j.tile_start[f] * kWinThreads, 0, n, mn, mx,
                                 WriteEmit{ends + so, cap, &idx, 0});
            counts[f] = idx;
            atomicAdd(&words[kJobTotal], (unsigned long long)min(idx, cap));
        }
        return;
    }
    uint64_t k0, k1;
    file_cands(j, tile_off, f, k0, k1);
    select_block(cands + k0, (uint32_t)(k1 - k0), 0, n, mn, mx, ends + so, cap, counts + f);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(&words[kJobTotal], (unsigned long long)min(counts[f], cap));
}

// Task list ordered by chunk length, longest first (counting sort on 1 KiB
// buckets), so the 32 chunks a warp hashes together have nearly equal serial
// chains and long chains start first.
constexpr int kLenBuckets = 64;
__device__ __forceinline__ int len_bucket(uint64_t len) {
    const uint64_t b = len >> 10;
    return (int)(kLenBuckets - 1 - (b < kLenBuckets - 1 ? b : kLenBuckets - 1));   // long first
}

__global__ void k_job_hist(JobDev j, const uint64_t *__restrict__ ends,
                           const uint64_t *__restrict__ counts, unsigned long long *hist) {
    __shared__ unsigned int h[kLenBuckets];
    for (int i = threadIdx.x; i < kLenBuckets; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint32_t f = blockIdx.x;
    const uint64_t so = j.slot_off[f];
    const uint64_t cnt = min(counts[f], j.slot_off[f + 1] - so);
    for (uint64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
        const uint64_t len = ends[so + i] - (i ? ends[so + i - 1] : 0);
        atomicAdd(&h[len_bucket(len)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kLenBuckets; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}

// exclusive scan of the bucket counts into cursors (one warp)
__global__ void k_job_hist_scan(unsigned long long *hist, unsigned long long *cursor) {
    const int lane = threadIdx.x;
    unsigned long long a = hist[lane], b = hist[lane + 32];
    unsigned long long x = a;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    const unsigned long long tot_a = __shfl_sync(0xffffffffu, x, 31);
    unsigned long long z = b;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, z, d);
        if (lane >= d) z += y;
    }
    cursor[lane] = x - a;
    cursor[lane + 32] = tot_a + z - b;
}

__global__ void k_job_tasks(JobDev j, const uint64_t *__restrict__ ends,
                            const uint64_t *__restrict__ counts, unsigned long long *cursor,
                            uint64_t *__restrict__ tasks) {
    const uint32_t f = blockIdx.x;
    const uint64_t so = j.slot_off[f];
    const uint64_t cnt = min(counts[f], j.slot_off[f + 1] - so);
    for (uint64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
        const uint64_t len = ends[so + i] - (i ? ends[so + i - 1] : 0);
        const unsigned long long at = atomicAdd(&cursor[len_bucket(len)], 1ull);
        tasks[at] = ((uint64_t)f << 32) | (uint32_t)i;
    }
}

// STAGED: the chains read through shared-memory rings (hash_range_staged);
// CTAs too large for the rings to fit use hash_range.
template <class H, bool STAGED>
__global__ void k_job_hash(JobDev j, const uint64_t *__restrict__ ends,
                           const uint64_t *__restrict__ tasks, unsigned long long *words,
                           uint8_t *__restrict__ digests, int *err) {
    const int lane = threadIdx.x & 31;
    const uint64_t total = words[kJobTotal];
    while (true) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&words[kJobTaskCtr], 32ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= total) break;
        const uint64_t k = base + lane;
        if (k < total) {
            const uint64_t tk = tasks[k];
            const uint32_t f = (uint32_t)(tk >> 32), i = (uint32_t)tk;
            if (!HG_DOK(f < j.nfile, err)) continue;
            const uint64_t so = j.slot_off[f];
            if (!HG_DOK(so + i < j.slot_off[f + 1], err)) continue;
            const uint64_t lo = i ? ends[so + i - 1] : 0, hi = ends[so + i];
            if (!HG_DOK(lo <= hi && hi <= jlen(j, f), err)) continue;
            H hs;
            if constexpr (STAGED) hash_range_staged(jptr(j, f) + lo, hi - lo, hs, stage_ring_dyn());
            else hash_range(jptr(j, f) + lo, hi - lo, hs);
            store_digest(hs, digests + (so + i) * H::kDigest);
        }
    }
}

// Rabin window over the batch's per-file tiles: persistent CTAs build the
// fingerprint tables once, then take groups of 4 global tiles; each 64-thread
// quarter handles one tile (128 window ends per thread) of whichever file
// owns it, in the same bitmap layout and tile counts as k_job_window. Files
// sit at any offset, so strips are realigned from 16-byte loads.
template <int W>
__global__ void __launch_bounds__(rabin::kThreads, 2)
    k_job_rabin(JobDev j, uint32_t wrt, uint32_t mask, uint32_t magic, uint32_t *__restrict__ bitmap,
                uint32_t *__restrict__ tile_cnt) {
    using namespace rabin;
    extern __shared__ __align__(16) uint32_t tabs[];
    __shared__ uint32_t warp_cnt[kThreads / 32];
    const uint32_t wlen = W ? (uint32_t)W : wrt;
    const int t = threadIdx.x, lane = t & 31;
    build_tables(tabs, wlen);
    const uint32_t *T = tabs + lane;
    const uint32_t *U = tabs + 256 * 32 + lane;
    const uint64_t ngroups = ((uint64_t)j.ntiles + kTilesPerGroup - 1) / kTilesPerGroup;
    const uint32_t sub = (uint32_t)t >> 6, q = (uint32_t)t & 63;
    for (uint64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const uint64_t tile = g * kTilesPerGroup + sub;
        uint32_t bits[4] = {0, 0, 0, 0};
        if (tile < j.ntiles) {
            const uint32_t f = tile_file(j, (uint32_t)tile);
            const uint64_t lo = (tile - j.tile_start[f]) * kWinTile;
            strip_bits<W, true>(jptr(j, f), jlen(j, f), lo + (uint64_t)q * kStrip, wlen, mask, magic,
                                T, U, bits);
            uint4 *dst = reinterpret_cast<uint4 *>(bitmap + tile * kWinThreads) + q;
            *dst = make_uint4(bits[0], bits[1], bits[2], bits[3]);
        }
        const uint32_t c = __reduce_add_sync(0xffffffffu, (uint32_t)(__popc(bits[0]) + __popc(bits[1]) +
                                                                   __popc(bits[2]) + __popc(bits[3])));
        if (lane == 0) warp_cnt[t >> 5] = c;
        __syncthreads();
        if (t < (int)kTilesPerGroup && g * kTilesPerGroup + t < j.ntiles)
            tile_cnt[g * kTilesPerGroup + t] = warp_cnt[2 * t] + warp_cnt[2 * t + 1];
        __syncthreads();
    }
}

template <int W>
cudaError_t job_rabin_opt_in() {
    return cudaFuncSetAttribute(k_job_rabin<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)rabin::kSmem);
}

template <int W>
void launch_job_rabin_t(int grid, const JobDev &j, uint32_t w, uint32_t mask, uint32_t magic,
                        uint32_t *bm, uint32_t *tc, cudaStream_t s) {
    k_job_rabin<W><<<grid, rabin::kThreads, rabin::kSmem, s>>>(j, w, mask, magic, bm, tc);
}

template <int W>
void launch_job_window_t(int grid, const JobDev &j, uint32_t w, uint32_t mask, uint32_t magic,
                         uint32_t *bm, uint32_t *tc, unsigned long long *ctr, int *err,
                         cudaStream_t s) {
    k_job_window<W><<<grid, kWinThreads, 0, s>>>(j, w, mask, magic, bm, tc, ctr, err, 1u);
}

template <int W>
void launch_job_window_span_t(const JobDev &j, uint32_t w, uint32_t mask, uint32_t magic,
                              uint32_t *bm, uint32_t *tc, int *err, cudaStream_t s) {
    const uint64_t spans = (uint64_t)j.ntiles * (kWinTile / kWinSpan);
    k_job_window_span<W><<<(unsigned)spans, 32, 0, s>>>(j, w, mask, magic, bm, tc, err, 1u);
}

template <int W>
int occupancy_t() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_job_window<W>, kWinThreads, 0);
    return nb > 0 ? nb : 1;
}

}  // namespace

int job_rabin_prepare() {
    if (job_rabin_opt_in<0>() != cudaSuccess || job_rabin_opt_in<16>() != cudaSuccess ||
        job_rabin_opt_in<20>() != cudaSuccess || job_rabin_opt_in<24>() != cudaSuccess ||
        job_rabin_opt_in<32>() != cudaSuccess || job_rabin_opt_in<48>() != cudaSuccess ||
        job_rabin_opt_in<64>() != cudaSuccess) {
        cudaGetLastError();
        return HG_ECUDA;
    }
    return HG_OK;
}

int job_window_occupancy(uint32_t w) {
    switch (w) {
        case 16: return occupancy_t<16>();
        case 20: return occupancy_t<20>();
        case 24: return occupancy_t<24>();
        case 32: return occupancy_t<32>();
        case 48: return occupancy_t<48>();
        default: return occupancy_t<0>();
    }
}

void job_plan(const uint64_t *len, uint32_t nfile, uint64_t min_chunk, JobHost *h) {
    h->tile_start.resize(nfile + 1);
    h->slot_off.resize(nfile + 1);
    h->small.clear();
    h->big.clear();
    uint64_t t = 0, so = 0;
    for (uint32_t f = 0; f < nfile; f++) {
        h->tile_start[f] = t;
        h->slot_off[f] = so;
        t += (len[f] + kWinTile - 1) / kWinTile;
        so += len[f] ? len[f] / min_chunk + 1 : 0;         // >= chunks the rule can make
        (len[f] >= kJobBigFileBytes ? h->big : h->small).push_back(f);
    }
    h->tile_start[nfile] = t;
    h->slot_off[nfile] = so;
    h->ntiles = t;
    h->total_slots = so;
}

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t job_scratch_bytes(uint64_t ntiles, uint64_t cand_cap, uint64_t total_slots) {
    return a256((ntiles * kWinThreads + 1) * 4) + a256((ntiles + 1) * 4) + a256((ntiles + 1) * 8) +
           a256(cand_cap * 8 + 8) + a256(total_slots * 8 + 8) + a256(kJobNumWords * 8 + 64);
}

void job_scratch_carve(char *mem, uint64_t ntiles, uint64_t cand_cap, uint64_t total_slots,
                       JobScratch *sc) {
    size_t off = 0;
    auto take = [&](size_t bytes) { char *p = mem + off; off += a256(bytes); return p; };
    sc->bitmap = (uint32_t *)take((ntiles * kWinThreads + 1) * 4);
    sc->tile_cnt = (uint32_t *)take((ntiles + 1) * 4);
    sc->tile_off = (uint64_t *)take((ntiles + 1) * 8);
    sc->cands = (uint64_t *)take(cand_cap * 8 + 8);
    sc->cand_cap = cand_cap;
    sc->tasks = (uint64_t *)take(total_slots * 8 + 8);
    char *w = take(kJobNumWords * 8 + 64);
    sc->words = (unsigned long long *)w;
    sc->err = (int *)(w + kJobNumWords * 8);
}

int enqueue_cdc_job(const JobDev &j, const JobScratch &sc, const hg_cdc_params &p, int algo,
                    const JobTuning &tn, int num_sms, uint64_t *d_ends, uint64_t *d_counts,
                    uint8_t *d_digests, cudaStream_t s) {
    if (cudaMemsetAsync(sc.words, 0, kJobNumWords * 8, s) != cudaSuccess ||
        (j.nfile && cudaMemsetAsync(d_counts, 0, (size_t)j.nfile * 8, s) != cudaSuccess))
        return HG_ECUDA;
    int r;
    if (j.ntiles) {
        const uint32_t mask = p.mask_bits >= 32 ? 0xffffffffu : ((1u << p.mask_bits) - 1u);
        const int grid = (int)std::min<uint64_t>(j.ntiles, (uint64_t)num_sms * tn.window_ctas);
        unsigned long long *ctr = sc.words + kJobTileCtr;
        if (p.window_hash == HG_WIN_RABIN) {
            if (p.window < 1 || p.window > (uint32_t)rabin::kPre) return HG_EUNSUPPORTED;
            const uint64_t groups = (j.ntiles + rabin::kTilesPerGroup - 1) / rabin::kTilesPerGroup;
            const int rgrid = (int)std::min<uint64_t>(groups, (uint64_t)num_sms * 2);
            switch (p.window) {
#define HG_JR(w)                                                                                \
    case w: launch_job_rabin_t<w>(rgrid, j, w, mask, p.magic, sc.bitmap, sc.tile_cnt, s); break;
                HG_JR(16) HG_JR(20) HG_JR(24) HG_JR(32) HG_JR(48) HG_JR(64)
#undef HG_JR
                default:
                    launch_job_rabin_t<0>(rgrid, j, p.window, mask, p.magic, sc.bitmap, sc.tile_cnt, s);
            }
        } else if (tn.window_ctas == 0) {
            // one-warp CTAs over the tiles' spans; their counts are added up
            if (cudaMemsetAsync(sc.tile_cnt, 0, (size_t)j.ntiles * 4, s) != cudaSuccess) return HG_ECUDA;
            switch (p.window) {
#define HG_JS(w)                                                                                \
    case w: launch_job_window_span_t<w>(j, w, mask, p.magic, sc.bitmap, sc.tile_cnt, sc.err, s); break;
                HG_JS(16) HG_JS(20) HG_JS(24) HG_JS(32) HG_JS(48)
#undef HG_JS
                default:
                    launch_job_window_span_t<0>(j, p.window, mask, p.magic, sc.bitmap, sc.tile_cnt,
                                                sc.err, s);
            }
        } else switch (p.window) {
#define HG_JW(w)                                                                                \
    case w:                                                                                     \
        launch_job_window_t<w>(grid, j, w, mask, p.magic, sc.bitmap, sc.tile_cnt, ctr, sc.err, s); \
        break;
            HG_JW(16) HG_JW(20) HG_JW(24) HG_JW(32) HG_JW(48)
#undef HG_JW
            default:
                launch_job_window_t<0>(grid, j, p.window, mask, p.magic, sc.bitmap, sc.tile_cnt,
                                       ctr, sc.err, s);
        }
        if ((r = launch_scan_tiles(sc.tile_cnt, j.ntiles, sc.tile_off, sc.tile_off + j.ntiles, s)))
            return r;
        k_job_compact<<<j.ntiles, kWinThreads, 0, s>>>(j, sc.bitmap, sc.tile_cnt, sc.tile_off,
                                                       sc.cands, sc.cand_cap);
    } else if (cudaMemsetAsync(sc.tile_off, 0, 8, s) != cudaSuccess) {
        return HG_ECUDA;
    }
    if (j.nsmall)
        k_job_select_small<<<(j.nsmall + 127) / 128, 128, 0, s>>>(
            j, sc.tile_off, sc.cands, sc.cand_cap, sc.bitmap, p.min_chunk, p.max_chunk, d_ends,
            d_counts, sc.words);
    if (j.nbig)
        k_job_select_big<<<j.nbig, kSelThreads, 0, s>>>(j, sc.tile_off, sc.cands, sc.cand_cap,
                                                       sc.bitmap, p.min_chunk, p.max_chunk, d_ends,
                                                       d_counts, sc.words);
    if (j.nfile) {
        unsigned long long *hist = sc.words + kJobHist, *cursor = sc.words + kJobHist + kLenBuckets;
        k_job_hist<<<j.nfile, 128, 0, s>>>(j, d_ends, d_counts, hist);
        k_job_hist_scan<<<1, 32, 0, s>>>(hist, cursor);
        k_job_tasks<<<j.nfile, 128, 0, s>>>(j, d_ends, d_counts, cursor, sc.tasks);
    }
    const int hgrid = num_sms * tn.hash_ctas;
    const size_t smem = stage_bytes((unsigned)tn.hash_threads);
    if (smem <= kStageSmemMax) {
        const void *k = algo == HG_MD5 ? (const void *)k_job_hash<Md5Chain, true>
                                       : (const void *)k_job_hash<Sha1, true>;
        if (allow_dyn_smem(k, smem) != cudaSuccess) return HG_ECUDA;
        if (algo == HG_MD5)
            k_job_hash<Md5Chain, true><<<hgrid, tn.hash_threads, smem, s>>>(j, d_ends, sc.tasks, sc.words,
                                                                           d_digests, sc.err);
        else
            k_job_hash<Sha1, true><<<hgrid, tn.hash_threads, smem, s>>>(j, d_ends, sc.tasks, sc.words,
                                                                       d_digests, sc.err);
    } else if (algo == HG_MD5) {
        k_job_hash<Md5Chain, false><<<hgrid, tn.hash_threads, 0, s>>>(j, d_ends, sc.tasks, sc.words,
                                                                       d_digests, sc.err);
    } else {
        k_job_hash<Sha1, false><<<hgrid, tn.hash_threads, 0, s>>>(j, d_ends, sc.tasks, sc.words,
                                                                   d_digests, sc.err);
    }
    return cuda_status(cudaGetLastError());
}

}  // namespace hg
