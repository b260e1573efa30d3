// Content-defined chunking kernels: window hashes, compaction, selection.
//
// Sec. 2.1 ("Content-based chunking") and Sec. 3.2.2: a small window is hashed
// with MD5 at every byte offset, independently per window, and a boundary is
// declared where the hash matches a predefined value. The paper leaves the
// boundary scan to the CPU because it could not synchronise all GPU threads;
// here the scan is done on the device by compaction and a selection kernel.
#include "hg_device.cuh"
#include "hg_internal.h"

namespace hg {
namespace {

constexpr int kHalo = 64;                              // >= window - 1, multiple of 16
constexpr int kSmemBytes = kHalo + (int)kWinTile + 16; // + a zeroed 16-byte pad
constexpr long kWaitLimit = 1L << 22;                  // bounded mbarrier polling

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// MD5 of one window given its data words d[] (little-endian, the last word may
// carry bytes past the window, which are masked). Only word A of the final
// state is formed: the window test reads the first four digest bytes.
template <int W>
__device__ __forceinline__ uint32_t window_a(const uint32_t (&d)[(W + 3) / 4]) {
    constexpr int NW = (W + 3) / 4;
    uint32_t M[16];
#pragma unroll
    for (int i = 0; i < 16; i++) M[i] = 0;
#pragma unroll
    for (int i = 0; i < NW; i++) M[i] = d[i];
    if (W % 4 == 0) {
        M[W / 4] = 0x80u;                             // padding marker after the data
    } else {
        constexpr uint32_t keep = (1u << (8 * (W % 4))) - 1u;
        M[NW - 1] = (d[NW - 1] & keep) | (0x80u << (8 * (W % 4)));
    }
    M[14] = (uint32_t)W * 8u;                         // bit length, little-endian
    uint32_t a = kMd5A, b = kMd5B, c = kMd5C, dd = kMd5D;
    md5_rounds<false>(a, b, c, dd, M);
    return a + kMd5A;
}

// Window number S (0..6) of a group, counted in bytes from word cur[0].
template <int W, int S>
__device__ __forceinline__ uint32_t window_at(const uint32_t (&cur)[(W + 3) / 4 + 2]) {
    constexpr int NW = (W + 3) / 4, SH = S & 3, WO = S >> 2;
    uint32_t d[NW];
#pragma unroll
    for (int k = 0; k < NW; k++)
        d[k] = SH == 0 ? cur[WO + k] : __funnelshift_r(cur[WO + k], cur[WO + k + 1], 8 * SH);
    return window_a<W>(d);
}

// Window hash for a window length known only at run time (any 1..55): the
// message words are gathered byte by byte from shared memory.
__device__ __forceinline__ uint32_t window_a_rt(const uint8_t *sbuf, int start, int w) {
    uint32_t M[16];
#pragma unroll
    for (int i = 0; i < 14; i++) {
        uint32_t x = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int k = 4 * i + j;
            const uint32_t byte = k < w ? (uint32_t)sbuf[start + k] : (k == w ? 0x80u : 0u);
            x |= byte << (8 * j);
        }
        M[i] = x;
    }
    M[14] = (uint32_t)w * 8u;
    M[15] = 0;
    uint32_t a = kMd5A, b = kMd5B, c = kMd5C, d = kMd5D;
    md5_rounds<false>(a, b, c, d, M);
    return a + kMd5A;
}

// One CTA covers kWinTile consecutive window ends; thread t owns ends
// [tile + 32t, tile + 32t + 32) and so exactly bitmap word tile/32 + t.
// The tile and a 64-byte halo before it are staged in shared memory, by one
// bulk asynchronous copy (TMA) for interior tiles of a 16-byte aligned input
// and by guarded byte loads at the edges.
template <int W>
__global__ void __launch_bounds__(kWinThreads) k_window_bitmap(const uint8_t *__restrict__ in,
                                                               uint64_t n, uint32_t wrt,
                                                               uint32_t mask,
                                                               uint32_t magic,
                                                               uint32_t *__restrict__ bitmap,
                                                               uint32_t *__restrict__ tile_cnt,
                                                               int *err) {
    constexpr int NW = W ? (W + 3) / 4 : 1;
    constexpr int OFF = kHalo - (W ? W - 1 : 0);      // local byte of window 0's start
    constexpr int B0 = OFF / 4, R0 = OFF % 4;
    const uint32_t wlen = W ? (uint32_t)W : wrt;
    __shared__ __align__(128) uint8_t sbuf[kSmemBytes];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t warp_cnt[kWinThreads / 32];

    const int t = threadIdx.x;
    const uint64_t tile = (uint64_t)blockIdx.x * kWinTile;
    const bool fast = ((reinterpret_cast<uintptr_t>(in) & 15) == 0) && tile >= (uint64_t)kHalo &&
                      tile + kWinTile <= n;
    if (t < 4) reinterpret_cast<uint32_t *>(sbuf + kHalo + kWinTile)[t] = 0;
    bool load_ok = true;
    if (fast) {
        const uint32_t mb = smem_u32(&mbar);
        if (t == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (t == 0) {
            const uint32_t bytes = (uint32_t)(kHalo + kWinTile);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb),
                         "r"(bytes)
                         : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                "[%3];" ::"r"(smem_u32(sbuf)),
                "l"(in + tile - kHalo), "r"(bytes), "r"(mb)
                : "memory");
        }
        bool done = false;
        for (long it = 0; it < kWaitLimit && !done; it++) done = mbar_try_wait(mb, 0);
        if (!done) {
            // give up on this tile; keep polling (bounded) so the copy cannot
            // land in shared memory after the CTA has left
            atomicCAS(err, 0, (int)HG_ETIMEDOUT);
            for (long it = 0; it < kWaitLimit && !done; it++) done = mbar_try_wait(mb, 0);
            load_ok = false;
        }
    } else {
        for (int i = t; i < kHalo + (int)kWinTile; i += kWinThreads) {
            const int64_t g = (int64_t)tile - kHalo + i;
            sbuf[i] = (g >= 0 && (uint64_t)g < n) ? in[g] : (uint8_t)0;
        }
    }
    __syncthreads();
    if (!load_ok) return;

    uint32_t bits = 0;
    if constexpr (W > 0) {
        const uint32_t *sw = reinterpret_cast<const uint32_t *>(sbuf);
        uint32_t cur[NW + 2];
#pragma unroll
        for (int i = 0; i < NW + 2; i++) cur[i] = sw[8 * t + B0 + i];
#pragma unroll 1
        for (int g = 0; g < 8; g++) {
            const uint32_t h0 = window_at<W, R0 + 0>(cur);
            const uint32_t h1 = window_at<W, R0 + 1>(cur);
            const uint32_t h2 = window_at<W, R0 + 2>(cur);
            const uint32_t h3 = window_at<W, R0 + 3>(cur);
            const uint32_t nib = (uint32_t)((h0 & mask) == magic) |
                                 ((uint32_t)((h1 & mask) == magic) << 1) |
                                 ((uint32_t)((h2 & mask) == magic) << 2) |
                                 ((uint32_t)((h3 & mask) == magic) << 3);
            bits |= nib << (4 * g);
#pragma unroll
            for (int i = 0; i < NW + 1; i++) cur[i] = cur[i + 1];
            cur[NW + 1] = sw[8 * t + B0 + g + NW + 2];       // stays inside the padded tile
        }
    } else {
        const int first = kHalo + 32 * t - (int)(wlen - 1);
#pragma unroll 1
        for (int j = 0; j < 32; j++)
            bits |= (uint32_t)((window_a_rt(sbuf, first + j, (int)wlen) & mask) == magic) << j;
    }
    // clear ends before the first full window and past the input
    const uint64_t p0 = tile + 32u * (uint64_t)t;
    const uint64_t lo = (uint64_t)(wlen - 1) > p0 ? (uint64_t)(wlen - 1) - p0 : 0;
    const uint64_t hi = n > p0 ? n - p0 : 0;
    if (lo >= 32 || hi == 0) bits = 0;
    else {
        if (lo) bits &= ~0u << lo;
        if (hi < 32) bits &= (1u << hi) - 1u;
    }
    const uint64_t nwords = (n + 31) / 32;
    const uint64_t widx = tile / 32 + t;
    if (widx < nwords) bitmap[widx] = bits;
    const uint32_t c = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(bits));
    if ((t & 31) == 0) warp_cnt[t >> 5] = c;
    __syncthreads();
    if (t == 0) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kWinThreads / 32; w++) s += warp_cnt[w];
        tile_cnt[blockIdx.x] = s;
    }
}

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

// Bitmap -> increasing cut positions. One CTA per window tile; tiles without
// candidates leave at once.
__global__ void __launch_bounds__(kWinThreads) k_compact(const uint32_t *__restrict__ bitmap,
                                                         uint64_t nwords,
                                                         const uint32_t *__restrict__ tile_cnt,
                                                         const uint64_t *__restrict__ tile_off,
                                                         uint64_t *__restrict__ cands,
                                                         uint64_t cap) {
    __shared__ uint32_t warp_sum[kWinThreads / 32];
    if (tile_cnt[blockIdx.x] == 0) return;
    const int t = threadIdx.x;
    const uint64_t widx = (uint64_t)blockIdx.x * kWinThreads + t;
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
    uint64_t idx = tile_off[blockIdx.x] + before;
    const uint64_t pos0 = widx * 32;
    while (w) {
        const int b = __ffs(w) - 1;
        w &= w - 1;
        if (idx < cap) cands[idx] = pos0 + b + 1;      // cut after the window's last byte
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

// Greedy min/max selection (one warp). Reads the sorted candidate list 32 at a
// time; if the list overflowed its capacity it scans the bitmap instead.
__global__ void k_select(const uint64_t *__restrict__ cands, const uint64_t *__restrict__ d_ncand,
                         uint64_t cand_cap, const uint32_t *__restrict__ bitmap, uint64_t n,
                         uint64_t mn, uint64_t mx, uint64_t *__restrict__ ends, uint64_t cap,
                         uint64_t *__restrict__ d_count) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32) return;
    const uint64_t ncand = *d_ncand;
    const bool use_list = ncand <= cand_cap;
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

template <int W>
void launch_window_t(const uint8_t *d_in, uint64_t n, uint32_t w, uint32_t mask, uint32_t magic,
                     uint32_t *d_bitmap, uint32_t *d_tile_cnt, uint64_t ntiles, cudaStream_t s,
                     int *d_err) {
    k_window_bitmap<W><<<(unsigned)ntiles, kWinThreads, 0, s>>>(d_in, n, w, mask, magic, d_bitmap,
                                                                 d_tile_cnt, d_err);
}

}  // namespace

int launch_window_bitmap(const uint8_t *d_in, uint64_t n, const hg_cdc_params &p,
                         uint32_t *d_bitmap, uint32_t *d_tile_cnt, cudaStream_t s, int *d_err) {
    const uint64_t ntiles = (n + kWinTile - 1) / kWinTile;
    if (ntiles == 0) return HG_OK;
    const uint32_t mask = p.mask_bits >= 32 ? 0xffffffffu : ((1u << p.mask_bits) - 1u);
    if (p.window < 1 || p.window > 55) return HG_EUNSUPPORTED;
    switch (p.window) {
#define HG_W(w)                                                                                \
    case w:                                                                                    \
        launch_window_t<w>(d_in, n, w, mask, p.magic, d_bitmap, d_tile_cnt, ntiles, s, d_err); \
        break;
        HG_W(16) HG_W(20) HG_W(24) HG_W(32) HG_W(48)
#undef HG_W
        default:
            launch_window_t<0>(d_in, n, p.window, mask, p.magic, d_bitmap, d_tile_cnt, ntiles, s,
                               d_err);
    }
    return cuda_status(cudaGetLastError());
}

int launch_compact(const uint32_t *d_bitmap, uint64_t n, const uint32_t *d_tile_cnt,
                   uint64_t *d_tile_off, uint64_t ntiles, uint64_t *d_cands, uint64_t cap,
                   uint64_t *d_count, cudaStream_t s) {
    if (ntiles == 0) return cuda_status(cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s));
    k_scan_tiles<<<1, 1024, 0, s>>>(d_tile_cnt, ntiles, d_tile_off, d_count);
    k_compact<<<(unsigned)ntiles, kWinThreads, 0, s>>>(d_bitmap, (n + 31) / 32, d_tile_cnt,
                                                       d_tile_off, d_cands, cap);
    return cuda_status(cudaGetLastError());
}

int launch_select(const uint64_t *d_cands, const uint64_t *d_ncand, uint64_t cand_cap,
                  const uint32_t *d_bitmap, uint64_t n, const hg_cdc_params &p, uint64_t *d_ends,
                  uint64_t cap, uint64_t *d_count, cudaStream_t s) {
    k_select<<<1, 32, 0, s>>>(d_cands, d_ncand, cand_cap, d_bitmap, n, p.min_chunk, p.max_chunk,
                              d_ends, cap, d_count);
    return cuda_status(cudaGetLastError());
}

}  // namespace hg
