// The MD5 window hash over a single buffer (the dominant kernel of chunking).
//
// Sec. 2.1 ("Content-based chunking") and Sec. 3.2.2: a small window is hashed
// with MD5 at every byte offset, independently per window, and a boundary is
// declared where the hash matches a predefined value. This file holds only
// that kernel and its launchers (its counters are recorded against this
// source), the Rabin variant is dispatched from here.
#include "hg_device.cuh"
#include "hg_internal.h"
#include "hg_window.cuh"

namespace hg {
namespace {

// One CTA covers kWinTile consecutive window ends; thread t owns ends
// [tile + 32t, tile + 32t + 32) and so exactly bitmap word tile/32 + t.
// The tile and a 64-byte halo before it are staged in shared memory, by one
// bulk asynchronous copy (TMA) for interior tiles of a 16-byte aligned input
// and by guarded byte loads at the edges. `one` is 1 (the run-time 1 of the
// FMA-pipe adds).
template <int W>
__global__ void __launch_bounds__(kWinThreads) k_window_bitmap(const uint8_t *__restrict__ in,
                                                               uint64_t n, uint32_t wrt,
                                                               uint32_t mask, uint32_t magic,
                                                               uint32_t *__restrict__ bitmap,
                                                               uint32_t *__restrict__ tile_cnt,
                                                               int *err, uint32_t tile0,
                                                               uint32_t one) {
    const uint32_t wlen = W ? (uint32_t)W : wrt;
    __shared__ __align__(128) uint8_t sbuf[kSmemBytes];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t warp_cnt[kWinThreads / 32];

    const int t = threadIdx.x;
    const uint32_t tix = blockIdx.x + tile0;
    const uint64_t tile = (uint64_t)tix * kWinTile;
    const bool fast = ((reinterpret_cast<uintptr_t>(in) & 15) == 0) && tile >= (uint64_t)kHalo &&
                      tile + kWinTile <= n;
    if (t < 4) reinterpret_cast<uint32_t *>(sbuf + kHalo + kWinTile)[t] = 0;
    bool timed_out = false;
    if (fast) {
        const uint32_t mb = smem_u32(&mbar);
        if (t == 0) mbar_init(mb);
        __syncthreads();
        if (t == 0) bulk_load(smem_u32(sbuf), in + tile - kHalo, (uint32_t)(kHalo + kWinTile), mb);
        timed_out = !mbar_wait(mb, 0);
        if (timed_out) {
            // keep polling (bounded) so the copy cannot land after the CTA left
            atomicCAS(err, 0, (int)HG_ETIMEDOUT);
            mbar_wait(mb, 0);
        }
    } else {
        for (int i = t; i < kHalo + (int)kWinTile; i += kWinThreads) {
            const int64_t g = (int64_t)tile - kHalo + i;
            sbuf[i] = (g >= 0 && (uint64_t)g < n) ? in[g] : (uint8_t)0;
        }
    }
    if (__syncthreads_or(timed_out)) return;

    const uint64_t p0 = tile + 32u * (uint64_t)t;
    const uint32_t bits = clip_bits(window_bits32<W>(sbuf, t, wlen, mask, magic, one), p0, wlen, n);
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
        if (HG_DOK((uint64_t)tix * kWinTile < n, err)) tile_cnt[tix] = s;
    }
}

template <int W>
void launch_window_t(const uint8_t *d_in, uint64_t n, uint32_t w, uint32_t mask, uint32_t magic,
                     uint32_t *d_bitmap, uint32_t *d_tile_cnt, uint64_t ntiles, cudaStream_t s,
                     int *d_err, uint32_t tile0) {
    k_window_bitmap<W><<<(unsigned)ntiles, kWinThreads, 0, s>>>(d_in, n, w, mask, magic, d_bitmap,
                                                                 d_tile_cnt, d_err, tile0, 1u);
}

}  // namespace

int launch_window_bitmap(const uint8_t *d_in, uint64_t n, const hg_cdc_params &p,
                         uint32_t *d_bitmap, uint32_t *d_tile_cnt, cudaStream_t s, int *d_err) {
    return launch_window_range(d_in, n, p, d_bitmap, d_tile_cnt, 0, (n + kWinTile - 1) / kWinTile, s,
                               d_err);
}

int launch_window_range(const uint8_t *d_in, uint64_t n, const hg_cdc_params &p,
                        uint32_t *d_bitmap, uint32_t *d_tile_cnt, uint32_t tile0, uint64_t ntiles,
                        cudaStream_t s, int *d_err) {
    if (ntiles == 0) return HG_OK;
    if (p.window_hash == HG_WIN_RABIN)
        return launch_window_rabin_range(d_in, n, p, d_bitmap, d_tile_cnt, tile0, ntiles, s);
    if (p.window_hash != HG_WIN_MD5) return HG_EINVAL;
    const uint32_t mask = p.mask_bits >= 32 ? 0xffffffffu : ((1u << p.mask_bits) - 1u);
    if (p.window < 1 || p.window > 55) return HG_EUNSUPPORTED;
    switch (p.window) {
#define HG_W(w)                                                                                \
    case w:                                                                                    \
        launch_window_t<w>(d_in, n, w, mask, p.magic, d_bitmap, d_tile_cnt, ntiles, s, d_err, tile0); \
        break;
        HG_W(16) HG_W(20) HG_W(24) HG_W(32) HG_W(48)
#undef HG_W
        default:
            launch_window_t<0>(d_in, n, p.window, mask, p.magic, d_bitmap, d_tile_cnt, ntiles, s,
                               d_err, tile0);
    }
    return cuda_status(cudaGetLastError());
}

}  // namespace hg
