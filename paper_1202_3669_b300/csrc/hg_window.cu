// The MD5 window hash over a single buffer (the dominant kernel of chunking).
//
// Sec. 2.1 ("Content-based chunking") and Sec. 3.2.2: a small window is hashed
// with MD5 at every byte offset, independently per window, and a boundary is
// declared where the hash matches a predefined value. This file holds only
// that kernel and its launchers (its counters are recorded against this
// source), the Rabin variant is dispatched from here.
#include <algorithm>

#include "hg_device.cuh"
#include "hg_internal.h"
#include "hg_window.cuh"

namespace hg {
namespace {

// One CTA is one warp and covers kWinSpan = 1024 consecutive window ends (an
// eighth of a tile); lane l owns ends [lo + 32l, lo + 32l + 32) and so exactly
// bitmap word lo/32 + l. The span and a 64-byte halo before it are staged in
// shared memory by one bulk asynchronous copy (TMA) for interior spans of a
// 16-byte aligned input and by guarded byte loads at the edges. The warp adds
// its candidate count to its tile's count (zeroed before the launch).
//
// Why one warp per CTA (measured on a 64 MiB pass, 20-byte window): with eight
// warps per CTA the warps of a CTA finish far apart under the scheduler's
// priorities, and ~40 % of resident warps sat at the CTA's final barrier
// (0.651 ms); one-warp CTAs let the hardware refill each SM slot as soon as its
// warp is done and leave ptxas ~56 registers for interleaving the four
// windows of a group: 0.616 ms with the pipe policies below, against 0.630 ms
// with the data-word steps' adds on the ALU and 0.640-0.68 ms for two- to
// eight-warp CTAs at 40-64 registers.
template <int W>
__global__ void __launch_bounds__(32, 32) k_window_bitmap(const uint8_t *__restrict__ in,
                                                          uint64_t n, uint32_t wrt, uint32_t mask,
                                                          uint32_t magic,
                                                          uint32_t *__restrict__ bitmap,
                                                          uint32_t *__restrict__ tile_cnt,
                                                          int *err, uint64_t span0, uint32_t one) {
    const uint32_t wlen = W ? (uint32_t)W : wrt;
    __shared__ __align__(128) uint8_t sbuf[kHalo + kWinSpan + 16];
    __shared__ __align__(8) uint64_t mbar;

    const int t = threadIdx.x;
    const uint64_t lo = (span0 + blockIdx.x) * (uint64_t)kWinSpan;
    const bool fast = ((reinterpret_cast<uintptr_t>(in) & 15) == 0) && lo >= (uint64_t)kHalo &&
                      lo + kWinSpan <= n;
    if (t < 4) reinterpret_cast<uint32_t *>(sbuf + kHalo + kWinSpan)[t] = 0;
    bool timed_out = false;
    if (fast) {
        const uint32_t mb = smem_u32(&mbar);
        if (t == 0) mbar_init(mb);
        __syncwarp();
        if (t == 0) bulk_load(smem_u32(sbuf), in + lo - kHalo, (uint32_t)(kHalo + kWinSpan), mb);
        timed_out = !mbar_wait(mb, 0);
        if (timed_out) {
            // keep polling (bounded) so the copy cannot land after the CTA left
            atomicCAS(err, 0, (int)HG_ETIMEDOUT);
            mbar_wait(mb, 0);
        }
    } else {
        for (int i = t; i < kHalo + kWinSpan; i += 32) {
            const int64_t g = (int64_t)lo - kHalo + i;
            sbuf[i] = (g >= 0 && (uint64_t)g < n) ? in[g] : (uint8_t)0;
        }
    }
    if (__any_sync(0xffffffffu, timed_out)) return;
    __syncwarp();

    const uint64_t p0 = lo + 32u * (uint64_t)t;
    const uint32_t bits = clip_bits(window_bits32<W>(sbuf, t, wlen, mask, magic, one), p0, wlen, n);
    const uint64_t nwords = (n + 31) / 32;
    const uint64_t widx = lo / 32 + t;
    if (widx < nwords) bitmap[widx] = bits;
    const uint32_t c = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(bits));
    if (t == 0 && c && HG_DOK(lo < n, err)) atomicAdd(&tile_cnt[lo / kWinTile], c);
}

template <int W>
void launch_window_t(const uint8_t *d_in, uint64_t n, uint32_t w, uint32_t mask, uint32_t magic,
                     uint32_t *d_bitmap, uint32_t *d_tile_cnt, uint64_t span0, uint64_t nspans,
                     cudaStream_t s, int *d_err) {
    k_window_bitmap<W><<<(unsigned)nspans, 32, 0, s>>>(d_in, n, w, mask, magic, d_bitmap, d_tile_cnt,
                                                      d_err, span0, 1u);
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
    // the warps add their counts into the tiles' counts
    if (cudaMemsetAsync(d_tile_cnt + tile0, 0, ntiles * sizeof(uint32_t), s) != cudaSuccess)
        return HG_ECUDA;
    // spans of the tiles that hold window ends below n (a last partial tile has fewer)
    const uint64_t lo = (uint64_t)tile0 * kWinTile;
    const uint64_t hi = std::min<uint64_t>((uint64_t)(tile0 + ntiles) * kWinTile, n);
    if (hi <= lo) return HG_OK;
    const uint64_t span0 = lo / kWinSpan, nspans = (hi - lo + kWinSpan - 1) / kWinSpan;
    switch (p.window) {
#define HG_W(w)                                                                                \
    case w:                                                                                    \
        launch_window_t<w>(d_in, n, w, mask, p.magic, d_bitmap, d_tile_cnt, span0, nspans, s, d_err); \
        break;
        HG_W(16) HG_W(20) HG_W(24) HG_W(32) HG_W(48)
#undef HG_W
        default:
            launch_window_t<0>(d_in, n, p.window, mask, p.magic, d_bitmap, d_tile_cnt, span0, nspans, s,
                               d_err);
    }
    return cuda_status(cudaGetLastError());
}

}  // namespace hg
