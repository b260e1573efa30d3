// Rabin fingerprint window hash: the variant window of content-defined
// chunking (HG_WIN_RABIN), single-buffer kernel.
//
// Sec. 2.1 cites LBFS for content-based chunking; LBFS fingerprints its
// windows with Rabin's scheme rather than a cryptographic digest. The
// fingerprint and its rolling form are in hg_rabin.cuh; the test on it and
// everything downstream (compaction, min/max selection, per-chunk digests)
// are those of the MD5 window. The kernel is persistent (CTAs per SM as the
// tables and registers allow, groups of 4 tiles pulled in a grid-stride loop)
// so each CTA builds its tables once.
#include <atomic>
#include <mutex>

#include "hg_rabin.cuh"

namespace hg {
namespace {

using namespace rabin;

// An aligned input runs three CTAs per SM; any other alignment realigns each
// strip from 16-byte loads, which needs more registers: two.
template <bool GENERAL>
constexpr int ctas_per_sm() { return GENERAL ? 2 : 3; }

template <int W, bool GENERAL>
__global__ void __launch_bounds__(kThreads, ctas_per_sm<GENERAL>())
    k_window_rabin(const uint8_t *__restrict__ in, uint64_t n, uint32_t wrt, uint32_t mask,
                   uint32_t magic, uint32_t *__restrict__ bitmap, uint32_t *__restrict__ tile_cnt,
                   uint32_t tile0, uint64_t ntiles) {
    extern __shared__ __align__(16) uint32_t tabs[];
    __shared__ uint32_t warp_cnt[kThreads / 32];
    const uint32_t wlen = W ? (uint32_t)W : wrt;
    const int t = threadIdx.x, lane = t & 31;
    build_tables(tabs, wlen);
    const uint32_t *T = tabs + lane;
    const uint32_t *U = tabs + 256 * 32 + lane;

    const uint64_t nwords = (n + 31) / 32;
    const uint64_t ngroups = (ntiles + kTilesPerGroup - 1) / kTilesPerGroup;
    const uint32_t sub = (uint32_t)t >> 6;                      // tile within the group
    for (uint64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const bool active = g * kTilesPerGroup + sub < ntiles;
        const uint64_t a = ((uint64_t)tile0 + g * kTilesPerGroup) * kWinTile + (uint64_t)t * kStrip;
        uint32_t bits[4] = {0, 0, 0, 0};
        if (active && a < n) {
            strip_bits<W, GENERAL>(in, n, a, wlen, mask, magic, T, U, bits);
            const uint64_t w0 = a / 32;
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (w0 + j < nwords) bitmap[w0 + j] = bits[j];
        }
        const uint32_t c = __reduce_add_sync(0xffffffffu, (uint32_t)(__popc(bits[0]) + __popc(bits[1]) +
                                                                   __popc(bits[2]) + __popc(bits[3])));
        if (lane == 0) warp_cnt[t >> 5] = c;
        __syncthreads();
        if (t < (int)kTilesPerGroup && g * kTilesPerGroup + t < ntiles)
            tile_cnt[tile0 + g * kTilesPerGroup + t] = warp_cnt[2 * t] + warp_cnt[2 * t + 1];
        __syncthreads();
    }
}

// Per device: the kernels' shared-memory opt-in (64 KiB of tables) and the SM
// count, set up outside any stream capture (hg_init calls rabin_prepare).
struct RabinDev {
    std::atomic<bool> ready{false};   // set (release) after sms, read (acquire) before launches
    int sms = 0;
};
RabinDev g_rdev[64];
std::mutex g_rmu;                     // serialises the set-up of rabin_prepare

template <int W>
cudaError_t opt_in() {
    cudaError_t e = cudaFuncSetAttribute(k_window_rabin<W, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_window_rabin<W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kSmem);
}

template <int W>
int launch_rabin_t(const uint8_t *d_in, uint64_t n, uint32_t w, uint32_t mask, uint32_t magic,
                   uint32_t *d_bitmap, uint32_t *d_tile_cnt, uint32_t tile0, uint64_t ntiles,
                   cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HG_ECUDA;
    if (dev < 0 || dev >= 64) return HG_EUNSUPPORTED;
    int r;
    if (!g_rdev[dev].ready.load(std::memory_order_acquire) && (r = rabin_prepare())) return r;
    const bool general = (reinterpret_cast<uintptr_t>(d_in) & 15) != 0;
    const uint64_t ngroups = (ntiles + kTilesPerGroup - 1) / kTilesPerGroup;
    const uint64_t slots = (uint64_t)g_rdev[dev].sms * (general ? ctas_per_sm<true>() : ctas_per_sm<false>());
    const unsigned grid = (unsigned)(ngroups < slots ? ngroups : slots);
    if (general)
        k_window_rabin<W, true><<<grid, kThreads, kSmem, s>>>(d_in, n, w, mask, magic, d_bitmap,
                                                              d_tile_cnt, tile0, ntiles);
    else
        k_window_rabin<W, false><<<grid, kThreads, kSmem, s>>>(d_in, n, w, mask, magic, d_bitmap,
                                                               d_tile_cnt, tile0, ntiles);
    return cuda_status(cudaGetLastError());
}

}  // namespace

int rabin_prepare() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HG_ECUDA;
    if (dev < 0 || dev >= 64) return HG_EUNSUPPORTED;
    if (g_rdev[dev].ready.load(std::memory_order_acquire)) return HG_OK;
    std::lock_guard<std::mutex> lock(g_rmu);
    if (g_rdev[dev].ready.load(std::memory_order_acquire)) return HG_OK;
    int sms = 0;
    if (opt_in<0>() || opt_in<16>() || opt_in<20>() || opt_in<24>() || opt_in<32>() ||
        opt_in<48>() || opt_in<64>() || job_rabin_prepare() != HG_OK ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return HG_ECUDA;
    }
    g_rdev[dev].sms = sms;
    g_rdev[dev].ready.store(true, std::memory_order_release);
    return HG_OK;
}

int launch_window_rabin_range(const uint8_t *d_in, uint64_t n, const hg_cdc_params &p,
                              uint32_t *d_bitmap, uint32_t *d_tile_cnt, uint32_t tile0,
                              uint64_t ntiles, cudaStream_t s) {
    if (ntiles == 0) return HG_OK;
    if (p.window < 1 || p.window > (uint32_t)kPre) return HG_EUNSUPPORTED;
    const uint32_t mask = p.mask_bits >= 32 ? 0xffffffffu : ((1u << p.mask_bits) - 1u);
    switch (p.window) {
#define HG_RW(w) \
    case w: return launch_rabin_t<w>(d_in, n, w, mask, p.magic, d_bitmap, d_tile_cnt, tile0, ntiles, s);
        HG_RW(16) HG_RW(20) HG_RW(24) HG_RW(32) HG_RW(48) HG_RW(64)
#undef HG_RW
        default:
            return launch_rabin_t<0>(d_in, n, p.window, mask, p.magic, d_bitmap, d_tile_cnt, tile0,
                                     ntiles, s);
    }
}

}  // namespace hg
