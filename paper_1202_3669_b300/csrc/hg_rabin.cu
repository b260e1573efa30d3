// Rabin fingerprint window hash: the variant window of content-defined
// chunking (HG_WIN_RABIN).
//
// Sec. 2.1 cites LBFS for content-based chunking; LBFS fingerprints its
// windows with Rabin's scheme rather than a cryptographic digest. The
// fingerprint of a byte string is its polynomial over GF(2) (bytes most
// significant first, bit 7 high) modulo the irreducible degree-31 polynomial
// HG_RABIN_POLY. The test on the fingerprint and everything downstream
// (compaction, min/max selection, per-chunk digests) are those of the MD5
// window.
//
// Unlike the MD5 window, the fingerprint rolls: with f the remainder of the
// window ending at p - 1 (W bytes),
//     f' = (f x^8 + b_p + b_{p-W} x^(8W)) mod P
//        = ((f << 8) | b_p) ^ T[f >> 23] ^ U[b_{p-W}]
// where T[t] = t x^31 mod P (plus bit 31 set to t's bit 0, which cancels the
// bit the 32-bit shift keeps) and U[b] = b x^(8W) mod P. A thread rolls along
// 128 consecutive window ends after W warm-up steps over the bytes before
// them. T and U (256 words each) are built by each CTA and replicated 32 times
// in shared memory, [value][lane], so every lane reads its own bank: the two
// lookups per byte never conflict. The kernel is persistent (one CTA per SM
// slot, groups of 4 tiles pulled in a grid-stride loop) so the tables are
// built once per CTA.
#include "hg_internal.h"

namespace hg {
namespace {

constexpr uint32_t kPoly = HG_RABIN_POLY;
constexpr int kRThreads = 256;
constexpr int kRStrip = 128;                                   // window ends per thread
constexpr int kRPre = 64;                                      // bytes loaded before a strip
constexpr uint64_t kRGroup = (uint64_t)kRThreads * kRStrip;    // 32 KiB of window ends
constexpr uint32_t kTilesPerGroup = (uint32_t)(kRGroup / kWinTile);
constexpr int kRCtasPerSm = 3;
constexpr size_t kRSmem = 2 * 256 * 32 * sizeof(uint32_t);     // T and U, 32 replicas each

static_assert(kRGroup % kWinTile == 0, "a group is whole tiles");
static_assert(kWinTile / kRStrip == 64, "two warps per tile");

// (f << 8) | byte k of w, in one byte permute: result bytes = {w.k, f.0, f.1, f.2}
__device__ __forceinline__ uint32_t shift_in(uint32_t f, uint32_t w, int k) {
    return __byte_perm(f, w, 0x2100u | (uint32_t)(4 + k));
}

// One rolling step: fingerprint of the window ending at the new byte, given
// the byte-shifted state s = (f << 8) | b_in, f's top byte index, and the
// byte leaving the window. T and U are the lane's replicas.
__device__ __forceinline__ uint32_t roll(uint32_t s, uint32_t top, uint32_t out,
                                         const uint32_t *__restrict__ T,
                                         const uint32_t *__restrict__ U) {
    return s ^ T[top << 5] ^ U[out << 5];
}

template <int W>
__global__ void __launch_bounds__(kRThreads, kRCtasPerSm)
    k_window_rabin(const uint8_t *__restrict__ in, uint64_t n, uint32_t wrt, uint32_t mask,
                   uint32_t magic, uint32_t *__restrict__ bitmap, uint32_t *__restrict__ tile_cnt,
                   uint32_t tile0, uint64_t ntiles) {
    extern __shared__ __align__(16) uint32_t tabs[];
    __shared__ uint32_t warp_cnt[kRThreads / 32];
    const uint32_t wlen = W ? (uint32_t)W : wrt;
    const int t = threadIdx.x, lane = t & 31;

    // T[v] = v x^31 mod P, bit 31 = v's bit 0; thread t builds entry t and
    // writes its 32 replicas in rotated order (one bank per lane per store)
    {
        uint32_t r = (uint32_t)t;
        for (int i = 0; i < 31; i++) {
            r <<= 1;
            if (r & 0x80000000u) r ^= kPoly;
        }
        r ^= ((uint32_t)t & 1u) << 31;
        for (int l = 0; l < 32; l++) tabs[t * 32 + ((l + lane) & 31)] = r;
    }
    __syncthreads();
    // U[b] = b x^(8W) mod P: W byte steps from b, with T
    {
        uint32_t r = (uint32_t)t;
        for (uint32_t i = 0; i < wlen; i++) r = (r << 8) ^ tabs[(r >> 23) * 32 + lane];
        for (int l = 0; l < 32; l++) tabs[256 * 32 + t * 32 + ((l + lane) & 31)] = r;
    }
    __syncthreads();
    const uint32_t *T = tabs + lane;
    const uint32_t *U = tabs + 256 * 32 + lane;

    const uint64_t nwords = (n + 31) / 32;
    const uint64_t ngroups = (ntiles + kTilesPerGroup - 1) / kTilesPerGroup;
    const bool aligned = (reinterpret_cast<uintptr_t>(in) & 15) == 0;
    const uint32_t sub = (uint32_t)t >> 6;                      // tile within the group
    for (uint64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const bool active = g * kTilesPerGroup + sub < ntiles;
        const uint64_t a = ((uint64_t)tile0 + g * kTilesPerGroup) * kWinTile + (uint64_t)t * kRStrip;
        uint32_t bits[4] = {0, 0, 0, 0};
        if (active && a < n) {
            if (W && aligned && a >= (uint64_t)kRPre && a + kRStrip <= n) {
                // interior strip: bytes [a - 64, a + 128) in registers, all
                // byte indexes below are compile-time constants
                uint32_t w[(kRPre + kRStrip) / 4];
                const uint4 *p4 = reinterpret_cast<const uint4 *>(in + a - kRPre);
#pragma unroll
                for (int i = 0; i < (kRPre + kRStrip) / 16; i++) {
                    const uint4 v = __ldg(p4 + i);
                    w[4 * i] = v.x; w[4 * i + 1] = v.y; w[4 * i + 2] = v.z; w[4 * i + 3] = v.w;
                }
                uint32_t f = 0;
#pragma unroll
                for (int i = kRPre - W; i < kRPre; i++)                 // warm-up: W bytes in
                    f = shift_in(f, w[i >> 2], i & 3) ^ T[(f >> 23) << 5];
#pragma unroll
                for (int m = 0; m < kRStrip; m++) {
                    const int i = kRPre + m, o = kRPre + m - W;
                    const uint32_t ob = (w[o >> 2] >> (8 * (o & 3))) & 0xffu;
                    f = roll(shift_in(f, w[i >> 2], i & 3), f >> 23, ob, T, U);
                    bits[m >> 5] |= (uint32_t)((f & mask) == magic) << (m & 31);
                }
            } else {
                // edges, unaligned input, or a window length without a
                // specialisation: byte loads, bytes outside [0, n) read as 0
                // (a leading zero byte does not change a polynomial)
                auto ld = [&](int64_t q) -> uint32_t {
                    return (q >= 0 && (uint64_t)q < n) ? (uint32_t)in[q] : 0u;
                };
                uint32_t f = 0;
                for (int64_t q = (int64_t)a - (int64_t)wlen; q < (int64_t)a; q++)
                    f = ((f << 8) | ld(q)) ^ T[(f >> 23) << 5];
                for (int m = 0; m < kRStrip; m++) {
                    const uint64_t pos = a + (uint64_t)m;
                    if (pos >= n) break;
                    const uint32_t ob = ld((int64_t)pos - (int64_t)wlen);
                    f = roll((f << 8) | ld((int64_t)pos), f >> 23, ob, T, U);
                    if (pos + 1 >= wlen && (f & mask) == magic) bits[m >> 5] |= 1u << (m & 31);
                }
            }
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
    bool ready = false;
    int sms = 0;
};
RabinDev g_rdev[64];

template <int W>
cudaError_t opt_in() {
    return cudaFuncSetAttribute(k_window_rabin<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kRSmem);
}

template <int W>
int launch_rabin_t(const uint8_t *d_in, uint64_t n, uint32_t w, uint32_t mask, uint32_t magic,
                   uint32_t *d_bitmap, uint32_t *d_tile_cnt, uint32_t tile0, uint64_t ntiles,
                   cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HG_ECUDA;
    if (dev < 0 || dev >= 64) return HG_EUNSUPPORTED;
    int r;
    if (!g_rdev[dev].ready && (r = rabin_prepare())) return r;
    const uint64_t ngroups = (ntiles + kTilesPerGroup - 1) / kTilesPerGroup;
    const uint64_t slots = (uint64_t)g_rdev[dev].sms * kRCtasPerSm;
    const unsigned grid = (unsigned)(ngroups < slots ? ngroups : slots);
    k_window_rabin<W><<<grid, kRThreads, kRSmem, s>>>(d_in, n, w, mask, magic, d_bitmap, d_tile_cnt,
                                                      tile0, ntiles);
    return cuda_status(cudaGetLastError());
}

}  // namespace

int rabin_prepare() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HG_ECUDA;
    if (dev < 0 || dev >= 64) return HG_EUNSUPPORTED;
    if (g_rdev[dev].ready) return HG_OK;
    int sms = 0;
    if (opt_in<0>() || opt_in<16>() || opt_in<20>() || opt_in<24>() || opt_in<32>() ||
        opt_in<48>() || opt_in<64>() ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return HG_ECUDA;
    }
    g_rdev[dev].sms = sms;
    g_rdev[dev].ready = true;
    return HG_OK;
}

int launch_window_rabin_range(const uint8_t *d_in, uint64_t n, const hg_cdc_params &p,
                              uint32_t *d_bitmap, uint32_t *d_tile_cnt, uint32_t tile0,
                              uint64_t ntiles, cudaStream_t s) {
    if (ntiles == 0) return HG_OK;
    if (p.window < 1 || p.window > (uint32_t)kRPre) return HG_EUNSUPPORTED;
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
