// Chunk boundaries without any allocation: hg_cdc_boundaries_static.
//
// Some callers cannot call cudaMalloc. A storage write path may not be allowed
// to stall on the device-wide synchronisation that cudaMalloc and cudaFree can
// cause while other streams are busy; a process may hand all of its device
// memory to another allocator (a framework's caching allocator) that this
// library cannot draw from; a service may need its device footprint fixed at
// load time. For them this entry point runs the same kernels as
// hg_cdc_boundaries, with the scratch those kernels need (candidate bitmap,
// per-tile counts and offsets, candidate list) in one statically sized
// __device__ array instead of context-owned allocations. The caller still
// passes its own input and output buffers.
//
// The array lives in this file, so every GPU that loads the library holds it
// (about 3.1 MiB for the 16 MiB input maximum) until the process exits.
#include <mutex>

#include "hg_internal.h"

namespace hg {
namespace {

constexpr uint64_t kMaxBytes = HG_STATIC_MAX_BYTES;
constexpr uint64_t kMaxWords = kMaxBytes / 32;                 // bitmap words
constexpr uint64_t kMaxTiles = kMaxBytes / kWinTile;           // window tiles
constexpr uint64_t kMaxCands = cand_capacity(kMaxBytes);        // as hg_cdc_boundaries sizes it
static_assert(kMaxBytes % kWinTile == 0, "maximum must be a whole number of tiles");

// byte offsets of the pieces inside the array (each 256-byte aligned)
constexpr uint64_t kOffBitmap = 0;
constexpr uint64_t kOffTileCnt = kOffBitmap + kMaxWords * 4;
constexpr uint64_t kOffTileOff = kOffTileCnt + ((kMaxTiles * 4 + 255) / 256) * 256;
constexpr uint64_t kOffCands = kOffTileOff + ((kMaxTiles * 8 + 255) / 256) * 256;
constexpr uint64_t kOffWords = kOffCands + kMaxCands * 8;      // ncand (8 B) + error word (4 B)
constexpr uint64_t kScratchBytes = kOffWords + 256;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device. In host code `g_scratch` names a
// host-side shadow, not device memory, so kernels get the address obtained
// from cudaGetSymbolAddress on that device. The first call on a device also
// does every other per-device set-up the launched kernels need (the Rabin
// window kernels' shared-memory opt-in), so that one call made before any
// stream capture covers both window hashes.
constexpr int kMaxDevices = 64;
unsigned char *g_addr[kMaxDevices] = {};
std::mutex g_mu;

int scratch_address(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return HG_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        int r = rabin_prepare();
        if (r) return r;
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return HG_ECUDA;
        }
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return HG_OK;
}

// If a bounded wait in the window kernel gave up, the results are incomplete:
// mark the count so the caller cannot take them for a full answer.
__global__ void k_static_mark_error(const int *err, uint64_t *d_count) {
    if (threadIdx.x == 0 && *err != 0) *d_count = UINT64_MAX;
}

}  // namespace
}  // namespace hg

using namespace hg;

extern "C" int hg_cdc_boundaries_static(const uint8_t *d_in, uint64_t n, const hg_cdc_params *p,
                                        uint64_t *d_ends, uint64_t cap, uint64_t *d_count,
                                        void *stream) {
    if (!p || (p->window_hash != HG_WIN_MD5 && p->window_hash != HG_WIN_RABIN) || !d_count ||
        (cap && !d_ends))
        return HG_EINVAL;
    if (p->window < 1 || p->window > (p->window_hash == HG_WIN_RABIN ? 64u : 55u)) return HG_EUNSUPPORTED;
    if (p->mask_bits < 1 || p->mask_bits > 32) return HG_EINVAL;
    if (p->mask_bits < 32 && (p->magic >> p->mask_bits) != 0) return HG_EINVAL;
    if (p->min_chunk < 1 || p->min_chunk > p->max_chunk) return HG_EINVAL;
    if (n > kMaxBytes) return HG_ECAPACITY;                // input above the static maximum
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return cuda_status(cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s));
    if (!d_in) return HG_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HG_ECUDA;
    unsigned char *base = nullptr;
    int r = scratch_address(dev, &base);
    if (r) return r;
    uint32_t *bitmap = reinterpret_cast<uint32_t *>(base + kOffBitmap);
    uint32_t *tile_cnt = reinterpret_cast<uint32_t *>(base + kOffTileCnt);
    uint64_t *tile_off = reinterpret_cast<uint64_t *>(base + kOffTileOff);
    uint64_t *cands = reinterpret_cast<uint64_t *>(base + kOffCands);
    uint64_t *ncand = reinterpret_cast<uint64_t *>(base + kOffWords);
    int *err = reinterpret_cast<int *>(base + kOffWords + 8);
    // the array keeps the previous call's contents; only the error word has to
    // start at zero (every other piece is fully written before it is read)
    if ((r = cuda_status(cudaMemsetAsync(err, 0, sizeof(int), s)))) return r;
    if ((r = launch_window_bitmap(d_in, n, *p, bitmap, tile_cnt, s, err))) return r;
    const uint64_t tiles = (n + kWinTile - 1) / kWinTile;
    if ((r = launch_compact(bitmap, n, tile_cnt, tile_off, tiles, cands, kMaxCands, ncand, s)))
        return r;
    if ((r = launch_select(cands, ncand, kMaxCands, bitmap, n, *p, d_ends, cap, d_count, s)))
        return r;
    k_static_mark_error<<<1, 32, 0, s>>>(err, d_count);
    return cuda_status(cudaGetLastError());
}
