// C ABI of libhashgpu.so: argument checks, scratch management and launches.
// Every computation is done by the kernels in hg_direct.cu and hg_cdc.cu.
#include <cstdlib>
#include <cstring>
#include <new>

#include "hg_internal.h"

namespace hg {

static int check_params(const hg_cdc_params *p) {
    if (!p || p->reserved != 0) return HG_EINVAL;
    if (p->window < 1 || p->window > 55) return HG_EUNSUPPORTED;
    if (p->mask_bits < 1 || p->mask_bits > 32) return HG_EINVAL;
    if (p->mask_bits < 32 && (p->magic >> p->mask_bits) != 0) return HG_EINVAL;
    if (p->min_chunk < 1 || p->min_chunk > p->max_chunk) return HG_EINVAL;
    return HG_OK;
}

int ensure(hg_ctx *ctx, void **p, uint64_t *cap, uint64_t count, size_t elem) {
    if (count <= *cap && *p) return HG_OK;
    uint64_t want = count + count / 4 + 1024;            // grow with headroom
    const size_t old_bytes = (size_t)(*cap) * elem;
    const size_t new_bytes = (size_t)want * elem;
    if (ctx->held - old_bytes + new_bytes > ctx->budget) {
        want = count;
        if (ctx->held - old_bytes + (size_t)want * elem > ctx->budget) return HG_ENOMEM;
    }
    if (*p) {
        cudaError_t e = cudaDeviceSynchronize();         // scratch may be in use by queued work
        if (e != cudaSuccess) return HG_ECUDA;
        cudaFree(*p);
        ctx->held -= old_bytes;
        *p = nullptr;
        *cap = 0;
    }
    void *q = nullptr;
    if (cudaMalloc(&q, (size_t)want * elem) != cudaSuccess) {
        cudaGetLastError();
        return HG_ENOMEM;
    }
    *p = q;
    *cap = want;
    ctx->held += (size_t)want * elem;
    return HG_OK;
}

// Scratch for chunking an n-byte input.
static int ensure_cdc(hg_ctx *ctx, uint64_t n) {
    const uint64_t words = (n + 31) / 32, tiles = (n + kWinTile - 1) / kWinTile;
    int r;
    if ((r = ensure(ctx, (void **)&ctx->d_bitmap, &ctx->bitmap_words, words ? words : 1, 4))) return r;
    if ((r = ensure(ctx, (void **)&ctx->d_tile_cnt, &ctx->tile_cap, tiles ? tiles : 1, 4))) return r;
    if ((r = ensure(ctx, (void **)&ctx->d_tile_off, &ctx->tile_off_cap, tiles ? tiles : 1, 8))) return r;
    if ((r = ensure(ctx, (void **)&ctx->d_cands, &ctx->cand_cap, cand_capacity(n), 8))) return r;
    return HG_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace hg

using namespace hg;

extern "C" {

void hg_cdc_default_params(hg_cdc_params *p) {
    if (!p) return;
    p->window = 20;
    p->mask_bits = 13;
    p->magic = 0x0F0F;
    p->reserved = 0;
    p->min_chunk = 2048;
    p->max_chunk = 65536;
}

const char *hg_strerror(int s) {
    switch (s) {
        case HG_OK: return "ok";
        case HG_EINVAL: return "invalid argument";
        case HG_ENOMEM: return "device budget or allocation exhausted";
        case HG_ECAPACITY: return "output capacity too small";
        case HG_ETIMEDOUT: return "bounded device wait timed out";
        case HG_ECUDA: return "CUDA runtime error";
        case HG_EAGAIN: return "not ready";
        case HG_ECANCELED: return "cancelled";
        case HG_EUNSUPPORTED: return "unsupported parameters";
        default: return "unknown status";
    }
}

int hg_digest_len(int algo) { return algo == HG_MD5 ? 16 : algo == HG_SHA1 ? 20 : HG_EINVAL; }

int hg_init(hg_ctx **out, int device, size_t budget) {
    if (!out) return HG_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return HG_ECUDA;
    }
    hg_ctx *c = new (std::nothrow) hg_ctx();
    if (!c) return HG_ENOMEM;
    c->device = device;
    c->budget = budget ? budget : ((size_t)32 << 30);
    DeviceGuard g(device);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&c->d_err, 64) != cudaSuccess || cudaMemset(c->d_err, 0, 64) != cudaSuccess) {
        cudaGetLastError();
        if (c->d_err) cudaFree(c->d_err);
        delete c;
        return HG_ECUDA;
    }
    c->d_ncand = reinterpret_cast<uint64_t *>(reinterpret_cast<char *>(c->d_err) + 8);
    c->held = 64;
    *out = c;
    return HG_OK;
}

int hg_destroy(hg_ctx *c) {
    if (!c) return HG_EINVAL;
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    cudaFree(c->d_bitmap);
    cudaFree(c->d_tile_cnt);
    cudaFree(c->d_tile_off);
    cudaFree(c->d_cands);
    cudaFree(c->d_err);
    delete c;
    return HG_OK;
}

int hg_reserve(hg_ctx *c, uint64_t max_bytes) {
    if (!c) return HG_EINVAL;
    DeviceGuard g(c->device);
    return ensure_cdc(c, max_bytes);
}

uint64_t hg_scratch_bytes(const hg_ctx *c) { return c ? c->held : 0; }

int hg_sync(hg_ctx *c, void *stream) {
    if (!c) return HG_EINVAL;
    DeviceGuard g(c->device);
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return HG_ECUDA;
    }
    int err = 0;
    if (cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return HG_ECUDA;
    if (err) cudaMemset(c->d_err, 0, sizeof(int));
    return err;
}

int hg_hash_blocks(hg_ctx *c, int algo, const uint8_t *d_in, uint64_t n, uint64_t block,
                   uint8_t *d_digests, uint8_t *d_root, void *stream) {
    if (!c || block == 0 || hg_digest_len(algo) < 0) return HG_EINVAL;
    const uint64_t nblk = (n + block - 1) / block;
    if ((n && !d_in) || (nblk && !d_digests)) return HG_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_digests) & 3) || (reinterpret_cast<uintptr_t>(d_root) & 3))
        return HG_EINVAL;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    int r = launch_hash_blocks(algo, d_in, n, block, d_digests, s, c->d_err);
    if (r) return r;
    if (d_root) r = launch_root(algo, d_digests, nblk * (uint64_t)hg_digest_len(algo), d_root, s);
    return r;
}

int hg_window_bitmap(hg_ctx *c, const uint8_t *d_in, uint64_t n, const hg_cdc_params *p,
                     uint32_t *d_bitmap, void *stream) {
    if (!c) return HG_EINVAL;
    int r = check_params(p);
    if (r) return r;
    if (n == 0) return HG_OK;
    if (!d_in || !d_bitmap || (reinterpret_cast<uintptr_t>(d_bitmap) & 3)) return HG_EINVAL;
    DeviceGuard g(c->device);
    const uint64_t tiles = (n + kWinTile - 1) / kWinTile;
    if ((r = ensure(c, (void **)&c->d_tile_cnt, &c->tile_cap, tiles, 4))) return r;
    return launch_window_bitmap(d_in, n, *p, d_bitmap, c->d_tile_cnt, (cudaStream_t)stream, c->d_err);
}

int hg_cdc_candidates(hg_ctx *c, const uint8_t *d_in, uint64_t n, const hg_cdc_params *p,
                      uint64_t *d_cands, uint64_t cap, uint64_t *d_count, void *stream) {
    if (!c || !d_count || (cap && !d_cands)) return HG_EINVAL;
    int r = check_params(p);
    if (r) return r;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return cuda_status(cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s));
    if (!d_in) return HG_EINVAL;
    if ((r = ensure_cdc(c, n))) return r;
    if ((r = launch_window_bitmap(d_in, n, *p, c->d_bitmap, c->d_tile_cnt, s, c->d_err))) return r;
    const uint64_t tiles = (n + kWinTile - 1) / kWinTile;
    return launch_compact(c->d_bitmap, n, c->d_tile_cnt, c->d_tile_off, tiles, d_cands, cap,
                          d_count, s);
}

int hg_cdc_boundaries(hg_ctx *c, const uint8_t *d_in, uint64_t n, const hg_cdc_params *p,
                      uint64_t *d_ends, uint64_t cap, uint64_t *d_count, void *stream) {
    if (!c || !d_count || (cap && !d_ends)) return HG_EINVAL;
    int r = check_params(p);
    if (r) return r;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return cuda_status(cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s));
    if (!d_in) return HG_EINVAL;
    if ((r = ensure_cdc(c, n))) return r;
    if ((r = launch_window_bitmap(d_in, n, *p, c->d_bitmap, c->d_tile_cnt, s, c->d_err))) return r;
    const uint64_t tiles = (n + kWinTile - 1) / kWinTile;
    if ((r = launch_compact(c->d_bitmap, n, c->d_tile_cnt, c->d_tile_off, tiles, c->d_cands,
                            c->cand_cap, c->d_ncand, s)))
        return r;
    return launch_select(c->d_cands, c->d_ncand, c->cand_cap, c->d_bitmap, n, *p, d_ends, cap,
                         d_count, s);
}

int hg_hash_chunks(hg_ctx *c, int algo, const uint8_t *d_in, uint64_t n, const uint64_t *d_ends,
                   uint64_t nchunk, const uint64_t *d_count, uint8_t *d_digests, void *stream) {
    if (!c || hg_digest_len(algo) < 0) return HG_EINVAL;
    if (nchunk == 0) return HG_OK;
    if ((n && !d_in) || !d_ends || !d_digests || (reinterpret_cast<uintptr_t>(d_digests) & 3))
        return HG_EINVAL;
    DeviceGuard g(c->device);
    return launch_hash_chunks(algo, d_in, n, d_ends, nchunk, d_count, d_digests,
                              (cudaStream_t)stream, c->d_err);
}

}  // extern "C"
