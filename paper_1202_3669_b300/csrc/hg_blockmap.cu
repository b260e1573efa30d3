// Device block map: similarity detection by chunk/block identifiers.
//
// Sec. 2.1: content addressing names a block by its digest, so comparing
// digests finds identical blocks; Sec. 4.3 measures how much of a new
// checkpoint version is found in chunks already stored. Here the stored
// digests live in an open-addressing hash table in HBM, built and probed by
// kernels, so the comparison of a version's chunk digests against everything
// stored before never leaves the device.
//
// Table: nslots (a power of two, at least twice the capacity) slots of
//   tags[s]  the digest's first 8 bytes (0 = empty; a digest whose first 8
//            bytes are all zero is tagged 1)
//   rest[s]  the remaining 8 (MD5) or 12 (SHA-1) digest bytes in x, y, z and,
//            in w, once x..z are written, 1 -- or 2 when the tag stands for
//            eight zero bytes, so that tag 1 stays exact
// The home slot comes from digest bytes 8..15 (independent of the tag bytes);
// probing is linear. An insert claims an empty slot with a 64-bit CAS on the
// tag, writes the rest, and publishes w; an insert that meets an equal tag
// compares the rest once w is published (a claim made in the same launch
// completes within a few instructions; the wait is bounded and reports
// HG_ETIMEDOUT through the context's error word if it ever runs out).
// Lookups run in a later launch, when every claimed slot is published.
#include <cstring>
#include <new>

#include "hg_internal.h"

struct hg_blockmap {
    hg_ctx *ctx = nullptr;
    int algo = HG_MD5;
    uint64_t capacity = 0, nslots = 0;
    unsigned long long *tags = nullptr;
    uint4 *rest = nullptr;
    unsigned long long *entries = nullptr;     // distinct digests stored
    void *mem = nullptr;
    size_t mem_bytes = 0;
    uint32_t wait_limit = 0;                    // polls of a claimed slot's publish word
};

namespace hg {
namespace {

constexpr unsigned kBmThreads = 256;
constexpr uint32_t kReadyWaitLimit = 1u << 20;

struct Key {
    unsigned long long tag;
    uint32_t r0, r1, r2;     // r2 = 0 for MD5
    uint32_t mark;           // published w: 1, or 2 for a zero tag
    uint64_t home;
};

__device__ __forceinline__ Key load_key(const uint8_t *__restrict__ d, int dl) {
    // digests are 4-byte aligned rows of 16 or 20 bytes
    const uint32_t *w = reinterpret_cast<const uint32_t *>(d);
    Key k;
    const unsigned long long t = (unsigned long long)w[0] | ((unsigned long long)w[1] << 32);
    k.tag = t ? t : 1ull;
    k.mark = t ? 1u : 2u;
    k.r0 = w[2];
    k.r1 = w[3];
    k.r2 = dl == 20 ? w[4] : 0u;
    k.home = (uint64_t)w[2] | ((uint64_t)w[3] << 32);
    return k;
}

__device__ __forceinline__ uint32_t ld_ready(const uint4 *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(&p->w) : "memory");
    return v;
}

// Waits (bounded: `limit` polls) until slot s is published; false if the wait
// ran out.
__device__ __forceinline__ bool wait_ready(const uint4 *rest, uint64_t s, uint32_t limit) {
    for (uint32_t i = 0; i < limit; i++)
        if (ld_ready(rest + s)) return true;
    return false;
}

__device__ __forceinline__ bool rest_equal(const uint4 *rest, uint64_t s, const Key &k) {
    const volatile uint4 *p = rest + s;
    return p->x == k.r0 && p->y == k.r1 && p->z == k.r2 && p->w == k.mark;
}

__global__ void __launch_bounds__(kBmThreads) k_bm_insert(const uint8_t *__restrict__ dg, int dl,
                                                          uint64_t count, const uint64_t *d_count,
                                                          unsigned long long *tags, uint4 *rest,
                                                          uint64_t mask,
                                                          unsigned long long *entries, int *err,
                                                          uint32_t wait_limit) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t cnt = count;
    if (d_count) cnt = min(cnt, *d_count);
    if (i >= cnt) return;
    const Key k = load_key(dg + i * (uint64_t)dl, dl);
    uint64_t s = k.home & mask;
    for (uint64_t probe = 0; probe <= mask; probe++, s = (s + 1) & mask) {
        unsigned long long t = *(volatile unsigned long long *)(tags + s);
        if (t == 0) {
            t = atomicCAS(tags + s, 0ull, k.tag);
            if (t == 0) {
                uint4 *p = rest + s;
                p->x = k.r0;
                p->y = k.r1;
                p->z = k.r2;
                asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&p->w), "r"(k.mark) : "memory");
                atomicAdd(entries, 1ull);
                return;
            }
        }
        if (t == k.tag) {
            if (!wait_ready(rest, s, wait_limit)) {
                atomicCAS(err, 0, (int)HG_ETIMEDOUT);
                return;
            }
            if (rest_equal(rest, s, k)) return;     // already stored
        }
    }
    atomicCAS(err, 0, (int)HG_ECAPACITY);           // every slot is taken
}

__global__ void __launch_bounds__(kBmThreads) k_bm_lookup(const uint8_t *__restrict__ dg, int dl,
                                                          const uint64_t *__restrict__ ends,
                                                          uint64_t count, const uint64_t *d_count,
                                                          const unsigned long long *__restrict__ tags,
                                                          const uint4 *__restrict__ rest, uint64_t mask,
                                                          uint8_t *__restrict__ hits,
                                                          unsigned long long *result, int *err) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t cnt = count;
    if (d_count) cnt = min(cnt, *d_count);
    bool hit = false;
    uint64_t bytes = 0;
    if (i < cnt) {
        const Key k = load_key(dg + i * (uint64_t)dl, dl);
        uint64_t s = k.home & mask;
        for (uint64_t probe = 0; probe <= mask; probe++, s = (s + 1) & mask) {
            const unsigned long long t = tags[s];
            if (t == 0) break;
            if (t == k.tag) {
                const uint4 r = rest[s];
                if (r.w == 0) {                 // inserts are done before lookups run
                    atomicCAS(err, 0, (int)HG_EINVAL);
                    break;
                }
                if (r.x == k.r0 && r.y == k.r1 && r.z == k.r2 && r.w == k.mark) {
                    hit = true;
                    break;
                }
            }
        }
        if (hits) hits[i] = hit ? 1 : 0;
        if (hit && ends) bytes = ends[i] - (i ? ends[i - 1] : 0);
    }
    if (result) {
        const unsigned mask32 = __ballot_sync(0xffffffffu, hit);
        unsigned long long b = bytes;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) b += __shfl_down_sync(0xffffffffu, b, o);
        if ((threadIdx.x & 31) == 0 && mask32) {
            atomicAdd(result, (unsigned long long)__popc(mask32));
            atomicAdd(result + 1, b);
        }
    }
}

}  // namespace
}  // namespace hg

using namespace hg;

extern "C" {

int hg_blockmap_create(hg_ctx *ctx, int algo, uint64_t capacity, hg_blockmap **out) {
    if (!ctx || !out || hg_digest_len(algo) < 0 || capacity == 0 || capacity > (1ull << 40))
        return HG_EINVAL;
    *out = nullptr;
    uint64_t nslots = 1024;
    while (nslots < 2 * capacity) nslots <<= 1;
    const size_t bytes = nslots * (sizeof(unsigned long long) + sizeof(uint4)) + 256;
    if (ctx->held + bytes > ctx->budget) return HG_ENOMEM;
    hg_blockmap *m = new (std::nothrow) hg_blockmap();
    if (!m) return HG_ENOMEM;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    int rc = HG_OK;
    if (cudaMalloc(&m->mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        rc = HG_ENOMEM;
    } else if (cudaMemset(m->mem, 0, bytes) != cudaSuccess) {
        rc = HG_ECUDA;
    }
    cudaSetDevice(prev);
    if (rc != HG_OK) {
        if (m->mem) cudaFree(m->mem);
        delete m;
        return rc;
    }
    char *b = static_cast<char *>(m->mem);
    m->ctx = ctx;
    m->algo = algo;
    m->capacity = capacity;
    m->nslots = nslots;
    m->rest = reinterpret_cast<uint4 *>(b);
    m->tags = reinterpret_cast<unsigned long long *>(b + nslots * sizeof(uint4));
    m->entries = reinterpret_cast<unsigned long long *>(b + nslots * (sizeof(uint4) + 8));
    m->mem_bytes = bytes;
    m->wait_limit = kReadyWaitLimit;
    ctx->held += bytes;
    *out = m;
    return HG_OK;
}

int hg_blockmap_insert(hg_blockmap *m, const uint8_t *d_digests, uint64_t count,
                       const uint64_t *d_count, void *stream) {
    if (!m || (count && !d_digests) || (reinterpret_cast<uintptr_t>(d_digests) & 3)) return HG_EINVAL;
    if (count == 0) return HG_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(m->ctx->device);
    const unsigned grid = (unsigned)((count + kBmThreads - 1) / kBmThreads);
    k_bm_insert<<<grid, kBmThreads, 0, (cudaStream_t)stream>>>(
        d_digests, hg_digest_len(m->algo), count, d_count, m->tags, m->rest, m->nslots - 1,
        m->entries, m->ctx->d_err, m->wait_limit);
    const int r = cuda_status(cudaGetLastError());
    cudaSetDevice(prev);
    return r;
}

int hg_blockmap_lookup(hg_blockmap *m, const uint8_t *d_digests, const uint64_t *d_ends,
                       uint64_t count, const uint64_t *d_count, uint8_t *d_hits, uint64_t *d_result,
                       void *stream) {
    if (!m || (count && !d_digests) || (reinterpret_cast<uintptr_t>(d_digests) & 3) ||
        (!d_hits && !d_result) || (reinterpret_cast<uintptr_t>(d_result) & 7))
        return HG_EINVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(m->ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    int r = HG_OK;
    if (d_result) r = cuda_status(cudaMemsetAsync(d_result, 0, 2 * sizeof(uint64_t), s));
    if (r == HG_OK && count) {
        const unsigned grid = (unsigned)((count + kBmThreads - 1) / kBmThreads);
        k_bm_lookup<<<grid, kBmThreads, 0, s>>>(d_digests, hg_digest_len(m->algo), d_ends, count,
                                                 d_count, m->tags, m->rest, m->nslots - 1, d_hits,
                                                 reinterpret_cast<unsigned long long *>(d_result),
                                                 m->ctx->d_err);
        r = cuda_status(cudaGetLastError());
    }
    cudaSetDevice(prev);
    return r;
}

int hg_blockmap_count(hg_blockmap *m, uint64_t *d_out, void *stream) {
    if (!m || !d_out) return HG_EINVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(m->ctx->device);
    const int r = cuda_status(cudaMemcpyAsync(d_out, m->entries, sizeof(uint64_t),
                                              cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    cudaSetDevice(prev);
    return r;
}

int hg_blockmap_clear(hg_blockmap *m, void *stream) {
    if (!m) return HG_EINVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(m->ctx->device);
    const int r = cuda_status(cudaMemsetAsync(m->mem, 0, m->mem_bytes, (cudaStream_t)stream));
    cudaSetDevice(prev);
    return r;
}

int hg_blockmap_set_wait_limit(hg_blockmap *m, uint32_t polls) {
    if (!m) return HG_EINVAL;
    m->wait_limit = polls ? polls : kReadyWaitLimit;
    return HG_OK;
}

int hg_blockmap_inject_claim(hg_blockmap *m, const uint8_t *h_digest, void *stream) {
    if (!m || !h_digest) return HG_EINVAL;
    // the tag and home slot of the digest, as the kernels form them
    uint32_t w[4];
    std::memcpy(w, h_digest, sizeof w);
    unsigned long long tag = (unsigned long long)w[0] | ((unsigned long long)w[1] << 32);
    if (tag == 0) tag = 1;
    const uint64_t s = ((uint64_t)w[2] | ((uint64_t)w[3] << 32)) & (m->nslots - 1);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(m->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long cur = 1;
    int r = cuda_status(cudaStreamSynchronize(st));
    if (r == HG_OK)
        r = cuda_status(cudaMemcpy(&cur, m->tags + s, sizeof cur, cudaMemcpyDeviceToHost));
    if (r == HG_OK && cur != 0) r = HG_EINVAL;              // the home slot is taken
    if (r == HG_OK)
        r = cuda_status(cudaMemcpy(m->tags + s, &tag, sizeof tag, cudaMemcpyHostToDevice));
    cudaSetDevice(prev);
    return r;
}

int hg_blockmap_destroy(hg_blockmap *m) {
    if (!m) return HG_EINVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(m->ctx->device);
    cudaDeviceSynchronize();
    cudaFree(m->mem);
    m->ctx->held -= m->mem_bytes;
    cudaSetDevice(prev);
    delete m;
    return HG_OK;
}

}  // extern "C"
