// The hash-of-hashes computed on a host core (Sec. 3.2.2: the GPU writes the
// segment digests to one output buffer and the CPU computes the final hash of
// those intermediate hashes).
//
// The root is a single Merkle-Damgard chain over the digest list: it cannot be
// split, and a host core runs a dependent chain of 32-bit operations several
// times faster than one GPU lane (about 1 cycle per dependent operation at a
// higher clock, against 15-20 cycles per MD5 step on a GPU lane). So for all but
// tiny digest lists the library copies the digests into a pinned staging buffer
// of the context, hashes them in a host function enqueued on the caller's stream
// (cudaLaunchHostFunc), and copies the root back -- all in stream order, so the
// call stays asynchronous.
//
// The MD5 (RFC 1321) and SHA-1 (FIPS 180-4) code below is the library's own
// host implementation, written for speed with the round constants as
// immediates; it is independent of the test oracle.
#include <cstdlib>
#include <cstring>
#include <mutex>
#if defined(__x86_64__)
#include <immintrin.h>
#endif
#include <new>

#include "hg_internal.h"

namespace hg {
namespace {

inline uint32_t rl(uint32_t x, int s) { return (x << s) | (x >> (32 - s)); }
inline uint32_t ld_le(const uint8_t *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
inline uint32_t ld_be(const uint8_t *p) {
    return ((uint32_t)p[0] << 24) | ((uint32_t)p[1] << 16) | ((uint32_t)p[2] << 8) | (uint32_t)p[3];
}

// ---- MD5: one 64-byte block into state h ----------------------------------------------------
#define HR_F(x, y, z) ((z) ^ ((x) & ((y) ^ (z))))
#define HR_G(x, y, z) ((y) ^ ((z) & ((x) ^ (y))))
#define HR_H(x, y, z) ((x) ^ (y) ^ (z))
#define HR_I(x, y, z) ((y) ^ ((x) | ~(z)))
#define HR_S(f, a, b, c, d, x, t, s) (a) = (b) + rl((a) + f((b), (c), (d)) + (x) + (t), (s))

void md5_block(uint32_t h[4], const uint8_t *blk) {
    uint32_t X[16];
    for (int i = 0; i < 16; i++) X[i] = ld_le(blk + 4 * i);
    uint32_t a = h[0], b = h[1], c = h[2], d = h[3];
    HR_S(HR_F, a, b, c, d, X[0], 0xd76aa478u, 7);   HR_S(HR_F, d, a, b, c, X[1], 0xe8c7b756u, 12);
    HR_S(HR_F, c, d, a, b, X[2], 0x242070dbu, 17);  HR_S(HR_F, b, c, d, a, X[3], 0xc1bdceeeu, 22);
    HR_S(HR_F, a, b, c, d, X[4], 0xf57c0fafu, 7);   HR_S(HR_F, d, a, b, c, X[5], 0x4787c62au, 12);
    HR_S(HR_F, c, d, a, b, X[6], 0xa8304613u, 17);  HR_S(HR_F, b, c, d, a, X[7], 0xfd469501u, 22);
    HR_S(HR_F, a, b, c, d, X[8], 0x698098d8u, 7);   HR_S(HR_F, d, a, b, c, X[9], 0x8b44f7afu, 12);
    HR_S(HR_F, c, d, a, b, X[10], 0xffff5bb1u, 17); HR_S(HR_F, b, c, d, a, X[11], 0x895cd7beu, 22);
    HR_S(HR_F, a, b, c, d, X[12], 0x6b901122u, 7);  HR_S(HR_F, d, a, b, c, X[13], 0xfd987193u, 12);
    HR_S(HR_F, c, d, a, b, X[14], 0xa679438eu, 17); HR_S(HR_F, b, c, d, a, X[15], 0x49b40821u, 22);
    HR_S(HR_G, a, b, c, d, X[1], 0xf61e2562u, 5);   HR_S(HR_G, d, a, b, c, X[6], 0xc040b340u, 9);
    HR_S(HR_G, c, d, a, b, X[11], 0x265e5a51u, 14); HR_S(HR_G, b, c, d, a, X[0], 0xe9b6c7aau, 20);
    HR_S(HR_G, a, b, c, d, X[5], 0xd62f105du, 5);   HR_S(HR_G, d, a, b, c, X[10], 0x02441453u, 9);
    HR_S(HR_G, c, d, a, b, X[15], 0xd8a1e681u, 14); HR_S(HR_G, b, c, d, a, X[4], 0xe7d3fbc8u, 20);
    HR_S(HR_G, a, b, c, d, X[9], 0x21e1cde6u, 5);   HR_S(HR_G, d, a, b, c, X[14], 0xc33707d6u, 9);
    HR_S(HR_G, c, d, a, b, X[3], 0xf4d50d87u, 14);  HR_S(HR_G, b, c, d, a, X[8], 0x455a14edu, 20);
    HR_S(HR_G, a, b, c, d, X[13], 0xa9e3e905u, 5);  HR_S(HR_G, d, a, b, c, X[2], 0xfcefa3f8u, 9);
    HR_S(HR_G, c, d, a, b, X[7], 0x676f02d9u, 14);  HR_S(HR_G, b, c, d, a, X[12], 0x8d2a4c8au, 20);
    HR_S(HR_H, a, b, c, d, X[5], 0xfffa3942u, 4);   HR_S(HR_H, d, a, b, c, X[8], 0x8771f681u, 11);
    HR_S(HR_H, c, d, a, b, X[11], 0x6d9d6122u, 16); HR_S(HR_H, b, c, d, a, X[14], 0xfde5380cu, 23);
    HR_S(HR_H, a, b, c, d, X[1], 0xa4beea44u, 4);   HR_S(HR_H, d, a, b, c, X[4], 0x4bdecfa9u, 11);
    HR_S(HR_H, c, d, a, b, X[7], 0xf6bb4b60u, 16);  HR_S(HR_H, b, c, d, a, X[10], 0xbebfbc70u, 23);
    HR_S(HR_H, a, b, c, d, X[13], 0x289b7ec6u, 4);  HR_S(HR_H, d, a, b, c, X[0], 0xeaa127fau, 11);
    HR_S(HR_H, c, d, a, b, X[3], 0xd4ef3085u, 16);  HR_S(HR_H, b, c, d, a, X[6], 0x04881d05u, 23);
    HR_S(HR_H, a, b, c, d, X[9], 0xd9d4d039u, 4);   HR_S(HR_H, d, a, b, c, X[12], 0xe6db99e5u, 11);
    HR_S(HR_H, c, d, a, b, X[15], 0x1fa27cf8u, 16); HR_S(HR_H, b, c, d, a, X[2], 0xc4ac5665u, 23);
    HR_S(HR_I, a, b, c, d, X[0], 0xf4292244u, 6);   HR_S(HR_I, d, a, b, c, X[7], 0x432aff97u, 10);
    HR_S(HR_I, c, d, a, b, X[14], 0xab9423a7u, 15); HR_S(HR_I, b, c, d, a, X[5], 0xfc93a039u, 21);
    HR_S(HR_I, a, b, c, d, X[12], 0x655b59c3u, 6);  HR_S(HR_I, d, a, b, c, X[3], 0x8f0ccc92u, 10);
    HR_S(HR_I, c, d, a, b, X[10], 0xffeff47du, 15); HR_S(HR_I, b, c, d, a, X[1], 0x85845dd1u, 21);
    HR_S(HR_I, a, b, c, d, X[8], 0x6fa87e4fu, 6);   HR_S(HR_I, d, a, b, c, X[15], 0xfe2ce6e0u, 10);
    HR_S(HR_I, c, d, a, b, X[6], 0xa3014314u, 15);  HR_S(HR_I, b, c, d, a, X[13], 0x4e0811a1u, 21);
    HR_S(HR_I, a, b, c, d, X[4], 0xf7537e82u, 6);   HR_S(HR_I, d, a, b, c, X[11], 0xbd3af235u, 10);
    HR_S(HR_I, c, d, a, b, X[2], 0x2ad7d2bbu, 15);  HR_S(HR_I, b, c, d, a, X[9], 0xeb86d391u, 21);
    h[0] += a; h[1] += b; h[2] += c; h[3] += d;
}

// ---- SHA-1: one 64-byte block into state h -------------------------------------------------
void sha1_block(uint32_t h[5], const uint8_t *blk) {
    uint32_t w[16];
    for (int i = 0; i < 16; i++) w[i] = ld_be(blk + 4 * i);
    uint32_t a = h[0], b = h[1], c = h[2], d = h[3], e = h[4];
    for (int t = 0; t < 80; t++) {
        if (t >= 16) w[t & 15] = rl(w[(t + 13) & 15] ^ w[(t + 8) & 15] ^ w[(t + 2) & 15] ^ w[t & 15], 1);
        uint32_t f, k;
        if (t < 20) { f = d ^ (b & (c ^ d)); k = 0x5a827999u; }
        else if (t < 40) { f = b ^ c ^ d; k = 0x6ed9eba1u; }
        else if (t < 60) { f = (b & c) | (d & (b | c)); k = 0x8f1bbcdcu; }
        else { f = b ^ c ^ d; k = 0xca62c1d6u; }
        const uint32_t tmp = rl(a, 5) + f + e + k + w[t & 15];
        e = d; d = c; c = rl(b, 30); b = a; a = tmp;
    }
    h[0] += a; h[1] += b; h[2] += c; h[3] += d; h[4] += e;
}

// ---- SHA-1 with the x86 SHA extensions (runtime-dispatched) -------------------------------
// The 80 rounds run as 20 groups of four (sha1rnds4, whose immediate picks the
// round function and constant of each 20-round stage). The state register
// holds a, b, c, d with a in the highest lane; e enters each group added to the
// group's first message word: the first group adds the saved e, every later
// group adds rotl(a, 30) of the state two groups back (sha1nexte). The message
// schedule runs four words at a time: group g >= 4 is
//   sha1msg2(sha1msg1(W[g-4], W[g-3]) ^ W[g-2], W[g-1]),
// sha1msg1 forming W[t-16] ^ W[t-14], sha1msg2 adding W[t-3] and the rotate.
#if defined(__x86_64__)
__attribute__((target("sha,sse4.1,ssse3"))) void sha1_blocks_ni(uint32_t h[5], const uint8_t *p,
                                                                 uint64_t nblk) {
    const __m128i bswap = _mm_set_epi64x(0x0001020304050607ll, 0x08090a0b0c0d0e0fll);
    __m128i abcd = _mm_shuffle_epi32(_mm_loadu_si128(reinterpret_cast<const __m128i *>(h)), 0x1B);
    __m128i e0 = _mm_set_epi32((int)h[4], 0, 0, 0);
    for (uint64_t k = 0; k < nblk; k++, p += 64) {
        const __m128i abcd_save = abcd, e_save = e0;
        __m128i w[4];
        __m128i prev = abcd;                  // state before the previous group
#pragma GCC unroll 20
        for (int g = 0; g < 20; g++) {
            __m128i wg;
            if (g < 4) {
                wg = _mm_shuffle_epi8(_mm_loadu_si128(reinterpret_cast<const __m128i *>(p + 16 * g)), bswap);
            } else {
                wg = _mm_sha1msg2_epu32(
                    _mm_xor_si128(_mm_sha1msg1_epu32(w[g & 3], w[(g + 1) & 3]), w[(g + 2) & 3]),
                    w[(g + 3) & 3]);
            }
            w[g & 3] = wg;
            const __m128i ein = g == 0 ? _mm_add_epi32(e0, wg) : _mm_sha1nexte_epu32(prev, wg);
            prev = abcd;
            switch (g / 5) {
                case 0: abcd = _mm_sha1rnds4_epu32(abcd, ein, 0); break;
                case 1: abcd = _mm_sha1rnds4_epu32(abcd, ein, 1); break;
                case 2: abcd = _mm_sha1rnds4_epu32(abcd, ein, 2); break;
                default: abcd = _mm_sha1rnds4_epu32(abcd, ein, 3); break;
            }
        }
        e0 = _mm_sha1nexte_epu32(prev, e_save);
        abcd = _mm_add_epi32(abcd, abcd_save);
    }
    _mm_storeu_si128(reinterpret_cast<__m128i *>(h), _mm_shuffle_epi32(abcd, 0x1B));
    h[4] = (uint32_t)_mm_extract_epi32(e0, 3);
}

bool use_sha_ni() {
    static const bool ok = [] {
        const char *env = std::getenv("HG_HOST_SHA1");
        if (env && std::strcmp(env, "portable") == 0) return false;
        __builtin_cpu_init();
        return __builtin_cpu_supports("sha") && __builtin_cpu_supports("sse4.1");
    }();
    return ok;
}
#else
void sha1_blocks_ni(uint32_t *, const uint8_t *, uint64_t) {}
bool use_sha_ni() { return false; }
#endif

}  // namespace

// Digest of n bytes at msg into out (16 or 20 bytes, standard byte order).
void host_digest(int algo, const uint8_t *msg, uint64_t n, uint8_t *out) {
    uint32_t h[5] = {0x67452301u, 0xefcdab89u, 0x98badcfeu, 0x10325476u, 0xc3d2e1f0u};
    const bool md5 = algo == HG_MD5;
    uint64_t i = 0;
    if (!md5 && use_sha_ni()) {
        i = n / 64 * 64;
        sha1_blocks_ni(h, msg, n / 64);
    }
    for (; i + 64 <= n; i += 64) md5 ? md5_block(h, msg + i) : sha1_block(h, msg + i);
    uint8_t tail[128];
    const uint64_t rem = n - i;
    std::memset(tail, 0, sizeof tail);
    if (rem) std::memcpy(tail, msg + i, rem);
    tail[rem] = 0x80;
    const uint64_t tl = rem < 56 ? 64 : 128;
    const uint64_t bits = n * 8;
    for (int k = 0; k < 8; k++)
        tail[tl - 8 + k] = md5 ? (uint8_t)(bits >> (8 * k)) : (uint8_t)(bits >> (56 - 8 * k));
    for (uint64_t j = 0; j < tl; j += 64) {
        if (md5) md5_block(h, tail + j);
        else if (use_sha_ni()) sha1_blocks_ni(h, tail + j, 1);
        else sha1_block(h, tail + j);
    }
    const int nw = md5 ? 4 : 5;
    for (int k = 0; k < nw; k++)
        for (int j = 0; j < 4; j++)
            out[4 * k + j] = md5 ? (uint8_t)(h[k] >> (8 * j)) : (uint8_t)(h[k] >> (24 - 8 * j));
}

namespace {

// Host function enqueued on the stream: hashes the staged digests of the
// oldest pending job of the context into the staging buffer's root slot.
void CUDART_CB root_host_fn(void *arg) {
    hg_ctx *c = static_cast<hg_ctx *>(arg);
    RootJob j{};
    {
        std::lock_guard<std::mutex> lock(c->root_mu);
        if (c->root_jobs.empty()) return;
        j = c->root_jobs.front();
        c->root_jobs.pop_front();
    }
    host_digest(j.algo, c->root_stage, j.nbytes, c->root_stage + c->root_cap);
}

}  // namespace

// Digest-list size from which the root is computed on the host. Measured on a
// B300 machine (root time alone, host path including its copies and host-function
// wake-up): the device chain runs MD5 at ~130 MB/s and SHA-1 at ~100 MB/s; a
// host core ran MD5 at 70-650 MB/s depending on the box and on how long the
// callback core had been idle, SHA-1 with the SHA extensions at ~1.1 GB/s
// after ~0.08 ms of fixed cost. Crossovers: MD5 between 256 KiB and 1 MiB of
// digests, SHA-1 (SHA extensions) near 10 KiB.
uint64_t host_root_min_bytes(int algo) {
    static const long long env = [] {
        const char *e = std::getenv("HG_HOST_ROOT_MIN");
        return e ? (long long)std::strtoull(e, nullptr, 10) : -1ll;
    }();
    if (env >= 0) return (uint64_t)env;
    if (algo == HG_MD5) return kHostRootMinMd5;
    return use_sha_ni() ? kHostRootMinSha1Ni : kHostRootMinSha1;
}

int enqueue_host_root(hg_ctx *c, int algo, const uint8_t *d_digests, uint64_t nbytes, uint8_t *d_root,
                      cudaStream_t s) {
    if (nbytes > c->root_cap || !c->root_stage) {
        // grow the staging buffer: earlier root jobs of this context may still use it
        if (cudaDeviceSynchronize() != cudaSuccess) return HG_ECUDA;
        if (c->root_stage) cudaFreeHost(c->root_stage);
        c->root_stage = nullptr;
        c->root_cap = 0;
        const uint64_t cap = nbytes + nbytes / 4 + 4096;
        void *p = nullptr;
        if (cudaHostAlloc(&p, cap + 64, cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            return HG_ENOMEM;
        }
        c->root_stage = static_cast<uint8_t *>(p);
        c->root_cap = cap;
    }
    if (cudaMemcpyAsync(c->root_stage, d_digests, nbytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return HG_ECUDA;
    {
        std::lock_guard<std::mutex> lock(c->root_mu);
        c->root_jobs.push_back(RootJob{algo, nbytes});
    }
    if (cudaLaunchHostFunc(s, root_host_fn, c) != cudaSuccess) {
        std::lock_guard<std::mutex> lock(c->root_mu);
        c->root_jobs.pop_back();
        return HG_ECUDA;
    }
    return cuda_status(cudaMemcpyAsync(d_root, c->root_stage + c->root_cap, algo == HG_MD5 ? 16 : 20,
                                       cudaMemcpyHostToDevice, s));
}

}  // namespace hg
