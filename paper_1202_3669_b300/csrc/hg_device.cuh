// Device-side building blocks of the HashGPU kernels (sm_103a).
//
// MD5 (RFC 1321) and SHA-1 (FIPS 180-4) compression functions written as
// straight-line integer code: every round constant is an instruction
// immediate, rotations are funnel shifts, and the boolean round functions are
// left to the compiler as single three-input logic ops. Message words arrive
// as little-endian 32-bit words (the natural load order); SHA-1 byte-swaps
// them itself.
#pragma once
#include <cstdint>
#include <utility>

namespace hg {

__device__ __forceinline__ uint32_t rotl(uint32_t x, int s) { return __funnelshift_l(x, x, s); }
__device__ __forceinline__ uint32_t bswap(uint32_t x) { return __byte_perm(x, 0, 0x0123); }

// ---------------------------------------------------------------- MD5 ------
// Round functions of RFC 1321 Sec. 3.4 in select form.
#define HG_MD5_F(x, y, z) ((z) ^ ((x) & ((y) ^ (z))))
#define HG_MD5_G(x, y, z) ((y) ^ ((z) & ((x) ^ (y))))
#define HG_MD5_H(x, y, z) ((x) ^ (y) ^ (z))
#define HG_MD5_I(x, y, z) ((y) ^ ((x) | ~(z)))
#define HG_MD5_STEP(f, a, b, c, d, m, k, s)          \
    do {                                              \
        (a) += f((b), (c), (d)) + (m) + (uint32_t)(k); \
        (a) = rotl((a), (s)) + (b);                   \
    } while (0)

// RFC 1321 Sec. 3.3 initial buffer words A, B, C, D.
constexpr uint32_t kMd5A = 0x67452301u, kMd5B = 0xefcdab89u, kMd5C = 0x98badcfeu,
                   kMd5D = 0x10325476u;

// The 64 operations on one block. With FULL = false it stops after operation
// 61 (index 60), the last one that writes word a, which is all the window
// test needs; the caller then adds the initial a itself.
template <bool FULL>
__device__ __forceinline__ void md5_rounds(uint32_t &a, uint32_t &b, uint32_t &c, uint32_t &d,
                                           const uint32_t (&M)[16]) {
    HG_MD5_STEP(HG_MD5_F, a, b, c, d, M[0], 0xd76aa478, 7);
    HG_MD5_STEP(HG_MD5_F, d, a, b, c, M[1], 0xe8c7b756, 12);
    HG_MD5_STEP(HG_MD5_F, c, d, a, b, M[2], 0x242070db, 17);
    HG_MD5_STEP(HG_MD5_F, b, c, d, a, M[3], 0xc1bdceee, 22);
    HG_MD5_STEP(HG_MD5_F, a, b, c, d, M[4], 0xf57c0faf, 7);
    HG_MD5_STEP(HG_MD5_F, d, a, b, c, M[5], 0x4787c62a, 12);
    HG_MD5_STEP(HG_MD5_F, c, d, a, b, M[6], 0xa8304613, 17);
    HG_MD5_STEP(HG_MD5_F, b, c, d, a, M[7], 0xfd469501, 22);
    HG_MD5_STEP(HG_MD5_F, a, b, c, d, M[8], 0x698098d8, 7);
    HG_MD5_STEP(HG_MD5_F, d, a, b, c, M[9], 0x8b44f7af, 12);
    HG_MD5_STEP(HG_MD5_F, c, d, a, b, M[10], 0xffff5bb1, 17);
    HG_MD5_STEP(HG_MD5_F, b, c, d, a, M[11], 0x895cd7be, 22);
    HG_MD5_STEP(HG_MD5_F, a, b, c, d, M[12], 0x6b901122, 7);
    HG_MD5_STEP(HG_MD5_F, d, a, b, c, M[13], 0xfd987193, 12);
    HG_MD5_STEP(HG_MD5_F, c, d, a, b, M[14], 0xa679438e, 17);
    HG_MD5_STEP(HG_MD5_F, b, c, d, a, M[15], 0x49b40821, 22);

    HG_MD5_STEP(HG_MD5_G, a, b, c, d, M[1], 0xf61e2562, 5);
    HG_MD5_STEP(HG_MD5_G, d, a, b, c, M[6], 0xc040b340, 9);
    HG_MD5_STEP(HG_MD5_G, c, d, a, b, M[11], 0x265e5a51, 14);
    HG_MD5_STEP(HG_MD5_G, b, c, d, a, M[0], 0xe9b6c7aa, 20);
    HG_MD5_STEP(HG_MD5_G, a, b, c, d, M[5], 0xd62f105d, 5);
    HG_MD5_STEP(HG_MD5_G, d, a, b, c, M[10], 0x02441453, 9);
    HG_MD5_STEP(HG_MD5_G, c, d, a, b, M[15], 0xd8a1e681, 14);
    HG_MD5_STEP(HG_MD5_G, b, c, d, a, M[4], 0xe7d3fbc8, 20);
    HG_MD5_STEP(HG_MD5_G, a, b, c, d, M[9], 0x21e1cde6, 5);
    HG_MD5_STEP(HG_MD5_G, d, a, b, c, M[14], 0xc33707d6, 9);
    HG_MD5_STEP(HG_MD5_G, c, d, a, b, M[3], 0xf4d50d87, 14);
    HG_MD5_STEP(HG_MD5_G, b, c, d, a, M[8], 0x455a14ed, 20);
    HG_MD5_STEP(HG_MD5_G, a, b, c, d, M[13], 0xa9e3e905, 5);
    HG_MD5_STEP(HG_MD5_G, d, a, b, c, M[2], 0xfcefa3f8, 9);
    HG_MD5_STEP(HG_MD5_G, c, d, a, b, M[7], 0x676f02d9, 14);
    HG_MD5_STEP(HG_MD5_G, b, c, d, a, M[12], 0x8d2a4c8a, 20);

    HG_MD5_STEP(HG_MD5_H, a, b, c, d, M[5], 0xfffa3942, 4);
    HG_MD5_STEP(HG_MD5_H, d, a, b, c, M[8], 0x8771f681, 11);
    HG_MD5_STEP(HG_MD5_H, c, d, a, b, M[11], 0x6d9d6122, 16);
    HG_MD5_STEP(HG_MD5_H, b, c, d, a, M[14], 0xfde5380c, 23);
    HG_MD5_STEP(HG_MD5_H, a, b, c, d, M[1], 0xa4beea44, 4);
    HG_MD5_STEP(HG_MD5_H, d, a, b, c, M[4], 0x4bdecfa9, 11);
    HG_MD5_STEP(HG_MD5_H, c, d, a, b, M[7], 0xf6bb4b60, 16);
    HG_MD5_STEP(HG_MD5_H, b, c, d, a, M[10], 0xbebfbc70, 23);
    HG_MD5_STEP(HG_MD5_H, a, b, c, d, M[13], 0x289b7ec6, 4);
    HG_MD5_STEP(HG_MD5_H, d, a, b, c, M[0], 0xeaa127fa, 11);
    HG_MD5_STEP(HG_MD5_H, c, d, a, b, M[3], 0xd4ef3085, 16);
    HG_MD5_STEP(HG_MD5_H, b, c, d, a, M[6], 0x04881d05, 23);
    HG_MD5_STEP(HG_MD5_H, a, b, c, d, M[9], 0xd9d4d039, 4);
    HG_MD5_STEP(HG_MD5_H, d, a, b, c, M[12], 0xe6db99e5, 11);
    HG_MD5_STEP(HG_MD5_H, c, d, a, b, M[15], 0x1fa27cf8, 16);
    HG_MD5_STEP(HG_MD5_H, b, c, d, a, M[2], 0xc4ac5665, 23);

    HG_MD5_STEP(HG_MD5_I, a, b, c, d, M[0], 0xf4292244, 6);
    HG_MD5_STEP(HG_MD5_I, d, a, b, c, M[7], 0x432aff97, 10);
    HG_MD5_STEP(HG_MD5_I, c, d, a, b, M[14], 0xab9423a7, 15);
    HG_MD5_STEP(HG_MD5_I, b, c, d, a, M[5], 0xfc93a039, 21);
    HG_MD5_STEP(HG_MD5_I, a, b, c, d, M[12], 0x655b59c3, 6);
    HG_MD5_STEP(HG_MD5_I, d, a, b, c, M[3], 0x8f0ccc92, 10);
    HG_MD5_STEP(HG_MD5_I, c, d, a, b, M[10], 0xffeff47d, 15);
    HG_MD5_STEP(HG_MD5_I, b, c, d, a, M[1], 0x85845dd1, 21);
    HG_MD5_STEP(HG_MD5_I, a, b, c, d, M[8], 0x6fa87e4f, 6);
    HG_MD5_STEP(HG_MD5_I, d, a, b, c, M[15], 0xfe2ce6e0, 10);
    HG_MD5_STEP(HG_MD5_I, c, d, a, b, M[6], 0xa3014314, 15);
    HG_MD5_STEP(HG_MD5_I, b, c, d, a, M[13], 0x4e0811a1, 21);
    HG_MD5_STEP(HG_MD5_I, a, b, c, d, M[4], 0xf7537e82, 6);
    if (FULL) {
        HG_MD5_STEP(HG_MD5_I, d, a, b, c, M[11], 0xbd3af235, 10);
        HG_MD5_STEP(HG_MD5_I, c, d, a, b, M[2], 0x2ad7d2bb, 15);
        HG_MD5_STEP(HG_MD5_I, b, c, d, a, M[9], 0xeb86d391, 21);
    }
}

struct Md5 {
    static constexpr int kDigest = 16;
    static constexpr int kWords = 4;
    uint32_t h[4];
    __device__ __forceinline__ void init() {
        h[0] = kMd5A; h[1] = kMd5B; h[2] = kMd5C; h[3] = kMd5D;
    }
    // Only the pipe-split forms (Md5Split, Sha1Split) use a run-time 1.
    __device__ __forceinline__ void set_one(uint32_t) {}
    // M: little-endian message words.
    __device__ __forceinline__ void compress(const uint32_t (&M)[16]) {
        uint32_t a = h[0], b = h[1], c = h[2], d = h[3];
        md5_rounds<true>(a, b, c, d, M);
        h[0] += a; h[1] += b; h[2] += c; h[3] += d;
    }
    // Bit length goes little-endian into words 14, 15.
    __device__ __forceinline__ static void put_length(uint32_t (&M)[16], uint64_t bytes) {
        const uint64_t bits = bytes * 8u;
        M[14] = (uint32_t)bits; M[15] = (uint32_t)(bits >> 32);
    }
    // Digest words in output byte order (little-endian words).
    __device__ __forceinline__ uint32_t out_word(int i) const { return h[i]; }
};

// MD5 with every operation written so the serial chain is as short as the
// hardware allows: a + M + T is formed off the chain, then one add of F, one
// wrap-around shift and one add of b. Used where one long message is the
// critical path (chunk digests, the hash-of-hashes); the throughput kernels
// keep Md5, whose form compiles to fewer instructions.
#define HG_MD5_CSTEP(f, a, b, c, d, m, k, s)                                                    \
    do {                                                                                        \
        const uint32_t fv_ = f((b), (c), (d));                                                  \
        const uint32_t t_ = (a) + (m) + (uint32_t)(k);                                          \
        uint32_t u_, r_;                                                                        \
        asm("add.u32 %0, %1, %2;" : "=r"(u_) : "r"(t_), "r"(fv_));                              \
        asm("shf.l.wrap.b32 %0, %1, %1, %2;" : "=r"(r_) : "r"(u_), "n"(s));                      \
        (a) = r_ + (b);                                                                         \
    } while (0)

__device__ __forceinline__ void md5_rounds_chain(uint32_t &a, uint32_t &b, uint32_t &c, uint32_t &d,
                                                 const uint32_t (&M)[16]) {
    HG_MD5_CSTEP(HG_MD5_F, a, b, c, d, M[0], 0xd76aa478, 7);
    HG_MD5_CSTEP(HG_MD5_F, d, a, b, c, M[1], 0xe8c7b756, 12);
    HG_MD5_CSTEP(HG_MD5_F, c, d, a, b, M[2], 0x242070db, 17);
    HG_MD5_CSTEP(HG_MD5_F, b, c, d, a, M[3], 0xc1bdceee, 22);
    HG_MD5_CSTEP(HG_MD5_F, a, b, c, d, M[4], 0xf57c0faf, 7);
    HG_MD5_CSTEP(HG_MD5_F, d, a, b, c, M[5], 0x4787c62a, 12);
    HG_MD5_CSTEP(HG_MD5_F, c, d, a, b, M[6], 0xa8304613, 17);
    HG_MD5_CSTEP(HG_MD5_F, b, c, d, a, M[7], 0xfd469501, 22);
    HG_MD5_CSTEP(HG_MD5_F, a, b, c, d, M[8], 0x698098d8, 7);
    HG_MD5_CSTEP(HG_MD5_F, d, a, b, c, M[9], 0x8b44f7af, 12);
    HG_MD5_CSTEP(HG_MD5_F, c, d, a, b, M[10], 0xffff5bb1, 17);
    HG_MD5_CSTEP(HG_MD5_F, b, c, d, a, M[11], 0x895cd7be, 22);
    HG_MD5_CSTEP(HG_MD5_F, a, b, c, d, M[12], 0x6b901122, 7);
    HG_MD5_CSTEP(HG_MD5_F, d, a, b, c, M[13], 0xfd987193, 12);
    HG_MD5_CSTEP(HG_MD5_F, c, d, a, b, M[14], 0xa679438e, 17);
    HG_MD5_CSTEP(HG_MD5_F, b, c, d, a, M[15], 0x49b40821, 22);

    HG_MD5_CSTEP(HG_MD5_G, a, b, c, d, M[1], 0xf61e2562, 5);
    HG_MD5_CSTEP(HG_MD5_G, d, a, b, c, M[6], 0xc040b340, 9);
    HG_MD5_CSTEP(HG_MD5_G, c, d, a, b, M[11], 0x265e5a51, 14);
    HG_MD5_CSTEP(HG_MD5_G, b, c, d, a, M[0], 0xe9b6c7aa, 20);
    HG_MD5_CSTEP(HG_MD5_G, a, b, c, d, M[5], 0xd62f105d, 5);
    HG_MD5_CSTEP(HG_MD5_G, d, a, b, c, M[10], 0x02441453, 9);
    HG_MD5_CSTEP(HG_MD5_G, c, d, a, b, M[15], 0xd8a1e681, 14);
    HG_MD5_CSTEP(HG_MD5_G, b, c, d, a, M[4], 0xe7d3fbc8, 20);
    HG_MD5_CSTEP(HG_MD5_G, a, b, c, d, M[9], 0x21e1cde6, 5);
    HG_MD5_CSTEP(HG_MD5_G, d, a, b, c, M[14], 0xc33707d6, 9);
    HG_MD5_CSTEP(HG_MD5_G, c, d, a, b, M[3], 0xf4d50d87, 14);
    HG_MD5_CSTEP(HG_MD5_G, b, c, d, a, M[8], 0x455a14ed, 20);
    HG_MD5_CSTEP(HG_MD5_G, a, b, c, d, M[13], 0xa9e3e905, 5);
    HG_MD5_CSTEP(HG_MD5_G, d, a, b, c, M[2], 0xfcefa3f8, 9);
    HG_MD5_CSTEP(HG_MD5_G, c, d, a, b, M[7], 0x676f02d9, 14);
    HG_MD5_CSTEP(HG_MD5_G, b, c, d, a, M[12], 0x8d2a4c8a, 20);

    HG_MD5_CSTEP(HG_MD5_H, a, b, c, d, M[5], 0xfffa3942, 4);
    HG_MD5_CSTEP(HG_MD5_H, d, a, b, c, M[8], 0x8771f681, 11);
    HG_MD5_CSTEP(HG_MD5_H, c, d, a, b, M[11], 0x6d9d6122, 16);
    HG_MD5_CSTEP(HG_MD5_H, b, c, d, a, M[14], 0xfde5380c, 23);
    HG_MD5_CSTEP(HG_MD5_H, a, b, c, d, M[1], 0xa4beea44, 4);
    HG_MD5_CSTEP(HG_MD5_H, d, a, b, c, M[4], 0x4bdecfa9, 11);
    HG_MD5_CSTEP(HG_MD5_H, c, d, a, b, M[7], 0xf6bb4b60, 16);
    HG_MD5_CSTEP(HG_MD5_H, b, c, d, a, M[10], 0xbebfbc70, 23);
    HG_MD5_CSTEP(HG_MD5_H, a, b, c, d, M[13], 0x289b7ec6, 4);
    HG_MD5_CSTEP(HG_MD5_H, d, a, b, c, M[0], 0xeaa127fa, 11);
    HG_MD5_CSTEP(HG_MD5_H, c, d, a, b, M[3], 0xd4ef3085, 16);
    HG_MD5_CSTEP(HG_MD5_H, b, c, d, a, M[6], 0x04881d05, 23);
    HG_MD5_CSTEP(HG_MD5_H, a, b, c, d, M[9], 0xd9d4d039, 4);
    HG_MD5_CSTEP(HG_MD5_H, d, a, b, c, M[12], 0xe6db99e5, 11);
    HG_MD5_CSTEP(HG_MD5_H, c, d, a, b, M[15], 0x1fa27cf8, 16);
    HG_MD5_CSTEP(HG_MD5_H, b, c, d, a, M[2], 0xc4ac5665, 23);

    HG_MD5_CSTEP(HG_MD5_I, a, b, c, d, M[0], 0xf4292244, 6);
    HG_MD5_CSTEP(HG_MD5_I, d, a, b, c, M[7], 0x432aff97, 10);
    HG_MD5_CSTEP(HG_MD5_I, c, d, a, b, M[14], 0xab9423a7, 15);
    HG_MD5_CSTEP(HG_MD5_I, b, c, d, a, M[5], 0xfc93a039, 21);
    HG_MD5_CSTEP(HG_MD5_I, a, b, c, d, M[12], 0x655b59c3, 6);
    HG_MD5_CSTEP(HG_MD5_I, d, a, b, c, M[3], 0x8f0ccc92, 10);
    HG_MD5_CSTEP(HG_MD5_I, c, d, a, b, M[10], 0xffeff47d, 15);
    HG_MD5_CSTEP(HG_MD5_I, b, c, d, a, M[1], 0x85845dd1, 21);
    HG_MD5_CSTEP(HG_MD5_I, a, b, c, d, M[8], 0x6fa87e4f, 6);
    HG_MD5_CSTEP(HG_MD5_I, d, a, b, c, M[15], 0xfe2ce6e0, 10);
    HG_MD5_CSTEP(HG_MD5_I, c, d, a, b, M[6], 0xa3014314, 15);
    HG_MD5_CSTEP(HG_MD5_I, b, c, d, a, M[13], 0x4e0811a1, 21);
    HG_MD5_CSTEP(HG_MD5_I, a, b, c, d, M[4], 0xf7537e82, 6);
    HG_MD5_CSTEP(HG_MD5_I, d, a, b, c, M[11], 0xbd3af235, 10);
    HG_MD5_CSTEP(HG_MD5_I, c, d, a, b, M[2], 0x2ad7d2bb, 15);
    HG_MD5_CSTEP(HG_MD5_I, b, c, d, a, M[9], 0xeb86d391, 21);
}

struct Md5Chain : Md5 {
    __device__ __forceinline__ void compress(const uint32_t (&M)[16]) {
        uint32_t a = h[0], b = h[1], c = h[2], d = h[3];
        md5_rounds_chain(a, b, c, d, M);
        h[0] += a; h[1] += b; h[2] += c; h[3] += d;
    }
};

// ------------------------------------------------ adds on the FMA pipe -----
// On sm_103a the logic op, the funnel shift and the rotate-add (b + rotl(x, s)
// is one instruction) of an MD5 or SHA-1 step issue only to the integer ALU
// pipe, which accepts one warp instruction every other cycle per scheduler;
// the FMA pipe beside it also runs integer multiply-adds and otherwise idles
// in these kernels. An add written as a multiply-add by a run-time 1 (`one`,
// a kernel argument, so the compiler cannot fold the multiply away) runs on
// the FMA pipe. Each step follows a policy:
//   0  its adds as plain code (the compiler places them, mostly on the ALU);
//   1  the adds that do not wait for the step's logic op (a + M + K for MD5,
//      e + K + W for SHA-1) as plain code, the add of the logic op's result
//      on the FMA pipe;
//   2  all of its adds on the FMA pipe;
//   3  the add of two words known early (a + M for MD5, e + W for SHA-1) on
//      the FMA pipe, the rest plain: the step's dependent chain keeps the
//      short ALU add.
// A pattern packs the policies of eight consecutive steps, two bits each
// (step n uses bits 2(n mod 8) .. 2(n mod 8) + 1), repeated over the steps.
__device__ __forceinline__ uint32_t add_fma(uint32_t x, uint32_t y, uint32_t one) {
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(one), "r"(y));
    return r;
}
// x + k with k a constant (it lands in the instruction's immediate field).
__device__ __forceinline__ uint32_t add_fma_k(uint32_t x, uint32_t k, uint32_t one) {
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(one), "r"(k), "r"(x));
    return r;
}
__host__ __device__ constexpr int pol_of(uint32_t pat, int n) { return (int)((pat >> (2 * (n & 7))) & 3u); }
constexpr uint32_t kPolAllPlain = 0x0000u, kPolAll1 = 0x5555u, kPolAll2 = 0xAAAAu;

// RFC 1321 Sec. 3.4: the additive constants T[1..64], the message word each
// step reads and the rotation amounts, indexed by step n = 0..63.
constexpr uint32_t kMd5T[64] = {
    0xd76aa478, 0xe8c7b756, 0x242070db, 0xc1bdceee, 0xf57c0faf, 0x4787c62a, 0xa8304613, 0xfd469501,
    0x698098d8, 0x8b44f7af, 0xffff5bb1, 0x895cd7be, 0x6b901122, 0xfd987193, 0xa679438e, 0x49b40821,
    0xf61e2562, 0xc040b340, 0x265e5a51, 0xe9b6c7aa, 0xd62f105d, 0x02441453, 0xd8a1e681, 0xe7d3fbc8,
    0x21e1cde6, 0xc33707d6, 0xf4d50d87, 0x455a14ed, 0xa9e3e905, 0xfcefa3f8, 0x676f02d9, 0x8d2a4c8a,
    0xfffa3942, 0x8771f681, 0x6d9d6122, 0xfde5380c, 0xa4beea44, 0x4bdecfa9, 0xf6bb4b60, 0xbebfbc70,
    0x289b7ec6, 0xeaa127fa, 0xd4ef3085, 0x04881d05, 0xd9d4d039, 0xe6db99e5, 0x1fa27cf8, 0xc4ac5665,
    0xf4292244, 0x432aff97, 0xab9423a7, 0xfc93a039, 0x655b59c3, 0x8f0ccc92, 0xffeff47d, 0x85845dd1,
    0x6fa87e4f, 0xfe2ce6e0, 0xa3014314, 0x4e0811a1, 0xf7537e82, 0xbd3af235, 0x2ad7d2bb, 0xeb86d391,
};
__host__ __device__ constexpr int md5_msg(int n) {
    return n < 16 ? n : n < 32 ? (1 + 5 * n) % 16 : n < 48 ? (5 + 3 * n) % 16 : (7 * n) % 16;
}
__host__ __device__ constexpr int md5_rot(int n) {
    return (n < 16)   ? ((n & 3) == 0 ? 7 : (n & 3) == 1 ? 12 : (n & 3) == 2 ? 17 : 22)
           : (n < 32) ? ((n & 3) == 0 ? 5 : (n & 3) == 1 ? 9 : (n & 3) == 2 ? 14 : 20)
           : (n < 48) ? ((n & 3) == 0 ? 4 : (n & 3) == 1 ? 11 : (n & 3) == 2 ? 16 : 23)
                      : ((n & 3) == 0 ? 6 : (n & 3) == 1 ? 10 : (n & 3) == 2 ? 15 : 21);
}

// One MD5 step a = b + rotl(a + f + m + T, S) with the adds placed by policy
// P. A message word that is a compile-time constant (DATA false) is folded
// with T into one immediate.
template <int P, bool DATA, int S, uint32_t T>
__device__ __forceinline__ void md5_pstep(uint32_t &a, uint32_t b, uint32_t f, uint32_t m,
                                          uint32_t one) {
    uint32_t x;
    if constexpr (!DATA) {
        if constexpr (P == 2) x = add_fma(f, add_fma_k(a, m + T, one), one);
        else x = a + f + (m + T);
    } else if constexpr (P == 2) {
        x = add_fma(f, add_fma(m, add_fma_k(a, T, one), one), one);
    } else if constexpr (P == 1) {
        x = add_fma(f, a + m + T, one);
    } else if constexpr (P == 3) {
        x = add_fma(a, m, one) + f + T;
    } else {
        x = a + f + m + T;
    }
    a = rotl(x, S) + b;
}

// Step n on the state st = {a, b, c, d}: it writes word (-n) mod 4 and reads
// the next three in order. Bit i of DM says message word i is data (else a
// constant after inlining); data steps take their policy from pattern PD,
// constant steps from pattern PC.
template <int n, uint32_t DM, uint32_t PC, uint32_t PD>
__device__ __forceinline__ void md5_pstep_n(uint32_t (&st)[4], const uint32_t (&M)[16],
                                            uint32_t one) {
    constexpr int t = (4 - (n & 3)) & 3;
    constexpr int i = md5_msg(n);
    constexpr bool data = ((DM >> i) & 1u) != 0;
    constexpr int P = data ? pol_of(PD, n) : pol_of(PC, n);
    const uint32_t b = st[(t + 1) & 3], c = st[(t + 2) & 3], d = st[(t + 3) & 3];
    uint32_t f;
    if constexpr (n < 16) f = HG_MD5_F(b, c, d);
    else if constexpr (n < 32) f = HG_MD5_G(b, c, d);
    else if constexpr (n < 48) f = HG_MD5_H(b, c, d);
    else f = HG_MD5_I(b, c, d);
    md5_pstep<P, data, md5_rot(n), kMd5T[n]>(st[t], b, f, M[i], one);
}

template <uint32_t DM, uint32_t PC, uint32_t PD, int... N>
__device__ __forceinline__ void md5_psteps(uint32_t (&st)[4], const uint32_t (&M)[16], uint32_t one,
                                           std::integer_sequence<int, N...>) {
    (md5_pstep_n<N, DM, PC, PD>(st, M, one), ...);
}

// The first NSTEPS operations of MD5 (64, or 61 for the window test) with
// the adds split between the pipes by the patterns above.
template <int NSTEPS, uint32_t DM, uint32_t PC, uint32_t PD>
__device__ __forceinline__ void md5_rounds_split(uint32_t (&st)[4], const uint32_t (&M)[16],
                                                 uint32_t one) {
    md5_psteps<DM, PC, PD>(st, M, one, std::make_integer_sequence<int, NSTEPS>{});
}

// MD5 with the adds of every step placed by pattern PD (all message words
// are data). `one` must be set to a run-time 1 before compress.
template <uint32_t PD>
struct Md5Split : Md5 {
    uint32_t one;
    __device__ __forceinline__ void set_one(uint32_t v) { one = v; }
    __device__ __forceinline__ void compress(const uint32_t (&M)[16]) {
        uint32_t st[4] = {h[0], h[1], h[2], h[3]};
        md5_rounds_split<64, 0xffffu, kPolAllPlain, PD>(st, M, one);
        h[0] += st[0]; h[1] += st[1]; h[2] += st[2]; h[3] += st[3];
    }
};

// --------------------------------------------------------------- SHA-1 -----

struct Sha1 {
    static constexpr int kDigest = 20;
    static constexpr int kWords = 5;
    uint32_t h[5];
    __device__ __forceinline__ void init() {
        // FIPS 180-4 Sec. 5.3.1 initial hash value
        h[0] = 0x67452301u; h[1] = 0xefcdab89u; h[2] = 0x98badcfeu; h[3] = 0x10325476u;
        h[4] = 0xc3d2e1f0u;
    }
    __device__ __forceinline__ void set_one(uint32_t) {}
    // M: little-endian message words (byte-swapped here to the big-endian
    // words FIPS 180-4 Sec. 5.2.1 parses).
    __device__ __forceinline__ void compress(const uint32_t (&M)[16]) {
        uint32_t W[16];
#pragma unroll
        for (int i = 0; i < 16; i++) W[i] = bswap(M[i]);
        compress_be(W);
    }
    __device__ __forceinline__ void compress_be(uint32_t (&W)[16]) {
        uint32_t a = h[0], b = h[1], c = h[2], d = h[3], e = h[4];
#pragma unroll
        for (int t = 0; t < 80; t++) {
            if (t >= 16)
                W[t & 15] = rotl(W[(t - 3) & 15] ^ W[(t - 8) & 15] ^ W[(t - 14) & 15] ^ W[t & 15], 1);
            uint32_t f, k;
            if (t < 20)      { f = d ^ (b & (c ^ d));       k = 0x5a827999u; }
            else if (t < 40) { f = b ^ c ^ d;               k = 0x6ed9eba1u; }
            else if (t < 60) { f = (b & c) | (d & (b | c)); k = 0x8f1bbcdcu; }
            else             { f = b ^ c ^ d;               k = 0xca62c1d6u; }
            const uint32_t T = rotl(a, 5) + f + e + k + W[t & 15];
            e = d; d = c; c = rotl(b, 30); b = a; a = T;
        }
        h[0] += a; h[1] += b; h[2] += c; h[3] += d; h[4] += e;
    }
    // Bit length goes big-endian into the last two big-endian words, i.e.
    // byte-swapped into the little-endian message words 14, 15.
    __device__ __forceinline__ static void put_length(uint32_t (&M)[16], uint64_t bytes) {
        const uint64_t bits = bytes * 8u;
        M[14] = bswap((uint32_t)(bits >> 32)); M[15] = bswap((uint32_t)bits);
    }
    __device__ __forceinline__ uint32_t out_word(int i) const { return bswap(h[i]); }
};

// SHA-1 with the adds of round t placed by policy pol_of(PAT, t) (see the
// pipe policies above): T = rotl(a, 5) + f + e + K + W. `one` must be set to
// a run-time 1 before compress.
template <uint32_t PAT>
struct Sha1Split : Sha1 {
    uint32_t one;
    __device__ __forceinline__ void set_one(uint32_t v) { one = v; }
    __device__ __forceinline__ void compress(const uint32_t (&M)[16]) {
        uint32_t W[16];
#pragma unroll
        for (int i = 0; i < 16; i++) W[i] = bswap(M[i]);
        uint32_t a = h[0], b = h[1], c = h[2], d = h[3], e = h[4];
#pragma unroll
        for (int t = 0; t < 80; t++) {
            if (t >= 16)
                W[t & 15] = rotl(W[(t - 3) & 15] ^ W[(t - 8) & 15] ^ W[(t - 14) & 15] ^ W[t & 15], 1);
            uint32_t f, k;
            if (t < 20)      { f = d ^ (b & (c ^ d));       k = 0x5a827999u; }
            else if (t < 40) { f = b ^ c ^ d;               k = 0x6ed9eba1u; }
            else if (t < 60) { f = (b & c) | (d & (b | c)); k = 0x8f1bbcdcu; }
            else             { f = b ^ c ^ d;               k = 0xca62c1d6u; }
            const int pol = pol_of(PAT, t);
            uint32_t x;
            if (pol == 2) x = add_fma(f, add_fma(W[t & 15], add_fma_k(e, k, one), one), one);
            else if (pol == 1) x = add_fma(f, e + k + W[t & 15], one);
            else if (pol == 3) x = add_fma(e, W[t & 15], one) + f + k;
            else x = f + e + k + W[t & 15];
            const uint32_t T = rotl(a, 5) + x;
            e = d; d = c; c = rotl(b, 30); b = a; a = T;
        }
        h[0] += a; h[1] += b; h[2] += c; h[3] += d; h[4] += e;
    }
};

// Very few latency-bound digest chains (large fixed blocks: 1024 chains of
// 1 MiB) run on half warps: a dependent MD5 step measured about 20 cycles
// with 16 of a warp's lanes active against 27 with all 32 (1 MiB blocks:
// 98 vs 92 GB/s). With more chains the integer pipes are the limit and full
// warps win (16384 SHA-1 chains of 64 KiB: 1570 vs 868 GB/s).
constexpr uint64_t kHalfWarpChainsMax = 4096;

// Task index of this thread when tasks are dealt to the first `lanes` (16 or
// 32) lanes of every warp; false on the idle lanes.
__device__ __forceinline__ bool chain_task(uint64_t &i, uint32_t lanes) {
    const uint32_t lane = threadIdx.x & 31;
    if (lane >= lanes) return false;
    i = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32 * lanes + lane;
    return true;
}

// Asks for the 16 bytes at p to be brought into L2 (no register result).
__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// The end of a digest of the len bytes at msg once its full 64-byte blocks
// are compressed: the remaining bytes, the 0x80 marker, zeros and the length
// (one or two blocks), assembled from byte loads inside the message.
template <class H>
__device__ __forceinline__ void hash_tail(const uint8_t *__restrict__ msg, uint64_t len, H &hs) {
    const uint32_t rem = (uint32_t)(len & 63);
    const uint8_t *t = msg + ((len >> 6) << 6);
    uint32_t M[16];
#pragma unroll
    for (int i = 0; i < 16; i++) {
        uint32_t w = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t idx = 4 * i + j;
            uint32_t byte = idx < rem ? (uint32_t)t[idx] : (idx == rem ? 0x80u : 0u);
            w |= byte << (8 * j);
        }
        M[i] = w;
    }
    if (rem < 56) {
        H::put_length(M, len);
        hs.compress(M);
    } else {
        hs.compress(M);
        uint32_t Z[16];
#pragma unroll
        for (int i = 0; i < 16; i++) Z[i] = 0;
        H::put_length(Z, len);
        hs.compress(Z);
    }
}

// Digest of the len bytes at msg, which may start at any byte address. Full
// 64-byte blocks are read as aligned 16-byte vectors; for a message that does
// not start on a 16-byte boundary they are shifted into place (the aligned
// vectors at either end stay inside the 16-byte granules that hold the first
// and last message bytes, so they never cross a page). The final partial block
// and the padding are assembled from byte loads inside the message.
template <class H>
__device__ void hash_range(const uint8_t *__restrict__ msg, uint64_t len, H &hs) {
    hs.init();
    const uint64_t nfull = len >> 6;
    const uintptr_t addr = reinterpret_cast<uintptr_t>(msg);
    const uint32_t sh = (uint32_t)(addr & 15);
    const uint32_t q = sh >> 2, r8 = (sh & 3) * 8;
    const uint4 *p = reinterpret_cast<const uint4 *>(addr - sh);
    // A chain is one dependent sequence: the loads of block k+1 are issued
    // before block k is compressed, and an L2 prefetch eight blocks ahead
    // keeps those loads from waiting on HBM. (Loading two blocks ahead into
    // registers measured slower for chunk digests: more live registers and
    // moves per block.)
    if (sh == 0) {
        // aligned message: four 16-byte loads per block, no shifting
        uint4 a0 = make_uint4(0, 0, 0, 0), a1 = a0, a2 = a0, a3 = a0;
        if (nfull) { a0 = __ldg(p); a1 = __ldg(p + 1); a2 = __ldg(p + 2); a3 = __ldg(p + 3); }
        for (uint64_t k = 0; k < nfull; k++) {
            const uint32_t M[16] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w,
                                    a2.x, a2.y, a2.z, a2.w, a3.x, a3.y, a3.z, a3.w};
            if (k + 8 < nfull) prefetch_l2(p + 4 * (k + 8));
            if (k + 1 < nfull) {
                const uint4 *q4 = p + 4 * (k + 1);
                a0 = __ldg(q4); a1 = __ldg(q4 + 1); a2 = __ldg(q4 + 2); a3 = __ldg(q4 + 3);
            }
            hs.compress(M);
        }
    } else {
        // unaligned message: five aligned loads per block, shifted into place
        uint4 x0 = make_uint4(0, 0, 0, 0), x1 = x0, x2 = x0, x3 = x0, x4 = x0;
        if (nfull) {
            x0 = __ldg(p); x1 = __ldg(p + 1); x2 = __ldg(p + 2); x3 = __ldg(p + 3); x4 = __ldg(p + 4);
        }
        for (uint64_t k = 0; k < nfull; k++) {
            const uint32_t v[20] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w,
                                    x2.x, x2.y, x2.z, x2.w, x3.x, x3.y, x3.z, x3.w,
                                    x4.x, x4.y, x4.z, x4.w};
            if (k + 8 < nfull) prefetch_l2(p + 4 * (k + 8));
            if (k + 1 < nfull) {
                const uint4 *q4 = p + 4 * (k + 1);
                x0 = __ldg(q4); x1 = __ldg(q4 + 1); x2 = __ldg(q4 + 2); x3 = __ldg(q4 + 3);
                x4 = __ldg(q4 + 4);
            }
            // shift by q words, then by r8 bits
            uint32_t u[17];
#pragma unroll
            for (int i = 0; i < 17; i++) {
                const uint32_t s1 = (q & 1) ? v[i + 1] : v[i];
                const uint32_t s2 = (q & 1) ? v[i + 3] : v[i + 2];
                u[i] = (q & 2) ? s2 : s1;
            }
            uint32_t M[16];
#pragma unroll
            for (int i = 0; i < 16; i++) M[i] = r8 ? __funnelshift_r(u[i], u[i + 1], r8) : u[i];
            hs.compress(M);
        }
    }
    hash_tail(msg, len, hs);
}

// ------------------------------------------------ staged chains ----------
// A chain's own loads of the next block cannot hide its latency once several
// lanes of a warp run chains over different regions (each warp load then
// touches one line per lane): measured per 64-byte MD5 block, 1330 cycles
// with one block loaded ahead into registers against 925 for the compression
// alone. hash_range_staged instead copies the message into a per-thread ring
// of 16-byte granules in shared memory with asynchronous copies
// (cp.async.cg) kStageDepth blocks ahead of the compression: 960-1000 cycles
// per block from 1 to 32 lanes a warp. The ring has kStageSlots granules (a
// power of two, at least the 4 x depth + 5 a block in use and the blocks in
// flight span) and threads sit kStageStride granules apart, an odd stride, so
// that a warp's lanes spread over the shared-memory banks.
constexpr int kStageDepth = 4;
constexpr uint32_t kStageSlots = 32;
constexpr uint32_t kStageStride = kStageSlots + 1;
static_assert(kStageSlots >= 4 * kStageDepth + 5 && (kStageSlots & (kStageSlots - 1)) == 0,
              "staging ring too small");
// Shared-memory bytes of the rings of `threads` threads.
constexpr size_t stage_bytes(unsigned threads) { return (size_t)threads * kStageStride * 16u; }

__device__ __forceinline__ void cp_async16(uint4 *dst, const uint4 *src) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// This thread's ring in the kernel's dynamic shared memory (launched with
// stage_bytes(blockDim.x) of it).
__device__ __forceinline__ uint4 *stage_ring_dyn() {
    extern __shared__ __align__(16) uint4 hg_stage_dyn[];
    return hg_stage_dyn + threadIdx.x * kStageStride;
}

// Digest of the len bytes at msg (any byte address), as hash_range, with the
// full blocks read through `ring` (this thread's kStageStride granules of
// shared memory). Copy group j brings the granules of block j not brought
// before: granules 0..3 (and 4 when the message is not 16-byte aligned) for
// j = 0, 4j + o .. 4j + 3 + o after (o = 1 when unaligned). Every granule
// holds message bytes, as in hash_range. Group j + depth is issued after
// block j's words are read out, so the slots it overwrites are free.
template <class H, bool UNALIGNED>
__device__ __forceinline__ void staged_blocks(const uint4 *__restrict__ p, uint64_t nfull, uint32_t sh,
                                              H &hs, uint4 *ring) {
    constexpr uint32_t o = UNALIGNED ? 1u : 0u, W = kStageSlots - 1;
    const uint32_t q = sh >> 2, r8 = (sh & 3) * 8;
    auto issue = [&](uint64_t j) {
        if (j < nfull) {
            const uint64_t g0 = 4 * j + (j ? o : 0u);
#pragma unroll
            for (uint32_t i = 0; i < 4; i++) cp_async16(ring + (((uint32_t)g0 + i) & W), p + g0 + i);
            if (UNALIGNED && j == 0) cp_async16(ring + 4, p + 4);
        }
        cp_async_commit();
    };
#pragma unroll
    for (int j = 0; j < kStageDepth; j++) issue((uint64_t)j);
    for (uint64_t k = 0; k < nfull; k++) {
        cp_async_wait<kStageDepth - 1>();       // groups 0..k have landed
        const uint32_t g = (uint32_t)(4 * k);
        uint32_t M[16];
        if constexpr (!UNALIGNED) {
#pragma unroll
            for (uint32_t i = 0; i < 4; i++) {
                const uint4 x = ring[(g + i) & W];
                M[4 * i] = x.x; M[4 * i + 1] = x.y; M[4 * i + 2] = x.z; M[4 * i + 3] = x.w;
            }
        } else {
            uint32_t v[20];
#pragma unroll
            for (uint32_t i = 0; i < 5; i++) {
                const uint4 x = ring[(g + i) & W];
                v[4 * i] = x.x; v[4 * i + 1] = x.y; v[4 * i + 2] = x.z; v[4 * i + 3] = x.w;
            }
            // shift by q words, then by r8 bits
            uint32_t u[17];
#pragma unroll
            for (int i = 0; i < 17; i++) {
                const uint32_t s1 = (q & 1) ? v[i + 1] : v[i];
                const uint32_t s2 = (q & 1) ? v[i + 3] : v[i + 2];
                u[i] = (q & 2) ? s2 : s1;
            }
#pragma unroll
            for (int i = 0; i < 16; i++) M[i] = r8 ? __funnelshift_r(u[i], u[i + 1], r8) : u[i];
        }
        issue(k + kStageDepth);
        hs.compress(M);
    }
    cp_async_wait<0>();
}

template <class H>
__device__ void hash_range_staged(const uint8_t *__restrict__ msg, uint64_t len, H &hs,
                                  uint4 *ring) {
    hs.init();
    const uintptr_t addr = reinterpret_cast<uintptr_t>(msg);
    const uint32_t sh = (uint32_t)(addr & 15);
    const uint4 *p = reinterpret_cast<const uint4 *>(addr - sh);
    if (sh == 0) staged_blocks<H, false>(p, len >> 6, 0u, hs, ring);
    else staged_blocks<H, true>(p, len >> 6, sh, hs, ring);
    hash_tail(msg, len, hs);
}

template <class H>
__device__ __forceinline__ void store_digest(const H &hs, uint8_t *out) {
    // digests are written word by word; `out` is 4-byte aligned for both algos
    uint32_t *o = reinterpret_cast<uint32_t *>(out);
#pragma unroll
    for (int i = 0; i < H::kWords; i++) o[i] = hs.out_word(i);
}

}  // namespace hg
