// Rabin fingerprint window: device building blocks shared by the
// single-buffer kernel (hg_rabin.cu) and the batch-job kernel (hg_job.cu).
//
// The fingerprint of a byte string is its polynomial over GF(2) (bytes most
// significant first, bit 7 high) modulo the irreducible degree-31 polynomial
// HG_RABIN_POLY. It rolls: with f the remainder of the window ending at
// p - 1 (W bytes),
//     f' = (f x^8 + b_p + b_{p-W} x^(8W)) mod P
//        = ((f << 8) | b_p) ^ T[f >> 23] ^ U[b_{p-W}]
// where T[t] = t x^31 mod P (plus bit 31 set to t's bit 0, which cancels the
// bit the 32-bit shift keeps) and U[b] = b x^(8W) mod P. A thread rolls along
// 128 consecutive window ends after W warm-up steps over the bytes before
// them. T and U (256 words each) are built by each CTA and replicated 32
// times in shared memory, [value][lane], so every lane reads its own bank.
#pragma once
#include <cstdint>

#include "hg_internal.h"

namespace hg {
namespace rabin {

constexpr uint32_t kPoly = HG_RABIN_POLY;
constexpr int kThreads = 256;
constexpr int kStrip = 128;                                    // window ends per thread
constexpr int kPre = 64;                                       // bytes loaded before a strip
constexpr uint64_t kGroup = (uint64_t)kThreads * kStrip;       // 32 KiB of window ends
constexpr uint32_t kTilesPerGroup = (uint32_t)(kGroup / kWinTile);
constexpr size_t kSmem = 2 * 256 * 32 * sizeof(uint32_t);      // T and U, 32 replicas each
static_assert(kGroup % kWinTile == 0, "a group is whole tiles");
static_assert(kWinTile / kStrip == 64, "two warps per tile");

// (f << 8) | byte k of w, in one byte permute: result bytes = {w.k, f.0, f.1, f.2}
__device__ __forceinline__ uint32_t shift_in(uint32_t f, uint32_t w, int k) {
    return __byte_perm(f, w, 0x2100u | (uint32_t)(4 + k));
}

// One rolling step: s = (f << 8) | b_in, top = f >> 23, out = the byte leaving.
__device__ __forceinline__ uint32_t roll(uint32_t s, uint32_t top, uint32_t out,
                                         const uint32_t *__restrict__ T,
                                         const uint32_t *__restrict__ U) {
    return s ^ T[top << 5] ^ U[out << 5];
}

// Fills the CTA's tables for a window of wlen bytes: threads 0..255 build one
// entry each (tabs holds 2 x 256 x 32 words); every thread of the CTA must
// call it (it synchronises the CTA).
static_assert(kThreads >= 256 && kThreads % 32 == 0, "one table entry per thread of the first 256");
__device__ __forceinline__ void build_tables(uint32_t *tabs, uint32_t wlen) {
    const int t = threadIdx.x, lane = t & 31;
    if (t < 256) {
        // T[v] = v x^31 mod P, bit 31 = v's bit 0; thread t builds entry t and
        // writes its 32 replicas in rotated order (one bank per lane per store)
        uint32_t r = (uint32_t)t;
        for (int i = 0; i < 31; i++) {
            r <<= 1;
            if (r & 0x80000000u) r ^= kPoly;
        }
        r ^= ((uint32_t)t & 1u) << 31;
        for (int l = 0; l < 32; l++) tabs[t * 32 + ((l + lane) & 31)] = r;
    }
    __syncthreads();
    if (t < 256) {
        // U[b] = b x^(8W) mod P: W byte steps from b, with T
        uint32_t r = (uint32_t)t;
        for (uint32_t i = 0; i < wlen; i++) r = (r << 8) ^ tabs[(r >> 23) * 32 + lane];
        for (int l = 0; l < 32; l++) tabs[256 * 32 + t * 32 + ((l + lane) & 31)] = r;
    }
    __syncthreads();
}

// Candidate bits of the 128 window ends [a, a + 128) of the n-byte buffer in
// (bit m of bits[m / 32] for end a + m). GENERAL accepts any alignment of in
// (the strip is realigned from 16-byte loads); otherwise in must be 16-byte
// aligned. Interior strips keep the strip in registers with compile-time byte
// indexes; edges and window lengths without a specialisation take byte loads
// (bytes outside [0, n) read as 0: a leading zero byte does not change a
// polynomial).
template <int W, bool GENERAL>
__device__ __forceinline__ void strip_bits(const uint8_t *__restrict__ in, uint64_t n, uint64_t a,
                                           uint32_t wlen, uint32_t mask, uint32_t magic,
                                           const uint32_t *__restrict__ T,
                                           const uint32_t *__restrict__ U, uint32_t (&bits)[4]) {
    bits[0] = bits[1] = bits[2] = bits[3] = 0;
    if (a >= n) return;
    constexpr int NW = (kPre + kStrip) / 4;
    const bool interior = GENERAL ? (a >= (uint64_t)kPre + 16 && a + kStrip + 16 <= n)
                                  : (a >= (uint64_t)kPre && a + kStrip <= n);
    if (W && interior) {
        uint32_t w[NW];
        if constexpr (GENERAL) {
            // 13 aligned loads cover [a - 64 - sh, a + 144 - sh), inside [0, n);
            // word j of the strip = bytes 4j .. 4j+3 from a - 64
            const uintptr_t addr = reinterpret_cast<uintptr_t>(in + a - kPre);
            const uint32_t sh = (uint32_t)(addr & 15), q = sh >> 2, r8 = (sh & 3) * 8;
            const uint4 *p4 = reinterpret_cast<const uint4 *>(addr - sh);
            uint32_t raw[NW + 4];
#pragma unroll
            for (int i = 0; i < (NW + 4) / 4; i++) {
                const uint4 v = __ldg(p4 + i);
                raw[4 * i] = v.x; raw[4 * i + 1] = v.y; raw[4 * i + 2] = v.z; raw[4 * i + 3] = v.w;
            }
            uint32_t u[NW + 1];
#pragma unroll
            for (int j = 0; j < NW + 1; j++) {
                const uint32_t s1 = (q & 1) ? raw[j + 1] : raw[j];
                const uint32_t s2 = (q & 1) ? raw[j + 3] : raw[j + 2];
                u[j] = (q & 2) ? s2 : s1;
            }
#pragma unroll
            for (int j = 0; j < NW; j++) w[j] = __funnelshift_r(u[j], u[j + 1], r8);
        } else {
            const uint4 *p4 = reinterpret_cast<const uint4 *>(in + a - kPre);
#pragma unroll
            for (int i = 0; i < NW / 4; i++) {
                const uint4 v = __ldg(p4 + i);
                w[4 * i] = v.x; w[4 * i + 1] = v.y; w[4 * i + 2] = v.z; w[4 * i + 3] = v.w;
            }
        }
        uint32_t f = 0;
#pragma unroll
        for (int i = kPre - W; i < kPre; i++)                 // warm-up: W bytes in
            f = shift_in(f, w[i >> 2], i & 3) ^ T[(f >> 23) << 5];
#pragma unroll
        for (int m = 0; m < kStrip; m++) {
            const int i = kPre + m, o = kPre + m - W;
            const uint32_t ob = (w[o >> 2] >> (8 * (o & 3))) & 0xffu;
            f = roll(shift_in(f, w[i >> 2], i & 3), f >> 23, ob, T, U);
            bits[m >> 5] |= (uint32_t)((f & mask) == magic) << (m & 31);
        }
    } else {
        auto ld = [&](int64_t q) -> uint32_t {
            return (q >= 0 && (uint64_t)q < n) ? (uint32_t)in[q] : 0u;
        };
        uint32_t f = 0;
        for (int64_t q = (int64_t)a - (int64_t)wlen; q < (int64_t)a; q++)
            f = ((f << 8) | ld(q)) ^ T[(f >> 23) << 5];
        for (int m = 0; m < kStrip; m++) {
            const uint64_t pos = a + (uint64_t)m;
            if (pos >= n) break;
            const uint32_t ob = ld((int64_t)pos - (int64_t)wlen);
            f = roll((f << 8) | ld((int64_t)pos), f >> 23, ob, T, U);
            if (pos + 1 >= wlen && (f & mask) == magic) bits[m >> 5] |= 1u << (m & 31);
        }
    }
}

}  // namespace rabin
}  // namespace hg
