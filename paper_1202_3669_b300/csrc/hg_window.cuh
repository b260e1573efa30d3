// Window-hash building blocks shared by the single-stream and the batched
// window kernels (Sec. 2.1 / Sec. 3.2.2: MD5 of a small window at every byte
// offset, compared with a predefined value).
#pragma once
#include <cstdint>

#include "hg_device.cuh"
#include "hg_internal.h"

namespace hg {

constexpr int kHalo = 64;                              // >= window - 1, multiple of 16
constexpr int kSmemBytes = kHalo + (int)kWinTile + 16; // + a zeroed 16-byte pad
constexpr long kWaitLimit = 1L << 22;                  // bounded mbarrier polling
// Pipe policies of the window hash's constant-word and data-word steps: the
// constant-word steps (42 of the 61) move both adds to the FMA pipe, the
// data-word steps move the add of the logic op's result (policy 1). Measured
// on a 64 MiB pass (20-byte window), one-warp CTAs: 0.616 ms, against 0.630
// with the data-word adds left on the ALU, 0.682 with every add on the ALU,
// 0.74-0.76 with policies 2/3 on the data-word steps. (In eight-warp CTAs at
// 32 registers the constant-word split alone took 0.688 -> 0.651 ms, ALU-pipe
// instructions per window 191 -> 149, FMA-pipe 20 -> 104.)
constexpr uint32_t kWinPolConst = kPolAll2, kWinPolData = kPolAll1;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// MD5 of one window given its data words d[] (little-endian, the last word may
// carry bytes past the window, which are masked). Only word A of the final
// state is formed: the window test reads the first four digest bytes. PC / PD
// split the adds of the constant-word / data-word steps between the integer
// ALU and FMA pipes (pipe policies in hg_device.cuh); `one` is a run-time 1.
template <int W, uint32_t PC, uint32_t PD>
__device__ __forceinline__ uint32_t window_a(const uint32_t (&d)[(W + 3) / 4], uint32_t one) {
    constexpr int NW = (W + 3) / 4;
    uint32_t M[16];
#pragma unroll
    for (int i = 0; i < 16; i++) M[i] = 0;
#pragma unroll
    for (int i = 0; i < NW; i++) M[i] = d[i];
    if (W % 4 == 0) {
        M[W / 4] = 0x80u;                             // padding marker after the data
    } else {
        constexpr uint32_t keep = (1u << (8 * (W % 4))) - 1u;
        M[NW - 1] = (d[NW - 1] & keep) | (0x80u << (8 * (W % 4)));
    }
    M[14] = (uint32_t)W * 8u;                         // bit length, little-endian
    if constexpr (PC == kPolAllPlain && PD == kPolAllPlain) {
        uint32_t a = kMd5A, b = kMd5B, c = kMd5C, dd = kMd5D;
        md5_rounds<false>(a, b, c, dd, M);
        return a + kMd5A;
    } else {
        // words 0 .. NW-1 carry window bytes; the rest are constants
        uint32_t st[4] = {kMd5A, kMd5B, kMd5C, kMd5D};
        md5_rounds_split<61, (1u << NW) - 1u, PC, PD>(st, M, one);
        return st[0] + kMd5A;
    }
}

// Window number S (0..6) of a group, counted in bytes from word cur[0].
template <int W, int S, uint32_t PC, uint32_t PD>
__device__ __forceinline__ uint32_t window_at(const uint32_t (&cur)[(W + 3) / 4 + 2], uint32_t one) {
    constexpr int NW = (W + 3) / 4, SH = S & 3, WO = S >> 2;
    uint32_t d[NW];
#pragma unroll
    for (int k = 0; k < NW; k++)
        d[k] = SH == 0 ? cur[WO + k] : __funnelshift_r(cur[WO + k], cur[WO + k + 1], 8 * SH);
    return window_a<W, PC, PD>(d, one);
}

// Window hash for a window length known only at run time (any 1..55): the
// message words are gathered byte by byte from shared memory.
__device__ __forceinline__ uint32_t window_a_rt(const uint8_t *sbuf, int start, int w) {
    uint32_t M[16];
#pragma unroll
    for (int i = 0; i < 14; i++) {
        uint32_t x = 0;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int k = 4 * i + j;
            const uint32_t byte = k < w ? (uint32_t)sbuf[start + k] : (k == w ? 0x80u : 0u);
            x |= byte << (8 * j);
        }
        M[i] = x;
    }
    M[14] = (uint32_t)w * 8u;
    M[15] = 0;
    uint32_t a = kMd5A, b = kMd5B, c = kMd5C, d = kMd5D;
    md5_rounds<false>(a, b, c, d, M);
    return a + kMd5A;
}

// Tile staging helpers: one bulk asynchronous copy (TMA engine) into shared
// memory, completion tracked by an mbarrier with a bounded wait.
__device__ __forceinline__ void mbar_init(uint32_t mb) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t mb) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(mb)
        : "memory");
}

// Bounded wait on phase `parity` of mbarrier mb; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t parity) {
    for (long it = 0; it < kWaitLimit; it++)
        if (mbar_try_wait(mb, parity)) return true;
    return false;
}

// The 32 candidate bits of one thread: window ends [p0, p0 + 32) where p0 is
// local byte kHalo + 32t of the staged tile sbuf (the tile starts kHalo bytes
// before its first window end).
template <int W, uint32_t PC = kWinPolConst, uint32_t PD = kWinPolData>
__device__ __forceinline__ uint32_t window_bits32(const uint8_t *sbuf, int t, uint32_t wlen,
                                                  uint32_t mask, uint32_t magic, uint32_t one) {
    constexpr int NW = W ? (W + 3) / 4 : 1;
    constexpr int OFF = kHalo - (W ? W - 1 : 0);      // local byte of window 0's start
    constexpr int B0 = OFF / 4, R0 = OFF % 4;
    // With T threads the buffer holds kHalo + 32T + 16 bytes and thread T-1 reads
    // words up to 8(T-1) + B0 + 7 + NW + 2: inside the buffer for every T exactly
    // when B0 + NW + 1 < kHalo/4 + 4.
    static_assert(W == 0 || B0 + NW + 1 < kHalo / 4 + 4, "window words read past the staged bytes");
    uint32_t bits = 0;
    if constexpr (W > 0) {
        const uint32_t *sw = reinterpret_cast<const uint32_t *>(sbuf);
        uint32_t cur[NW + 2];
#pragma unroll
        for (int i = 0; i < NW + 2; i++) cur[i] = sw[8 * t + B0 + i];
#pragma unroll 1
        for (int g = 0; g < 8; g++) {
            const uint32_t h0 = window_at<W, R0 + 0, PC, PD>(cur, one);
            const uint32_t h1 = window_at<W, R0 + 1, PC, PD>(cur, one);
            const uint32_t h2 = window_at<W, R0 + 2, PC, PD>(cur, one);
            const uint32_t h3 = window_at<W, R0 + 3, PC, PD>(cur, one);
            const uint32_t nib = (uint32_t)((h0 & mask) == magic) |
                                 ((uint32_t)((h1 & mask) == magic) << 1) |
                                 ((uint32_t)((h2 & mask) == magic) << 2) |
                                 ((uint32_t)((h3 & mask) == magic) << 3);
            bits |= nib << (4 * g);
#pragma unroll
            for (int i = 0; i < NW + 1; i++) cur[i] = cur[i + 1];
            cur[NW + 1] = sw[8 * t + B0 + g + NW + 2];   // stays inside the padded tile
        }
    } else {
        const int first = kHalo + 32 * t - (int)(wlen - 1);
#pragma unroll 1
        for (int j = 0; j < 32; j++)
            bits |= (uint32_t)((window_a_rt(sbuf, first + j, (int)wlen) & mask) == magic) << j;
    }
    return bits;
}

// Clear the bits of window ends before the first full window (p < wlen - 1)
// and past the input (p >= n).
__device__ __forceinline__ uint32_t clip_bits(uint32_t bits, uint64_t p0, uint32_t wlen, uint64_t n) {
    const uint64_t lo = (uint64_t)(wlen - 1) > p0 ? (uint64_t)(wlen - 1) - p0 : 0;
    const uint64_t hi = n > p0 ? n - p0 : 0;
    if (lo >= 32 || hi == 0) return 0;
    if (lo) bits &= ~0u << lo;
    if (hi < 32) bits &= (1u << hi) - 1u;
    return bits;
}

}  // namespace hg
