/*
 * SHA-1 as FIPS 180-4 defines it -- oracle, test infrastructure only.
 *
 * The paper only uses MD5 (Sec. 3.2.2); SHA-1 is the second standard digest
 * the library offers for the same direct and per-chunk hashing. Written from
 * FIPS 180-4: padding (Sec. 5.1.1), big-endian parsing (Sec. 5.2.1), initial
 * hash value (Sec. 5.3.1), functions (Sec. 4.1.1), constants (Sec. 4.2.1) and
 * the computation (Sec. 6.1.2). The four constants are the integer parts of
 * 2^30 * sqrt(2), sqrt(3), sqrt(5) and sqrt(10), computed here rather than
 * typed in.
 */
#include <math.h>
#include <pthread.h>
#include <string.h>
#include "hg_oracle.h"

static uint32_t rotl(uint32_t x, int s) { return (x << s) | (x >> (32 - s)); }

static uint32_t Kc[4];
static pthread_once_t k_once = PTHREAD_ONCE_INIT;

static void make_constants(void) {
    const double r[4] = {2.0, 3.0, 5.0, 10.0};
    for (int i = 0; i < 4; i++) Kc[i] = (uint32_t)floor(1073741824.0 * sqrt(r[i]));
}

/* FIPS 180-4 Sec. 4.1.1: Ch, Parity, Maj by t range. */
static uint32_t f_t(int t, uint32_t x, uint32_t y, uint32_t z) {
    if (t < 20) return (x & y) ^ (~x & z);
    if (t < 40) return x ^ y ^ z;
    if (t < 60) return (x & y) ^ (x & z) ^ (y & z);
    return x ^ y ^ z;
}

static void sha1_block(uint32_t Hs[5], const uint8_t blk[64]) {
    uint32_t W[80];
    for (int t = 0; t < 16; t++)
        W[t] = ((uint32_t)blk[4 * t] << 24) | ((uint32_t)blk[4 * t + 1] << 16) |
               ((uint32_t)blk[4 * t + 2] << 8) | (uint32_t)blk[4 * t + 3];
    for (int t = 16; t < 80; t++) W[t] = rotl(W[t - 3] ^ W[t - 8] ^ W[t - 14] ^ W[t - 16], 1);
    uint32_t a = Hs[0], b = Hs[1], c = Hs[2], d = Hs[3], e = Hs[4];
    for (int t = 0; t < 80; t++) {
        uint32_t T = rotl(a, 5) + f_t(t, b, c, d) + e + Kc[t / 20] + W[t];
        e = d; d = c; c = rotl(b, 30); b = a; a = T;
    }
    Hs[0] += a; Hs[1] += b; Hs[2] += c; Hs[3] += d; Hs[4] += e;
}

void hgo_sha1(const uint8_t *msg, uint64_t len, uint8_t out[20]) {
    pthread_once(&k_once, make_constants);
    /* Sec. 5.3.1 initial hash value. */
    uint32_t Hs[5] = {0x67452301u, 0xefcdab89u, 0x98badcfeu, 0x10325476u, 0xc3d2e1f0u};
    uint64_t full = len / 64;
    for (uint64_t i = 0; i < full; i++) sha1_block(Hs, msg + 64 * i);
    /* Sec. 5.1.1: a 1 bit, zeros to 448 mod 512 bits, then the 64-bit
     * big-endian bit length. */
    uint8_t tail[128];
    uint64_t rem = len - 64 * full;
    memset(tail, 0, sizeof tail);
    memcpy(tail, msg + 64 * full, (size_t)rem);
    tail[rem] = 0x80;
    uint64_t tlen = (rem < 56) ? 64 : 128;
    uint64_t bits = len * 8u;
    for (int j = 0; j < 8; j++) tail[tlen - 1 - j] = (uint8_t)(bits >> (8 * j));
    for (uint64_t off = 0; off < tlen; off += 64) sha1_block(Hs, tail + off);
    for (int w = 0; w < 5; w++)
        for (int j = 0; j < 4; j++) out[4 * w + j] = (uint8_t)(Hs[w] >> (24 - 8 * j));
}
