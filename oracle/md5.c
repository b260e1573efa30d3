/*
 * MD5 as RFC 1321 defines it -- oracle, test infrastructure only.
 *
 * The paper hashes every segment and every sliding window with MD5 ("MD5 in
 * all our experiments", Sec. 3.2.2). This file writes the RFC out step by
 * step: padding (RFC 1321 Sec. 3.1-3.2), the four buffer words (Sec. 3.3),
 * the sixty-four operations on each 16-word block (Sec. 3.4) and the output
 * order (Sec. 3.5). The sine table T[i] is computed from its definition,
 * floor(2^32 * |sin(i)|) for i = 1..64, rather than typed in.
 */
#include <math.h>
#include <pthread.h>
#include <string.h>
#include "hg_oracle.h"

static uint32_t T[65];
static pthread_once_t t_once = PTHREAD_ONCE_INIT;

static void make_sine_table(void) {
    /* RFC 1321 Sec. 3.4: T[i] = integer part of 4294967296 * abs(sin(i)),
     * i in radians. Done once; the doubles are exact enough that the floor
     * lands on the right integer for all 64 entries (checked by the pins). */
    for (int i = 1; i <= 64; i++)
        T[i] = (uint32_t)floor(4294967296.0 * fabs(sin((double)i)));
}

static uint32_t rotl(uint32_t x, int s) { return (x << s) | (x >> (32 - s)); }

/* The four auxiliary functions of RFC 1321 Sec. 3.4. */
static uint32_t F(uint32_t x, uint32_t y, uint32_t z) { return (x & y) | (~x & z); }
static uint32_t G(uint32_t x, uint32_t y, uint32_t z) { return (x & z) | (y & ~z); }
static uint32_t H(uint32_t x, uint32_t y, uint32_t z) { return x ^ y ^ z; }
static uint32_t I(uint32_t x, uint32_t y, uint32_t z) { return y ^ (x | ~z); }

/* Shift amounts of each round, in the order the RFC lists the operations. */
static const int S[4][4] = {{7, 12, 17, 22}, {5, 9, 14, 20}, {4, 11, 16, 23}, {6, 10, 15, 21}};

static void md5_block(uint32_t st[4], const uint8_t blk[64]) {
    uint32_t X[16];
    for (int j = 0; j < 16; j++)                         /* little-endian words */
        X[j] = (uint32_t)blk[4 * j] | ((uint32_t)blk[4 * j + 1] << 8) |
               ((uint32_t)blk[4 * j + 2] << 16) | ((uint32_t)blk[4 * j + 3] << 24);
    uint32_t a = st[0], b = st[1], c = st[2], d = st[3];
    for (int i = 0; i < 64; i++) {
        int round = i / 16, k;
        uint32_t f;
        switch (round) {                                  /* word index per round */
        case 0: f = F(b, c, d); k = i;                 break;
        case 1: f = G(b, c, d); k = (5 * i + 1) % 16;  break;
        case 2: f = H(b, c, d); k = (3 * i + 5) % 16;  break;
        default: f = I(b, c, d); k = (7 * i) % 16;     break;
        }
        /* [abcd k s i]: a = b + ((a + Fn(b,c,d) + X[k] + T[i]) <<< s), then the
         * next operation names the buffer words shifted by one (d a b c). */
        uint32_t t = a + f + X[k] + T[i + 1];
        uint32_t na = b + rotl(t, S[round][i % 4]);
        a = d; d = c; c = b; b = na;
    }
    st[0] += a; st[1] += b; st[2] += c; st[3] += d;     /* Sec. 3.4 end of block */
}

void hgo_md5(const uint8_t *msg, uint64_t len, uint8_t out[16]) {
    pthread_once(&t_once, make_sine_table);
    /* Sec. 3.3: word A = 01 23 45 67, B = 89 ab cd ef, C = fe dc ba 98,
     * D = 76 54 32 10 (low-order byte first). */
    uint32_t st[4] = {0x67452301u, 0xefcdab89u, 0x98badcfeu, 0x10325476u};
    uint64_t full = len / 64;
    for (uint64_t i = 0; i < full; i++) md5_block(st, msg + 64 * i);
    /* Sec. 3.1-3.2: one 1 bit, zeros to 56 mod 64, then the bit length as a
     * 64-bit little-endian number. */
    uint8_t tail[128];
    uint64_t rem = len - 64 * full;
    memset(tail, 0, sizeof tail);
    memcpy(tail, msg + 64 * full, (size_t)rem);
    tail[rem] = 0x80;
    uint64_t tlen = (rem < 56) ? 64 : 128;
    uint64_t bits = len * 8u;
    for (int j = 0; j < 8; j++) tail[tlen - 8 + j] = (uint8_t)(bits >> (8 * j));
    for (uint64_t off = 0; off < tlen; off += 64) md5_block(st, tail + off);
    for (int w = 0; w < 4; w++)                           /* Sec. 3.5 output */
        for (int j = 0; j < 4; j++) out[4 * w + j] = (uint8_t)(st[w] >> (8 * j));
}
