/*
 * Rabin fingerprint window hash -- oracle, test infrastructure only.
 *
 * A variant of the sliding-window hash, not the paper's: Sec. 2.1 names LBFS
 * as a content-based chunking system, and LBFS hashes its windows with Rabin
 * fingerprints instead of a cryptographic digest. The fingerprint of a byte
 * string is the remainder of its polynomial over GF(2) modulo a fixed
 * irreducible polynomial P of degree 31 (Rabin, "Fingerprinting by random
 * polynomials", 1981).
 *
 * Conventions (readings; the paper defines none of this):
 *  - the string b_0 .. b_{L-1} is the polynomial whose coefficients are its
 *    bits read most significant first: b_0's bit 7 is the highest term and
 *    b_{L-1}'s bit 0 is the constant term, i.e. the string read as one
 *    big-endian binary number;
 *  - the remainder is returned as a 31-bit integer, bit k = coefficient of x^k;
 *  - P = x^31 + (0x1E3779BB), written HGO_RABIN_POLY with the x^31 bit set:
 *    the first odd value at or above floor(2^31 (sqrt(5) - 2)) for which the
 *    polynomial is irreducible (checked in the CPU tests).
 * The remainder is computed here by long division, one message bit at a time,
 * straight from the definition; no tables and no rolling update.
 */
#include "hg_oracle.h"

uint32_t hgo_rabin_fingerprint(const uint8_t *msg, uint64_t len) {
    uint32_t r = 0;                         /* remainder, degree < 31 */
    for (uint64_t i = 0; i < len; i++) {
        for (int j = 7; j >= 0; j--) {
            r = (r << 1) | ((msg[i] >> j) & 1u);      /* r * x + next bit */
            if (r & 0x80000000u) r ^= HGO_RABIN_POLY; /* degree 31: subtract P */
        }
    }
    return r;
}
