/*
 * HashGPU CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct C99 restatement of what the hashing hot
 * path computes, used by the test-suite, the smoke check and the CPU baseline
 * of the benchmark to check the CUDA library. It shares no code, header,
 * table or constant generator with the CUDA path, and the product never
 * links, loads or calls it.
 *
 * Every routine cites the passage of "GPUs as Storage System Accelerators"
 * (Al-Kiswany, Gharaibeh, Ripeanu) or of the hash standard it follows.
 * Pins (what each routine is checked against in the CPU test-suite):
 *   hgo_md5 / hgo_sha1        -> hashlib (OpenSSL) at every length 0..2048 and
 *                                on random MiB-sized inputs
 *   hgo_hash_blocks           -> hashlib per block and over the digest list
 *   hgo_hash_blocks_pmd       -> hashlib per segment and over each block's
 *                                segment digests; reduces to H(H(block)) when
 *                                segment == block
 *   hgo_window_hash/_candidates -> hashlib.md5 of every window (brute force)
 *   hgo_rabin_fingerprint     -> GF(2) facts: P irreducible (Ben-Or test),
 *                                low-degree strings are their own remainder,
 *                                x^31 leaves P - x^31, linearity in the bits,
 *                                x^(2^31 - 1) = 1 (P primitive, 2^31 - 1 prime),
 *                                and the one-byte shift identity
 *   hgo_select                -> hand-worked fixtures in tests/golden and a
 *                                checker of the properties that determine the
 *                                greedy chunking uniquely
 *   hgo_hash_chunks           -> hashlib per chunk
 * Nothing here is "parity unpinned".
 */
#ifndef HG_ORACLE_H
#define HG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { HGO_MD5 = 0, HGO_SHA1 = 1 };
/* window hash kinds: the paper's MD5 window, or a Rabin fingerprint window */
enum { HGO_WIN_MD5 = 0, HGO_WIN_RABIN = 1 };
/* the degree-31 irreducible polynomial of the Rabin window (bit k = x^k) */
#define HGO_RABIN_POLY 0x9E3779BBu

/* RFC 1321: MD5 of len bytes; 16-byte digest in the standard byte order. */
void hgo_md5(const uint8_t *msg, uint64_t len, uint8_t out[16]);
/* FIPS 180-4 Sec. 6.1: SHA-1 of len bytes; 20-byte big-endian digest. */
void hgo_sha1(const uint8_t *msg, uint64_t len, uint8_t out[20]);
/* Digest length of algo (16 or 20), 0 for an unknown algo. */
int hgo_digest_len(int algo);
/* Digest of len bytes with algo; returns 0, or -1 for an unknown algo. */
int hgo_digest(int algo, const uint8_t *msg, uint64_t len, uint8_t *out);

/*
 * Direct hashing (Sec. 2.1 "Direct Hashing", Sec. 3.2.2): digest of every
 * fixed-size block [i*block, min((i+1)*block, n)), then, when root is not
 * NULL, the hash-of-hashes over the block digests concatenated in block order.
 * Returns the number of blocks, or -1 on bad arguments.
 */
int64_t hgo_hash_blocks(int algo, const uint8_t *in, uint64_t n, uint64_t block,
                        uint8_t *digests, uint8_t *root);

/*
 * Two-level block identifiers (Sec. 3.2.2 "Direct Hashing", the parallel
 * Merkle-Damgard construction): block i = [i*block, min((i+1)*block, n)) is
 * cut into segments of `segment` bytes (the last one may be short), each
 * segment is digested, and ids[i] = digest of the block's segment digests in
 * order. block must be a multiple of segment. Returns the number of blocks,
 * or -1 on bad arguments.
 */
int64_t hgo_hash_blocks_pmd(int algo, const uint8_t *in, uint64_t n, uint64_t block,
                            uint64_t segment, uint8_t *ids);

/*
 * Sliding-window hash (Sec. 2.1 "Content-based chunking", Sec. 3.2.2): the
 * first four MD5 digest bytes, read little-endian, of the `window` bytes at win.
 */
uint32_t hgo_window_hash(const uint8_t *win, uint32_t window);

/*
 * Rabin fingerprint (variant window hash, LBFS-style; see rabin.c): the
 * remainder modulo HGO_RABIN_POLY of the polynomial of the len bytes at msg,
 * read as one big-endian binary number. A 31-bit value.
 */
uint32_t hgo_rabin_fingerprint(const uint8_t *msg, uint64_t len);

/*
 * As hgo_window_candidates, with the window hash chosen by kind: HGO_WIN_MD5
 * (hgo_window_hash) or HGO_WIN_RABIN (hgo_rabin_fingerprint of the window).
 * Returns the total count, or UINT64_MAX for an unknown kind.
 */
uint64_t hgo_window_candidates_kind(const uint8_t *in, uint64_t n, int kind, uint32_t window,
                                    uint32_t mask_bits, uint32_t magic,
                                    uint64_t *cuts, uint64_t cap, int nthreads);

/*
 * Boundary candidates: every cut position c = p + 1, p in [window-1, n-1],
 * whose window hash h (of bytes p-window+1..p) satisfies
 * (h & (2^mask_bits - 1)) == magic. Written in increasing order, at most cap
 * of them; returns the total count. nthreads > 1 splits the positions into
 * that many contiguous ranges handled by POSIX threads.
 */
uint64_t hgo_window_candidates(const uint8_t *in, uint64_t n, uint32_t window,
                               uint32_t mask_bits, uint32_t magic,
                               uint64_t *cuts, uint64_t cap, int nthreads);

/*
 * Chunk boundary selection with minimum and maximum chunk sizes (Sec. 2.1,
 * Sec. 4.3 workload set-up): chunk ends, strictly increasing, the last one n.
 * At most cap written; returns the total count.
 */
uint64_t hgo_select(const uint64_t *cands, uint64_t ncand, uint64_t n,
                    uint64_t min_chunk, uint64_t max_chunk,
                    uint64_t *ends, uint64_t cap);

/* Per-chunk digests (Fig. 3): chunk i is [ends[i-1] (0 for i = 0), ends[i]). */
int hgo_hash_chunks(int algo, const uint8_t *in, const uint64_t *ends,
                    uint64_t nchunk, uint8_t *digests);

#ifdef __cplusplus
}
#endif
#endif
