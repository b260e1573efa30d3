/*
 * Direct hashing and per-chunk hashing -- oracle, test infrastructure only.
 *
 * Sec. 2.1 ("Direct Hashing"): a block's identifier is the hash of its bytes.
 * Sec. 3.2.2 ("Direct Hashing", and the stage description that follows it):
 * the data is split into fixed-size segments, each segment is hashed with the
 * standard sequential hash, the segment digests are placed in one output
 * buffer, and that buffer is hashed once more to give the final value.
 * Fig. 3: after boundaries are known, each content-defined chunk is hashed
 * with the direct-hashing kernel.
 *
 * Readings where the paper is silent: the final (hash-of-hashes) step uses the
 * same digest as the segments; it is one level, not a tree; a short last
 * segment is hashed as it is, without padding to the segment size; zero
 * segments give the digest of the empty string.
 */
#include <stdlib.h>
#include "hg_oracle.h"

int hgo_digest_len(int algo) {
    return algo == HGO_MD5 ? 16 : algo == HGO_SHA1 ? 20 : 0;
}

int hgo_digest(int algo, const uint8_t *msg, uint64_t len, uint8_t *out) {
    if (algo == HGO_MD5) { hgo_md5(msg, len, out); return 0; }
    if (algo == HGO_SHA1) { hgo_sha1(msg, len, out); return 0; }
    return -1;
}

int64_t hgo_hash_blocks(int algo, const uint8_t *in, uint64_t n, uint64_t block,
                        uint8_t *digests, uint8_t *root) {
    int dl = hgo_digest_len(algo);
    if (dl == 0 || block == 0) return -1;
    uint64_t nblk = (n + block - 1) / block;
    for (uint64_t i = 0; i < nblk; i++) {
        uint64_t lo = i * block;
        uint64_t hi = lo + block < n ? lo + block : n;
        hgo_digest(algo, in + lo, hi - lo, digests + i * (uint64_t)dl);
    }
    if (root) hgo_digest(algo, digests, nblk * (uint64_t)dl, root);
    return (int64_t)nblk;
}

/*
 * Two-level (parallel Merkle-Damgard) block identifiers, Sec. 3.2.2 "Direct
 * Hashing": inside each block the segments are hashed independently and the
 * block's identifier is the hash of its segment digests in order. Written out
 * block by block, segment by segment, as the definition reads.
 */
int64_t hgo_hash_blocks_pmd(int algo, const uint8_t *in, uint64_t n, uint64_t block,
                            uint64_t segment, uint8_t *ids) {
    int dl = hgo_digest_len(algo);
    if (dl == 0 || block == 0 || segment == 0 || block % segment != 0) return -1;
    uint64_t nblk = (n + block - 1) / block;
    uint8_t *buf = malloc((block / segment) * (uint64_t)dl + 1);
    if (!buf) return -1;
    for (uint64_t i = 0; i < nblk; i++) {
        uint64_t lo = i * block;
        uint64_t blk_end = lo + block < n ? lo + block : n;
        uint64_t nseg = 0;
        for (uint64_t a = lo; a < blk_end; a += segment) {
            uint64_t b = a + segment < blk_end ? a + segment : blk_end;
            hgo_digest(algo, in + a, b - a, buf + nseg * (uint64_t)dl);
            nseg++;
        }
        hgo_digest(algo, buf, nseg * (uint64_t)dl, ids + i * (uint64_t)dl);
    }
    free(buf);
    return (int64_t)nblk;
}

int hgo_hash_chunks(int algo, const uint8_t *in, const uint64_t *ends,
                    uint64_t nchunk, uint8_t *digests) {
    int dl = hgo_digest_len(algo);
    if (dl == 0) return -1;
    uint64_t start = 0;
    for (uint64_t i = 0; i < nchunk; i++) {
        if (ends[i] < start) return -1;
        hgo_digest(algo, in + start, ends[i] - start, digests + i * (uint64_t)dl);
        start = ends[i];
    }
    return 0;
}
