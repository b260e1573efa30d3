/*
 * Content-based chunking -- oracle, test infrastructure only.
 *
 * Sec. 2.1 ("Content-based chunking"): many overlapping windows of the data
 * are hashed and a block boundary is declared where the hash matches a
 * predefined value. Sec. 3.2.2: one small hash per window, windows overlap,
 * the window hash is MD5, and the buffer of window hashes is then checked for
 * boundaries. Sec. 4.3: chunking runs with a minimum and a maximum chunk size.
 *
 * Readings where the paper is silent (all parameters, not constants):
 *  - the window is `window` bytes (20 in the workloads), one window ends at
 *    every byte offset p >= window-1 (stride 1) over the whole stream;
 *  - "the hash value" compared is the first four MD5 digest bytes read as a
 *    little-endian 32-bit word; "matches a predefined value" means its low
 *    mask_bits bits equal magic;
 *  - a matching window ending at byte p puts a candidate cut at p + 1;
 *  - selection is greedy from the start of the stream: from chunk start s,
 *    cut at the first candidate c with s + min <= c <= s + max; with none,
 *    cut at s + max when s + max < n, else the chunk is the rest [s, n).
 *    Candidates closer than min to s are skipped; the last chunk may be
 *    shorter than min.
 */
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include "hg_oracle.h"

uint32_t hgo_window_hash(const uint8_t *win, uint32_t window) {
    uint8_t d[16];
    hgo_md5(win, window, d);
    return (uint32_t)d[0] | ((uint32_t)d[1] << 8) | ((uint32_t)d[2] << 16) | ((uint32_t)d[3] << 24);
}

static int is_candidate(const uint8_t *in, uint64_t p, int kind, uint32_t window,
                        uint32_t mask, uint32_t magic) {
    const uint8_t *w = in + p + 1 - window;
    uint32_t h = kind == HGO_WIN_RABIN ? hgo_rabin_fingerprint(w, window)
                                       : hgo_window_hash(w, window);
    return (h & mask) == magic;
}

typedef struct {
    const uint8_t *in;
    uint64_t p_lo, p_hi;          /* window end positions [p_lo, p_hi) */
    int kind;
    uint32_t window, mask, magic;
    uint64_t *cuts, count, cap;
} range_job;

static void *scan_range(void *arg) {
    range_job *j = (range_job *)arg;
    for (uint64_t p = j->p_lo; p < j->p_hi; p++) {
        if (is_candidate(j->in, p, j->kind, j->window, j->mask, j->magic)) {
            if (j->count == j->cap) {             /* grow the private list */
                uint64_t nc = j->cap ? 2 * j->cap : 1024;
                uint64_t *nb = (uint64_t *)realloc(j->cuts, nc * sizeof(uint64_t));
                if (!nb) return (void *)1;
                j->cuts = nb; j->cap = nc;
            }
            j->cuts[j->count++] = p + 1;
        }
    }
    return NULL;
}

uint64_t hgo_window_candidates(const uint8_t *in, uint64_t n, uint32_t window,
                               uint32_t mask_bits, uint32_t magic,
                               uint64_t *cuts, uint64_t cap, int nthreads) {
    return hgo_window_candidates_kind(in, n, HGO_WIN_MD5, window, mask_bits, magic, cuts, cap,
                                      nthreads);
}

uint64_t hgo_window_candidates_kind(const uint8_t *in, uint64_t n, int kind, uint32_t window,
                                    uint32_t mask_bits, uint32_t magic,
                                    uint64_t *cuts, uint64_t cap, int nthreads) {
    if (kind != HGO_WIN_MD5 && kind != HGO_WIN_RABIN) return UINT64_MAX;
    if (window == 0 || n < window) return 0;
    uint32_t mask = mask_bits >= 32 ? 0xffffffffu : ((1u << mask_bits) - 1u);
    uint64_t first = window - 1, npos = n - first;
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > npos) nthreads = (int)npos;
    range_job *jobs = (range_job *)calloc((size_t)nthreads, sizeof(range_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; t++) {
        jobs[t].in = in;
        jobs[t].p_lo = first + npos * (uint64_t)t / (uint64_t)nthreads;
        jobs[t].p_hi = first + npos * (uint64_t)(t + 1) / (uint64_t)nthreads;
        jobs[t].kind = kind;
        jobs[t].window = window; jobs[t].mask = mask; jobs[t].magic = magic;
    }
    if (nthreads == 1) scan_range(&jobs[0]);
    else {
        for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, scan_range, &jobs[t]);
        for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    }
    uint64_t total = 0;
    for (int t = 0; t < nthreads; t++) {            /* ranges are in order */
        for (uint64_t i = 0; i < jobs[t].count; i++, total++)
            if (total < cap) cuts[total] = jobs[t].cuts[i];
        free(jobs[t].cuts);
    }
    free(jobs); free(th);
    return total;
}

uint64_t hgo_select(const uint64_t *cands, uint64_t ncand, uint64_t n,
                    uint64_t min_chunk, uint64_t max_chunk,
                    uint64_t *ends, uint64_t cap) {
    uint64_t s = 0, k = 0, count = 0;
    while (s < n) {
        /* first candidate at or after s + min */
        while (k < ncand && cands[k] < s + min_chunk) k++;
        uint64_t cut;
        if (k < ncand && cands[k] <= s + max_chunk && cands[k] <= n) cut = cands[k];
        else if (s + max_chunk < n) cut = s + max_chunk;
        else cut = n;
        if (count < cap) ends[count] = cut;
        count++;
        s = cut;
    }
    return count;
}
