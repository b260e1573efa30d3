/*
 * hashgpu.h -- C ABI of the B300 HashGPU hashing library (libhashgpu.so).
 *
 * The library offloads the two hashing primitives of "GPUs as Storage System
 * Accelerators" (Al-Kiswany, Gharaibeh, Ripeanu), Sec. 2.1 and Sec. 3.2.2:
 *   - direct hashing: the digest of every fixed-size block of a buffer, plus
 *     the hash-of-hashes over the block digests;
 *   - content-based chunking: a hash of a small window at every byte offset,
 *     chunk boundaries where the window hash matches a predefined value under
 *     minimum and maximum chunk sizes, then the digest of every chunk.
 * As the paper asks of an offloaded primitive (Sec. 3.1, "Minimizing the
 * integration effort"), the calls keep the shape of a CPU hash call: bytes
 * in, digests out, plus a library allocator for pinned host buffers
 * (Sec. 3.2.4 "Fixed-Size Blocks Hashing Integration") and asynchronous job
 * submission with completion polling (Sec. 3.2.3).
 *
 * Conventions for every call:
 *  - Pointers named d_* are device pointers on the context's device; h_*
 *    are host pointers. The caller owns all of them. The context owns only
 *    its internal scratch memory, which counts against its device budget.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls
 *    enqueue work on it and return once it is enqueued; results are valid
 *    after the stream is synchronised. Calls on one context must not be made
 *    from two host threads at once, and work on two streams of one context
 *    must not overlap unless each stream has its own context.
 *  - Every call returns HG_OK (0) or a negative hg_status. Argument errors are
 *    detected on the host before anything is enqueued. Errors found on the
 *    device (a bounded wait that ran out, an inconsistent offsets array) are
 *    recorded in the context's device error word and returned by the next
 *    hg_sync() on that context.
 *  - Digests are written in the standard byte order of each algorithm (the
 *    bytes of hashlib's digest()): 16 bytes for MD5, 20 for SHA-1. Digest
 *    buffers must be 4-byte aligned.
 */
#ifndef HASHGPU_H
#define HASHGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HG_OK = 0,
    HG_EINVAL = -1,       /* bad argument (null pointer, size, alignment, algo) */
    HG_ENOMEM = -2,       /* device budget or an allocation exhausted */
    HG_ECAPACITY = -3,    /* an output array was too small (count still reported) */
    HG_ETIMEDOUT = -4,    /* a bounded device-side wait gave up */
    HG_ECUDA = -5,        /* a CUDA runtime call failed */
    HG_EAGAIN = -6,       /* asynchronous result not ready yet */
    HG_ECANCELED = -7,    /* request cancelled before it ran */
    HG_EUNSUPPORTED = -8, /* parameters outside what this build supports */
    HG_EBOUNDS = -9       /* debug build only: a kernel's bounds check failed */
} hg_status;

typedef enum { HG_MD5 = 0, HG_SHA1 = 1 } hg_algo;

typedef struct hg_ctx hg_ctx;

/*
 * Window hash of content-defined chunking. HG_WIN_MD5 is the paper's (Sec.
 * 3.2.2: MD5 of each window). HG_WIN_RABIN is a variant with no counterpart
 * in the paper's experiments: the Rabin fingerprint used by LBFS, the
 * chunking system Sec. 2.1 cites -- the window's bytes (first byte most
 * significant, bit 7 high) as a polynomial over GF(2), modulo the irreducible
 * degree-31 polynomial HG_RABIN_POLY (bit k = coefficient of x^k); the 31-bit
 * remainder is the window hash. It rolls, so it costs a few operations per
 * byte instead of one MD5 compression per byte.
 */
typedef enum { HG_WIN_MD5 = 0, HG_WIN_RABIN = 1 } hg_window_hash;
#define HG_RABIN_POLY 0x9E3779BBu

/*
 * Content-defined chunking parameters (Sec. 2.1 "Content-based chunking";
 * min/max chunk sizes as in the Sec. 4.3 set-up). A window of `window` bytes
 * ends at every offset p >= window-1; its hash h is, for HG_WIN_MD5, the first
 * four MD5 digest bytes read little-endian, for HG_WIN_RABIN the fingerprint
 * above; when (h & (2^mask_bits - 1)) == magic the position p + 1 is a
 * candidate cut. Cuts are chosen greedily from offset 0: from chunk start s,
 * the first candidate c with s + min_chunk <= c <= s + max_chunk; with none,
 * s + max_chunk if that is < n, else n.
 * Supported: 1 <= window <= 55 (MD5) or 64 (Rabin), 1 <= mask_bits <= 32,
 * magic < 2^mask_bits, 1 <= min_chunk <= max_chunk. Every chunking call,
 * the batch and server calls included, accepts both window hashes.
 */
typedef struct {
    uint32_t window;      /* bytes per window (20) */
    uint32_t mask_bits;   /* low bits of the window hash compared (13) */
    uint32_t magic;       /* value they must equal (0x0F0F) */
    uint32_t window_hash; /* hg_window_hash (HG_WIN_MD5) */
    uint64_t min_chunk;   /* 2048 */
    uint64_t max_chunk;   /* 65536 */
} hg_cdc_params;

/* Fill p with the defaults used throughout (20, 13, 0x0F0F, 2 KiB, 64 KiB). */
void hg_cdc_default_params(hg_cdc_params *p);

/* Human-readable name of a status code (static string). */
const char *hg_strerror(int status);

/* Digest length in bytes of algo (16, 20), or HG_EINVAL. */
int hg_digest_len(int algo);

/*
 * The library's host-side digest (MD5 or SHA-1 of n bytes at msg into out,
 * standard byte order), synchronous, on the calling thread; no device is
 * needed. hg_hash_blocks computes the hash-of-hashes with it on a host core,
 * as the paper does (Sec. 3.2.2: the CPU computes the final hash over the
 * intermediate digests). HG_EINVAL for a bad algo or null pointers.
 */
int hg_host_digest(int algo, const uint8_t *msg, uint64_t n, uint8_t *out);

/*
 * Create a context on CUDA device `device`. `device_budget_bytes` caps the
 * scratch memory the context may hold (0 = 32 GiB). Scratch is allocated on
 * first use and grown as needed. Growing it synchronises the whole device
 * (queued work may still use the old scratch: cudaDeviceSynchronize, then
 * cudaFree and cudaMalloc), so a call that grows scratch is not asynchronous;
 * hg_reserve() allocates the scratch for inputs up to a given size ahead of
 * time, after which calls on such inputs never synchronise.
 */
int hg_init(hg_ctx **out, int device, size_t device_budget_bytes);
/* Free the context and all its scratch (synchronises its device first).
 * Destroy the objects made on a context (servers, batches, streams, block
 * maps) before the context, and all of them before the process exits and the
 * CUDA runtime is torn down; the Python binding does this in an exit handler. */
int hg_destroy(hg_ctx *ctx);
/* Pre-allocate scratch for chunking inputs of up to max_bytes bytes (may
 * synchronise the device once, see hg_init). HG_ENOMEM over the budget. */
int hg_reserve(hg_ctx *ctx, uint64_t max_bytes);
/* Synchronise `stream` and return (then clear) the device error word. */
int hg_sync(hg_ctx *ctx, void *stream);
/* Bytes of scratch currently held by the context. */
uint64_t hg_scratch_bytes(const hg_ctx *ctx);

/*
 * Pinned host buffers from a pool owned by the context: the library allocator
 * the paper asks for. Data the application writes into page-locked host
 * memory crosses the host link in one DMA copy (Sec. 3.1, "One-copy host to
 * device data transfers"), and page-locked buffers are too costly to allocate
 * per request, so they are allocated once and reused (Sec. 3.1, "Hiding memory
 * allocation overheads"; Sec. 3.2.3, the runtime's memory-management module;
 * Sec. 3.2.4, buffers obtained through the library call).
 *
 * hg_alloc_pinned: a page-locked host buffer of at least `bytes` bytes,
 *   mapped for device access (usable as h_in of hg_cdc_hash_h2d and as
 *   hg_request.h_data, whose small inputs the server then gathers with one
 *   kernel). Sizes are rounded up to a class (64 KiB, else the next of
 *   2^k x {1, 1.25, 1.5, 1.75}, hg_pinned_class); a free buffer of the class
 *   (or a larger one up to twice it) is reused without a new host allocation.
 *   A new allocation counts against the pool's host budget (16 GiB unless set),
 *   releasing free buffers, largest first, if needed. Returns NULL when ctx is
 *   NULL, bytes is 0, the budget cannot hold the buffer, or the host
 *   allocation fails. Thread-safe.
 * hg_free_pinned: gives p back to the pool (it stays allocated, for reuse).
 *   p must come from hg_alloc_pinned on the same context and no enqueued work
 *   may still read or write it (synchronise first). HG_EINVAL for a pointer
 *   the pool does not own or that is already free.
 * hg_pinned_set_budget: host bytes the pool may hold (0 = 16 GiB); free
 *   buffers above a lowered budget are released at once, busy ones as they
 *   are freed.
 * hg_pinned_trim: releases every free buffer.
 * hg_pinned_stats: bytes held / handed out, host allocations made, requests
 *   served by reuse, and buffers owned.
 * All buffers, free or not, are released by hg_destroy.
 */
typedef struct {
    uint64_t budget_bytes, held_bytes, in_use_bytes;
    uint64_t host_allocs, reuses, buffers;
} hg_pinned_info;
void *hg_alloc_pinned(hg_ctx *ctx, size_t bytes);
int hg_free_pinned(hg_ctx *ctx, void *p);
int hg_pinned_set_budget(hg_ctx *ctx, uint64_t bytes);
int hg_pinned_trim(hg_ctx *ctx);
int hg_pinned_stats(hg_ctx *ctx, hg_pinned_info *out);
uint64_t hg_pinned_class(uint64_t bytes);

/*
 * Direct hashing, Sec. 2.1 "Direct Hashing" and Sec. 3.2.2: the digest of
 * every block [i*block, min((i+1)*block, n)) of d_in (the last block may be
 * short), written to d_digests[i*dlen .. (i+1)*dlen), nblk = ceil(n/block).
 * If d_root is not NULL it receives the hash-of-hashes: the digest, with the
 * same algorithm, of the nblk*dlen digest bytes in block order (Sec. 3.2.2,
 * the final step that hashes the buffer of intermediate digests). n = 0 gives
 * no blocks and the digest of the empty string as root. That final step is
 * one serial chain; as in the paper it runs on a host core: the digests are
 * copied to a pinned staging buffer of the context, hashed by a host function
 * enqueued on `stream`, and the root is copied back, all in stream order
 * (the staging buffer grows on demand, which synchronises the device once).
 * Shorter digest lists (MD5: under 1 MiB; SHA-1: under 16 KiB when the host
 * CPU has the SHA extensions, else under 256 KiB; the environment variable
 * HG_HOST_ROOT_MIN, in bytes, overrides both), and calls made while `stream`
 * is being captured into a CUDA graph, use a single-thread device kernel.
 * d_in: n bytes, any alignment. d_digests: nblk*dlen bytes, 4-byte aligned.
 * d_root: dlen bytes or NULL. Errors: HG_EINVAL (block == 0, bad algo,
 * null or misaligned buffer).
 */
int hg_hash_blocks(hg_ctx *ctx, int algo, const uint8_t *d_in, uint64_t n, uint64_t block,
                   uint8_t *d_digests, uint8_t *d_root, void *stream);

/*
 * Two-level block identifiers, the parallel Merkle-Damgard construction of
 * Sec. 3.2.2 "Direct Hashing": block i = [i*block, min((i+1)*block, n)) is cut
 * into segments of `segment` bytes (the last may be short), every segment is
 * digested independently, and d_ids[i] = H(segment digests of block i, in
 * order) with the same algo. This is a different identifier from the plain
 * digest of the block (hg_hash_blocks): it removes the block-long serial chain.
 * block must be a multiple of segment (HG_EINVAL otherwise).
 * d_seg_digests: ceil(n/segment)*dlen bytes, 16-byte aligned, receives the
 * segment digests; NULL keeps them in context scratch (counted against the
 * budget, HG_ENOMEM if it does not fit). d_ids: ceil(n/block)*dlen bytes,
 * 4-byte aligned. n = 0 writes nothing.
 */
int hg_hash_blocks_pmd(hg_ctx *ctx, int algo, const uint8_t *d_in, uint64_t n, uint64_t block,
                       uint64_t segment, uint8_t *d_seg_digests, uint8_t *d_ids, void *stream);

/*
 * Sliding-window hashing, Sec. 3.2.2 "Content-based chunking": bit p of the
 * bitmap (word p/32, bit p%32) is set when the window ending at byte p is a
 * candidate (see hg_cdc_params); bits for p < window-1 and p >= n are 0.
 * d_bitmap: ceil(n/32) uint32 words.
 */
int hg_window_bitmap(hg_ctx *ctx, const uint8_t *d_in, uint64_t n, const hg_cdc_params *params,
                     uint32_t *d_bitmap, void *stream);

/*
 * Candidate cut positions (the window-hash test of Sec. 2.1 followed by the
 * boundary check the paper leaves to the CPU in Sec. 3.2.2, done here on the
 * device): all c = p + 1 with window p a candidate, increasing. At most cap
 * are written to d_cands; the total count goes to *d_count (device uint64).
 */
int hg_cdc_candidates(hg_ctx *ctx, const uint8_t *d_in, uint64_t n, const hg_cdc_params *params,
                      uint64_t *d_cands, uint64_t cap, uint64_t *d_count, void *stream);

/*
 * Chunk boundaries, Sec. 2.1 with the min/max rule of hg_cdc_params: chunk
 * end offsets, strictly increasing, the last equal to n (none when n = 0).
 * At most cap are written to d_ends; the total count goes to *d_count
 * (device uint64). A count above cap means d_ends was too small. With cap >=
 * n/min_chunk + 1 it never is.
 */
int hg_cdc_boundaries(hg_ctx *ctx, const uint8_t *d_in, uint64_t n, const hg_cdc_params *params,
                      uint64_t *d_ends, uint64_t cap, uint64_t *d_count, void *stream);

/*
 * Per-chunk digests, Fig. 3 (the second job, direct hashing of each chunk):
 * chunk i is [d_ends[i-1] (0 for i = 0), d_ends[i]) of the n-byte input d_in.
 * nchunk is the host-side number of entries; when d_count is not NULL the
 * number actually hashed is min(nchunk, *d_count) (as written by
 * hg_cdc_boundaries), so the two calls chain on one stream without a host
 * round trip. d_digests: nchunk*dlen bytes, 4-byte aligned. An end that is
 * below the previous one or above n records HG_EINVAL in the device error
 * word and leaves that digest unwritten.
 */
int hg_hash_chunks(hg_ctx *ctx, int algo, const uint8_t *d_in, uint64_t n, const uint64_t *d_ends,
                   uint64_t nchunk, const uint64_t *d_count, uint8_t *d_digests, void *stream);

/*
 * Chunk boundaries and per-chunk digests of one buffer in one call: the same
 * results as hg_cdc_boundaries followed by hg_hash_chunks (Fig. 3: sliding-
 * window hashing, boundary detection, then direct hashing of each chunk). The
 * launches are captured once into a CUDA graph (per context, replayed while
 * the arguments stay the same). Buffers above 64 MiB are window-hashed and
 * their boundaries selected in segments of at least 32 MiB (hg_cdc_hash_plan
 * gives the bounds), each segment's selection overlapping the next segment's
 * window hashing; the chunk digests of such buffers run in one launch after
 * the last selection, longest chunks first. Up to 64 MiB the buffer is one
 * segment and its digests follow its selection. Runs on context-owned
 * streams forked from and joined back into `stream`. d_ends needs cap >= n / min_chunk + 1 entries (HG_ECAPACITY
 * otherwise, before anything is enqueued); d_digests cap * dlen bytes;
 * *d_count (device) gets the count.
 */
int hg_cdc_hash(hg_ctx *ctx, int algo, const uint8_t *d_in, uint64_t n, const hg_cdc_params *params,
                uint64_t *d_ends, uint64_t cap, uint64_t *d_count, uint8_t *d_digests,
                void *stream);
/*
 * hg_cdc_hash on input that is still in host memory: the call itself copies
 * h_in (n bytes, pinned for an asynchronous copy, Sec. 3.1 "One-copy host to
 * device data transfers") into the device buffer d_in in pieces of 8 MiB and
 * up, on a context copy stream, and each piece's window hashing starts as
 * soon as it has landed, so the copy overlaps the hashing (Sec. 3.2.3,
 * overlapping the transfer of one block with the computation on another).
 * The copies of all contexts on a device share one copy stream, so calls made
 * on several streams transfer one after the other rather than interleaved.
 * d_in keeps the bytes afterwards. Other arguments as hg_cdc_hash (launched
 * directly rather than from a graph).
 */
int hg_cdc_hash_h2d(hg_ctx *ctx, int algo, const uint8_t *h_in, uint8_t *d_in, uint64_t n,
                    const hg_cdc_params *params, uint64_t *d_ends, uint64_t cap,
                    uint64_t *d_count, uint8_t *d_digests, void *stream);
/* The segment schedule hg_cdc_hash uses for n bytes: returns the number of
 * segments S (0 for n = 0) and writes up to max of the S + 1 bounds (0 ...
 * n) when bounds is not NULL. Each segment enqueues five kernels. */
uint32_t hg_cdc_hash_plan(uint64_t n, uint64_t *bounds, uint32_t max);

/*
 * Streaming chunking (Sec. 3.2.4, "Content-based Chunking Integration"): a
 * stream written in buffers of any size is chunked buffer by buffer; when a
 * chunk boundary does not line up with the end of a buffer, the leftover
 * bytes (the still-open chunk) are carried into the next buffer. The stream
 * keeps that chunk plus the window - 1 bytes before it in its own device
 * working buffers, so the caller's buffer may be reused once the call's work
 * has run. Each feed writes the chunks the data seen so far decides: their
 * ends as offsets in the whole stream, their digests, and their number in
 * *d_count (device); close writes the rest. Over the whole stream the results
 * equal hg_cdc_hash on the concatenated bytes.
 * max_feed_bytes bounds len per feed (HG_ECAPACITY above it); cap (entries
 * of d_ends, rows of d_digests) must be >= (max_feed_bytes + max_chunk +
 * window) / min_chunk + 2, or >= (carried + len) / min_chunk + 1 for that
 * feed. A feed waits on the host for the previous feed's work to finish (to
 * learn how many bytes it carried), then enqueues its own on `stream`.
 */
typedef struct hg_cdc_stream hg_cdc_stream;
int hg_stream_open(hg_ctx *ctx, int algo, const hg_cdc_params *params, uint64_t max_feed_bytes,
                   hg_cdc_stream **out);
int hg_stream_feed(hg_cdc_stream *st, const uint8_t *d_data, uint64_t len, uint64_t *d_ends,
                   uint64_t cap, uint64_t *d_count, uint8_t *d_digests, void *stream);
int hg_stream_close(hg_cdc_stream *st, uint64_t *d_ends, uint64_t cap, uint64_t *d_count,
                    uint8_t *d_digests, void *stream);
int hg_stream_destroy(hg_cdc_stream *st);

/*
 * Batched chunking and chunk digests for many files in one pass (Sec. 3.2.3:
 * the runtime batches a stream of hashing jobs; Sec. 4.1: the gains need
 * batches; Sec. 3.2.4: writes are buffered so one GPU job covers many chunks).
 * The nfile files are stored back to back in one device buffer: file f is
 * bytes [h_file_off[f], h_file_off[f+1]) with h_file_off[0] = 0 and the
 * offsets non-decreasing (empty files allowed). Every file is chunked on its
 * own exactly as hg_cdc_boundaries would (no window crosses a file start) and
 * every chunk is digested as hg_hash_chunks would.
 *
 * Output layout ("slots"): file f owns slots [slot_off[f], slot_off[f+1]),
 * slot_off[f+1] - slot_off[f] = size_f / min_chunk + 1 (0 for an empty file),
 * which is at least the number of chunks the rule can make. Chunk i of file f
 * ends at d_ends[slot_off[f] + i] (offset relative to the file's start) and
 * its digest is d_digests[(slot_off[f] + i) * dlen ...]; d_counts[f] receives
 * the file's chunk count. hg_batch_slots() returns the total number of slots
 * and, when h_slot_off is not NULL, writes the nfile + 1 slot offsets there.
 *
 * hg_batch_create copies the offsets, classifies files for the selection step
 * and allocates all scratch once (counted against the context's budget);
 * hg_batch_cdc_hash only enqueues memsets and kernels (no allocation, no host
 * synchronisation); hg_batch_cdc_hash_graph does the same through a CUDA graph
 * captured on the first call and replayed while the pointers, algorithm and
 * tuning stay the same. hg_batch_sync synchronises the stream and returns the
 * batch's device error word. A plan may be used by one stream at a time.
 */
typedef struct hg_batch hg_batch;
typedef struct {
    int32_t window_ctas_per_sm;   /* persistent window kernel CTAs per SM; 0 = one-warp CTAs
                                     over the tiles' 1024-window spans (MD5 window) */
    int32_t hash_threads;         /* chunk-hash kernel threads per CTA (32..512, power of 2) */
    int32_t hash_ctas_per_sm;     /* chunk-hash kernel CTAs per SM */
    int32_t reserved;
    uint64_t long_chunk_bytes;    /* chunks at least this long are hashed first */
} hg_batch_tuning;

int hg_batch_create(hg_ctx *ctx, const uint64_t *h_file_off, uint32_t nfile,
                    const hg_cdc_params *params, hg_batch **out);
int hg_batch_destroy(hg_batch *batch);
uint64_t hg_batch_slots(const hg_batch *batch, uint64_t *h_slot_off);
int hg_batch_cdc_hash(hg_batch *batch, int algo, const uint8_t *d_data, uint64_t *d_ends,
                      uint64_t *d_counts, uint8_t *d_digests, void *stream);
int hg_batch_cdc_hash_graph(hg_batch *batch, int algo, const uint8_t *d_data, uint64_t *d_ends,
                            uint64_t *d_counts, uint8_t *d_digests, void *stream);
int hg_batch_sync(hg_batch *batch, void *stream);
int hg_batch_get_tuning(const hg_batch *batch, hg_batch_tuning *tuning);
int hg_batch_set_tuning(hg_batch *batch, const hg_batch_tuning *tuning);
/* Time a small set of tunings on this batch (synchronous: runs the batch about
 * 100 times; each candidate keeps the fastest of three timed runs, the window
 * forms are timed twice) and keep the fastest; it is also written to *best if
 * not NULL. */
int hg_batch_autotune(hg_batch *batch, int algo, const uint8_t *d_data, uint64_t *d_ends,
                      uint64_t *d_counts, uint8_t *d_digests, void *stream, hg_batch_tuning *best);
/* hg_batch_autotune through a cache file (JSON Lines, one
 * {"key": {...}, "tuning": {...}} object per line) keyed by the GPU name and SM
 * count, the algorithm, the chunking parameters and the batch's shape (file
 * count, log2 of its bytes, files of 1 MiB and more): a matching line sets the
 * tuning without running anything (*from_cache = 1); otherwise the batch is
 * tuned and a line is appended (*from_cache = 0). An unwritable file only
 * skips the append. HG_EINVAL if cache_path is NULL. */
int hg_batch_autotune_cached(hg_batch *batch, int algo, const uint8_t *d_data, uint64_t *d_ends,
                             uint64_t *d_counts, uint8_t *d_digests, void *stream,
                             const char *cache_path, hg_batch_tuning *best, int *from_cache);

/*
 * Request server with continuous batching (Sec. 3.2.3: applications submit
 * jobs to an outstanding queue, a manager thread per GPU runs them and
 * notifies completion; buffers are preallocated and reused; transfers overlap
 * computation). One progress thread per server admits requests in arrival
 * order while their input fits in a device arena of device_budget bytes
 * (allocated once at creation, with the per-wave scratch carved from the same
 * budget), copies them to the device on a copy stream (inputs up to 2 MiB
 * that lie in pinned host memory the device has mapped are pulled by one
 * gather kernel per wave instead of one copy call each), and runs everything
 * admitted together as one wave: one batched chunking job for the chunking
 * requests and the fixed-block kernels for the block requests, then one copy
 * of the wave's outputs to pinned host memory. Up to max_inflight_waves waves
 * are on the GPU at once; requests that arrive meanwhile are admitted as soon
 * as arena memory and a wave slot free up.
 *
 * Results are exactly those of hg_cdc_boundaries + hg_hash_chunks (kind
 * HG_REQ_CDC, chunking with the server's cdc parameters) or hg_hash_blocks
 * (kind HG_REQ_BLOCKS) on the request alone.
 */
typedef enum { HG_REQ_CDC = 0, HG_REQ_BLOCKS = 1 } hg_req_kind;

typedef struct {
    int32_t kind;            /* hg_req_kind */
    int32_t algo;            /* HG_MD5 / HG_SHA1 */
    const uint8_t *h_data;   /* host bytes; pinned memory gives one-copy DMA (Sec. 3.1) */
    uint64_t n;              /* bytes */
    uint64_t block;          /* HG_REQ_BLOCKS: block size */
    int32_t want_root;       /* HG_REQ_BLOCKS: also the hash-of-hashes */
    int32_t reserved;
} hg_request;

typedef struct {
    int32_t status;          /* HG_OK or HG_ECANCELED */
    int32_t algo;
    uint64_t count;          /* chunks or blocks */
    const uint64_t *ends;    /* HG_REQ_CDC: chunk ends (count), NULL otherwise */
    const uint8_t *digests;  /* count * dlen bytes */
    uint8_t root[20];        /* HG_REQ_BLOCKS with want_root */
    uint64_t t_submit_ns, t_admit_ns, t_done_ns;   /* steady-clock timestamps */
} hg_result;

typedef struct {
    uint64_t device_budget;       /* device bytes for staging + wave scratch (32 GiB) */
    uint64_t max_wave_bytes;      /* input bytes per wave; larger requests are refused (1 GiB) */
    uint32_t max_wave_requests;   /* requests per wave (4096) */
    uint32_t max_inflight_waves;  /* waves on the GPU at once, 1..8 (3) */
    hg_cdc_params cdc;            /* chunking parameters of HG_REQ_CDC requests */
    uint64_t wave_target_bytes;   /* a wave takes no further request once that would
                                     bring its input past this many bytes; a single
                                     larger request (up to max_wave_bytes) still forms
                                     a wave of its own; 0 means max_wave_bytes
                                     (default 256 MiB) */
} hg_server_config;

typedef struct {
    uint64_t submitted, completed, cancelled, waves, bytes_done;
    uint64_t arena_used, arena_bytes, queued;
} hg_server_stats;

typedef struct hg_server hg_server;

void hg_server_default_config(hg_server_config *cfg);
/* HG_ENOMEM when the budget cannot hold the wave scratch plus one maximal wave
 * or exceeds the context's budget. Starts the progress thread. */
int hg_server_create(hg_ctx *ctx, const hg_server_config *cfg, hg_server **out);
/* Cancels requests not yet admitted, waits for the waves on the GPU, frees everything. */
int hg_server_destroy(hg_server *srv);
/* Queue a request; returns at once with a ticket. HG_ENOMEM if the request
 * alone exceeds a wave or the arena (it could never be admitted). The host
 * bytes must stay valid and unchanged until the request completes. */
int hg_submit(hg_server *srv, const hg_request *req, uint64_t *ticket);
/* Cancel a request that is still queued (HG_EAGAIN once admitted). */
int hg_cancel(hg_server *srv, uint64_t ticket);
/* Wait up to timeout_us (-1: forever, 0: do not wait) for a request; HG_EAGAIN
 * if not done. The result's arrays stay valid until hg_release. */
int hg_poll(hg_server *srv, uint64_t ticket, hg_result *res, int64_t timeout_us);
int hg_release(hg_server *srv, uint64_t ticket);
/* Tickets completed since the previous call (up to max), waiting up to timeout_us for one. */
int hg_server_wait_any(hg_server *srv, uint64_t *tickets, uint32_t max, int64_t timeout_us,
                       uint32_t *n_out);
int hg_server_get_stats(hg_server *srv, hg_server_stats *stats);
/* Replay an open-loop trace: request i is submitted at arrival_ns[i] after the
 * call starts (non-decreasing); latency_ns[i] receives its completion time
 * minus its scheduled arrival; *span_ns the whole replay's duration. */
int hg_server_replay(hg_server *srv, const hg_request *reqs, const uint64_t *arrival_ns,
                     uint32_t nreq, uint64_t *latency_ns, uint64_t *span_ns);

/*
 * Device block map: similarity detection by digests (Sec. 2.1: identical
 * blocks have equal identifiers; Sec. 4.3: the share of a new version found in
 * chunks already stored). A hash table of distinct digests (algo fixes the
 * digest length, 16 or 20 bytes) in device memory, built and probed by
 * kernels, so a version's chunk digests are compared with everything stored
 * before without leaving the device. Digest arrays are rows of dlen bytes,
 * 4-byte aligned, as written by hg_hash_chunks / hg_cdc_hash.
 *
 * hg_blockmap_create: room for `capacity` distinct digests (2*capacity slots
 *   or more, 24 bytes each, counted against the context budget: HG_ENOMEM).
 * hg_blockmap_insert: adds count digests (min(count, *d_count) when d_count
 *   is not NULL); a digest already stored is not added again. Inserting more
 *   distinct digests than there are slots records HG_ECAPACITY in the context
 *   error word (read by hg_sync). Inserts and lookups on different streams
 *   must be ordered by the caller.
 * hg_blockmap_lookup: for query digest i, d_hits[i] = 1 if it is stored,
 *   else 0 (d_hits may be NULL); d_result[0] = number found and, when d_ends
 *   (the queried version's chunk ends) is not NULL, d_result[1] = bytes in the
 *   chunks found (d_result, 8-byte aligned, may be NULL; not both NULL).
 * hg_blockmap_count: enqueues a copy of the number of distinct digests stored
 *   to *d_out (device uint64).
 * hg_blockmap_clear: empties the map (stream-ordered).
 */
typedef struct hg_blockmap hg_blockmap;
int hg_blockmap_create(hg_ctx *ctx, int algo, uint64_t capacity, hg_blockmap **out);
int hg_blockmap_insert(hg_blockmap *map, const uint8_t *d_digests, uint64_t count,
                       const uint64_t *d_count, void *stream);
int hg_blockmap_lookup(hg_blockmap *map, const uint8_t *d_digests, const uint64_t *d_ends,
                       uint64_t count, const uint64_t *d_count, uint8_t *d_hits,
                       uint64_t *d_result, void *stream);
int hg_blockmap_count(hg_blockmap *map, uint64_t *d_out, void *stream);
int hg_blockmap_clear(hg_blockmap *map, void *stream);
int hg_blockmap_destroy(hg_blockmap *map);
/*
 * Bounded wait of hg_blockmap_insert: an insert that meets a slot claimed by
 * another insert of the same tag polls that slot's publish word at most
 * `polls` times (0 restores the default, 2^20) before it gives up and records
 * HG_ETIMEDOUT in the context's error word (returned by hg_sync); the kernel
 * then returns normally and the context stays usable.
 * hg_blockmap_inject_claim is fault injection for tests of that path, made on
 * the host: it synchronises `stream`, and writes h_digest's tag (host bytes,
 * dlen long) into its home slot without publishing it, as an insert that
 * claimed the slot and never finished would leave it. HG_EINVAL if the home
 * slot is already taken. Clear the map afterwards (hg_blockmap_clear).
 */
int hg_blockmap_set_wait_limit(hg_blockmap *map, uint32_t polls);
int hg_blockmap_inject_claim(hg_blockmap *map, const uint8_t *h_digest, void *stream);

/*
 * Chunk boundaries without allocating: the same result as hg_cdc_boundaries,
 * for callers that cannot call cudaMalloc -- a write path that must not stall
 * on the device-wide synchronisation cudaMalloc/cudaFree can cause, a process
 * whose device memory belongs to another allocator, or a service whose device
 * footprint must be fixed at load time. The paper has no counterpart.
 * No context is needed and nothing is allocated or freed: the scratch lives in
 * one static device array of the library (about 3.1 MiB, held by every GPU
 * that loads the library until the process exits). Inputs above
 * HG_STATIC_MAX_BYTES are rejected with HG_ECAPACITY before anything is
 * enqueued. Runs on the current CUDA device. Its first call on each device
 * looks up that device's address of the array and does the per-device
 * set-up of both window hashes (MD5 and Rabin); make that first call before
 * any stream capture. The looked-up address is kept for the life of the
 * process: after cudaDeviceReset on a device it is stale, so do not use this
 * call on a device that was reset. All calls share the one array: calls whose
 * work overlaps on the GPU (two streams, two host threads) race and corrupt
 * each other's results, so serialise them. If a bounded device-side wait gave
 * up, *d_count is set to UINT64_MAX. Other arguments and results as for
 * hg_cdc_boundaries.
 */
#define HG_STATIC_MAX_BYTES (16ull << 20)
int hg_cdc_boundaries_static(const uint8_t *d_in, uint64_t n, const hg_cdc_params *params,
                             uint64_t *d_ends, uint64_t cap, uint64_t *d_count, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* HASHGPU_H */
