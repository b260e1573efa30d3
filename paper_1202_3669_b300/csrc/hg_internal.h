// Internal declarations shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <deque>
#include <mutex>
#include <vector>
#include <cuda_runtime.h>

#include "hashgpu.h"

namespace hg {
struct PinnedPool;
struct RootJob {          // a hash-of-hashes computed on the host (hg_hostroot.cu)
    int algo;
    uint64_t nbytes;
};
}

struct hg_ctx {
    int device = 0;
    int num_sms = 0;
    size_t budget = 0;
    size_t held = 0;
    int *d_err = nullptr;            // device error word (first error wins)
    // content-defined chunking scratch
    uint32_t *d_bitmap = nullptr;    uint64_t bitmap_words = 0;
    uint32_t *d_tile_cnt = nullptr;  uint64_t tile_cap = 0;
    uint64_t *d_tile_off = nullptr;  uint64_t tile_off_cap = 0;
    uint64_t *d_cands = nullptr;     uint64_t cand_cap = 0;
    uint64_t *d_ncand = nullptr;     // one word
    uint8_t *d_segdig = nullptr;     uint64_t segdig_cap = 0;   // two-level segment digests
    uint32_t *d_tasks = nullptr;     uint64_t tasks_cap = 0;    // sorted chunk-digest tasks
    // pipelined chunking (hg_cdc_hash): streams, events, device state
    bool pipe_ready = false;
    cudaStream_t p_win = nullptr, p_sel = nullptr, p_hash[64] = {};
    cudaEvent_t p_fork = nullptr, p_done_sel = nullptr, p_join[64] = {};
    cudaEvent_t p_ev_win[64] = {}, p_ev_sel[64] = {};
    void *d_pipe = nullptr;
    cudaStream_t p_cap = nullptr;           // capture origin of the pipeline graph
    cudaStream_t p_copy = nullptr;          // host -> device segment copies (hg_cdc_hash_h2d)
    cudaEvent_t p_ev_copy[64] = {};
    cudaGraphExec_t p_exec = nullptr;       // replayed while p_key matches
    uint64_t p_key[16] = {};
    uint64_t scratch_gen = 0;               // bumped whenever scratch is reallocated
    // pinned host buffer pool (hg_pinned.cu), created on first use
    std::mutex pinned_mu;
    struct hg::PinnedPool *pinned = nullptr;
    // host-side hash-of-hashes: pinned staging (digests, then a 64-byte root
    // slot at root_cap) and the jobs enqueued but not yet run, in stream order
    uint8_t *root_stage = nullptr;
    uint64_t root_cap = 0;
    std::mutex root_mu;
    std::deque<hg::RootJob> root_jobs;
};

namespace hg {

// Window kernel geometry: 256 threads x 32 consecutive window ends per CTA.
constexpr int kWinThreads = 256;
constexpr int kWinPerThread = 32;
constexpr uint64_t kWinTile = (uint64_t)kWinThreads * kWinPerThread;
// The single-buffer MD5 window kernel runs one warp per CTA over a span of
// kWinSpan window ends (an eighth of a tile).
constexpr int kWinSpan = 32 * kWinPerThread;

// Grid of a chain kernel whose tasks are dealt to `lanes` lanes of each warp
// (see chain_task) for ntask tasks and `threads` threads per CTA.
inline unsigned chain_grid(uint64_t ntask, unsigned lanes, unsigned threads) {
    return (unsigned)((ntask * (32 / lanes) + threads - 1) / threads);
}

// Candidate-list capacity used by hg_cdc_boundaries for an n-byte input. The
// expected density is 2^-mask_bits per byte; denser inputs fall back to
// scanning the bitmap during selection.
constexpr uint64_t cand_capacity(uint64_t n) { return n / 128 + 4096; }

// Scratch management (hg_api.cu). Grows *p to hold `count` elements of
// `elem` bytes; returns HG_OK / HG_ENOMEM / HG_ECUDA.
int ensure(hg_ctx *ctx, void **p, uint64_t *cap, uint64_t count, size_t elem);

// hg_direct.cu
int launch_hash_blocks(int algo, const uint8_t *d_in, uint64_t n, uint64_t block,
                       uint8_t *d_digests, cudaStream_t s, int *d_err);
int launch_root(int algo, const uint8_t *d_digests, uint64_t nbytes, uint8_t *d_root,
                cudaStream_t s);
int launch_hash_chunks(int algo, const uint8_t *d_in, uint64_t n, const uint64_t *d_ends,
                       uint64_t nchunk,
                       const uint64_t *d_count, uint8_t *d_digests, cudaStream_t s, int *d_err);

// Fixed-block request of a batched launch: blocks of `block` bytes of ptr[0..len),
// digests to out (4-byte aligned), root (if asked) right after them.
struct BlkReq {
    const uint8_t *ptr;
    uint64_t len, block;
    uint64_t first;        // global index of its first block in the launch
    uint8_t *out;
    int32_t algo, root;
};
int launch_multi_blocks(const BlkReq *d_reqs, uint32_t nreq, uint64_t total_blocks, cudaStream_t s);

// Pipelined chunking of one buffer (hg_cdc_hash): device state.
constexpr int kMaxSeg = 64;
struct PipeState {
    uint64_t carry;      // start of the chunk still open after the last segment
    uint64_t count;      // chunks finalized so far
    uint64_t ncand;      // candidates found so far
    uint64_t start0;     // start of the first chunk (0 for a whole buffer)
    uint64_t seg_cnt[kMaxSeg + 1];   // chunks finalized after segment k-1 (seg_cnt[0] = 0)
    uint64_t thr[kMaxSeg];           // segment k: chunks at least this long run on lone lanes
    uint32_t nlong[kMaxSeg];         // segment k: how many (listed in the long lists)
    uint32_t band_cnt[128];          // deferred digests: chunks per length band (longest first)
    uint32_t band_cur[128];          // and the bands' next free task slots
    unsigned long long task_ctr;     // deferred digests: next 32-task group for the bulk warps
};
// Longest chunks of a segment given a warp of their own (one lane active):
// a lone chain measured about 15-20 cycles per MD5 step against 27 when 32
// chains share a warp, and the longest chain is the step's tail. As many
// such warps per call as SMs (two concurrent 64 MiB calls: 63.1 GB/s against
// 60.8 with four times as many, which crowds the schedulers), capped at
// kLongMax.
constexpr uint32_t kLongMax = 1024;
constexpr size_t kLongListBytes = (size_t)kMaxSeg * kLongMax * sizeof(uint32_t);
inline uint32_t long_chains(int num_sms) {
    const uint32_t k = (uint32_t)(num_sms > 0 ? num_sms : 1);
    return k < kLongMax ? k : kLongMax;
}
struct PipeBufs {
    uint32_t *bitmap, *tile_cnt;
    uint64_t *tile_off, *cands, cand_cap;
    uint64_t *ends, cap;
    uint8_t *digests;
    PipeState *st;
    int *err;
    uint32_t *long_idx;   // kMaxSeg lists of kLongMax chunk indexes (relative to the segment)
    uint32_t klong;       // lone-lane chains per segment (<= kLongMax)
    uint32_t *tasks;      // deferred digests: chunk indexes sorted by length (cap entries)
};

// hg_cdc.cu
int launch_window_bitmap(const uint8_t *d_in, uint64_t n, const hg_cdc_params &p,
                         uint32_t *d_bitmap, uint32_t *d_tile_cnt, cudaStream_t s, int *d_err);
int launch_compact(const uint32_t *d_bitmap, uint64_t n, const uint32_t *d_tile_cnt,
                   uint64_t *d_tile_off, uint64_t ntiles, uint64_t *d_cands, uint64_t cap,
                   uint64_t *d_count, cudaStream_t s);
int launch_window_range(const uint8_t *d_in, uint64_t n, const hg_cdc_params &p,
                        uint32_t *d_bitmap, uint32_t *d_tile_cnt, uint32_t tile0, uint64_t ntiles,
                        cudaStream_t s, int *d_err);
// Rabin fingerprint window (hg_rabin.cu): same bitmap and tile counts.
// rabin_prepare: per-device kernel set-up for the current device, to be
// called outside stream capture (hg_init does).
int rabin_prepare();
int launch_window_rabin_range(const uint8_t *d_in, uint64_t n, const hg_cdc_params &p,
                              uint32_t *d_bitmap, uint32_t *d_tile_cnt, uint32_t tile0,
                              uint64_t ntiles, cudaStream_t s);
// n: bytes in d_in; n_sel: end of the stream for selection (n, or ~0 when the
// stream continues beyond d_in).
// Digests of all chunks a pipeline decided, after its last selection, in one
// launch: chunks counting-sorted by length (longest first), the longest klong
// on lone lanes, the rest 32 to a warp in that order. Used when a buffer has
// several segments, where per-segment digest launches would share the SMs
// with the later segments' window kernels.
int launch_hash_sorted(const uint8_t *d_in, uint64_t n, uint64_t max_chunks, const hg_cdc_params &p,
                       int algo, const PipeBufs &b, cudaStream_t s);
// digests = false: the segment's digests are left to launch_hash_sorted.
int launch_pipe_segment(const uint8_t *d_in, uint64_t n, uint64_t n_sel, const hg_cdc_params &p,
                        int algo, uint32_t tile0, uint32_t ntiles, uint64_t L, int seg,
                        uint64_t max_chunks, const PipeBufs &b, cudaStream_t s_win,
                        cudaStream_t s_sel, cudaStream_t s_hash, cudaEvent_t ev_win,
                        cudaEvent_t ev_sel, cudaEvent_t ev_input, bool digests = true);
// streaming chunking (hg_stream.cu helpers in hg_cdc.cu)
int launch_stream_init(PipeState *st, uint64_t start0, cudaStream_t s);
int launch_stream_out(const uint64_t *ends, const PipeState *st, uint64_t base, uint64_t *d_ends_out,
                      uint64_t cap, uint64_t *d_count_out, cudaStream_t s);
int launch_stream_carry(const uint8_t *src, uint64_t wl, const PipeState *st, uint32_t halo,
                        uint8_t *dst, uint64_t *info, cudaStream_t s);
int launch_scan_tiles(const uint32_t *d_tile_cnt, uint64_t ntiles, uint64_t *d_tile_off,
                      uint64_t *d_total, cudaStream_t s);
int launch_select(const uint64_t *d_cands, const uint64_t *d_ncand, uint64_t cand_cap,
                  const uint32_t *d_bitmap, uint64_t n, const hg_cdc_params &p, uint64_t *d_ends,
                  uint64_t cap, uint64_t *d_count, cudaStream_t s);

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? HG_OK : HG_ECUDA; }

// A kernel that takes more than the default 48 KiB of dynamic shared memory
// (the staged chains' rings) needs its limit raised before the launch; the
// call enqueues nothing, so it is also made while a stream is captured.
// Largest per-CTA dynamic shared memory used for staging rings (sm_103a
// allows 227 KiB a block; 256 threads' rings take 132 KiB).
constexpr size_t kStageSmemMax = 160u * 1024u;
inline cudaError_t allow_dyn_smem(const void *kernel, size_t bytes) {
    return bytes > 48u * 1024u
               ? cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)
               : cudaSuccess;
}

// Debug build (HG_DEBUG, libhashgpu_debug.so): kernels check the index of a
// global access that is not in range by construction alone; a failed check
// records HG_EBOUNDS in the error word and the access is skipped. In the
// release build HG_DOK is `true` and costs nothing.
#ifdef HG_DEBUG
#ifdef __CUDACC__
__device__ __forceinline__ bool hg_dok(bool ok, int *err) {
    if (!ok && err) atomicCAS(err, 0, (int)HG_EBOUNDS);
    return ok;
}
#endif
#define HG_DOK(cond, err) (::hg::hg_dok((cond), (err)))
#else
#define HG_DOK(cond, err) true
#endif

// hg_hostroot.cu: the library's host MD5/SHA-1, and the hash-of-hashes
// computed on a host core in stream order (digests copied to pinned staging,
// hashed by a host function, the root copied back). Digest lists shorter than
// host_root_min_bytes(algo), and calls on a capturing stream, use the device
// chain.
// HG_HOST_ROOT_MIN (bytes, read once) overrides the thresholds.
constexpr uint64_t kHostRootMinMd5 = 1ull << 20, kHostRootMinSha1Ni = 16ull << 10,
                   kHostRootMinSha1 = 256ull << 10;
uint64_t host_root_min_bytes(int algo);
void host_digest(int algo, const uint8_t *msg, uint64_t n, uint8_t *out);
int enqueue_host_root(hg_ctx *c, int algo, const uint8_t *d_digests, uint64_t nbytes, uint8_t *d_root,
                      cudaStream_t s);

// hg_pinned.cu: the pinned host buffer pool.
constexpr uint64_t kPinnedDefaultBudget = 16ull << 30;
uint64_t pinned_class(uint64_t n);
void pinned_destroy(hg_ctx *c);   // frees every buffer of the pool (device synchronised first)

// ---- batched chunking jobs (hg_job.cu) -------------------------------------------------
// Files from this size up select their boundaries with a whole CTA.
constexpr uint64_t kJobBigFileBytes = 1ull << 20;
// counters of a job (device words)
enum { kJobTotal = 0, kJobTaskCtr = 1, kJobTileCtr = 2, kJobHist = 8, kJobNumWords = 8 + 128 };

// Device view of a job: file f is jptr(f) .. + jlen(f): base + file_off[f] when
// base is set (files back to back), else file_ptr[f] / file_len[f]. Its tiles
// are [tile_start[f], tile_start[f+1]), its output slots [slot_off[f],
// slot_off[f+1]); small / big list the files by selection method.
struct JobDev {
    const uint8_t *base;
    const uint64_t *file_off;
    const uint8_t *const *file_ptr;
    const uint64_t *file_len;
    const uint64_t *tile_start;
    const uint64_t *slot_off;
    const uint32_t *small;
    const uint32_t *big;
    uint32_t nfile, nsmall, nbig, ntiles;
};

struct JobScratch {
    uint32_t *bitmap;      // ntiles * kWinThreads words
    uint32_t *tile_cnt;    // ntiles
    uint64_t *tile_off;    // ntiles + 1 (last = candidate count)
    uint64_t *cands;
    uint64_t cand_cap;
    uint64_t *tasks;       // total_slots
    unsigned long long *words;
    int *err;
};

struct JobTuning {
    int window_ctas;       // persistent window CTAs per SM
    int hash_threads;
    int hash_ctas;         // chunk-hash CTAs per SM
    uint64_t long_bytes;   // kept for the tuning record; tasks are ordered by length
};

struct JobHost {
    std::vector<uint64_t> tile_start, slot_off;
    std::vector<uint32_t> small, big;
    uint64_t ntiles = 0, total_slots = 0;
};

void job_plan(const uint64_t *len, uint32_t nfile, uint64_t min_chunk, JobHost *h);
size_t job_scratch_bytes(uint64_t ntiles, uint64_t cand_cap, uint64_t total_slots);
void job_scratch_carve(char *mem, uint64_t ntiles, uint64_t cand_cap, uint64_t total_slots,
                       JobScratch *sc);
int job_window_occupancy(uint32_t window);
// Shared-memory opt-in of the batch-job Rabin window kernels (current device).
int job_rabin_prepare();
int enqueue_cdc_job(const JobDev &j, const JobScratch &sc, const hg_cdc_params &p, int algo,
                    const JobTuning &tn, int num_sms, uint64_t *d_ends, uint64_t *d_counts,
                    uint8_t *d_digests, cudaStream_t s);

}  // namespace hg
