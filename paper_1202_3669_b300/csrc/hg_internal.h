// Internal declarations shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "hashgpu.h"

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
};

namespace hg {

// Window kernel geometry: 256 threads x 32 consecutive window ends per CTA.
constexpr int kWinThreads = 256;
constexpr int kWinPerThread = 32;
constexpr uint64_t kWinTile = (uint64_t)kWinThreads * kWinPerThread;

// Candidate-list capacity used by hg_cdc_boundaries for an n-byte input. The
// expected density is 2^-mask_bits per byte; denser inputs fall back to
// scanning the bitmap during selection.
inline uint64_t cand_capacity(uint64_t n) { return n / 128 + 4096; }

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

// hg_cdc.cu
int launch_window_bitmap(const uint8_t *d_in, uint64_t n, const hg_cdc_params &p,
                         uint32_t *d_bitmap, uint32_t *d_tile_cnt, cudaStream_t s, int *d_err);
int launch_compact(const uint32_t *d_bitmap, uint64_t n, const uint32_t *d_tile_cnt,
                   uint64_t *d_tile_off, uint64_t ntiles, uint64_t *d_cands, uint64_t cap,
                   uint64_t *d_count, cudaStream_t s);
int launch_select(const uint64_t *d_cands, const uint64_t *d_ncand, uint64_t cand_cap,
                  const uint32_t *d_bitmap, uint64_t n, const hg_cdc_params &p, uint64_t *d_ends,
                  uint64_t cap, uint64_t *d_count, cudaStream_t s);

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? HG_OK : HG_ECUDA; }

}  // namespace hg
