// Direct hashing kernels: fixed-size blocks, the hash-of-hashes, and chunks.
//
// Sec. 3.2.2 ("Direct Hashing"): the data is split into segments hashed in
// parallel by independent GPU threads with the standard sequential digest,
// the digests go to one output buffer, and that buffer is hashed once more.
// Fig. 3: content-defined chunks are hashed by the same direct kernel.
#include "hg_device.cuh"
#include "hg_internal.h"

namespace hg {
namespace {

template <class H>
__global__ void __launch_bounds__(128) k_hash_blocks(const uint8_t *__restrict__ in, uint64_t n,
                                                     uint64_t block, uint64_t nblk,
                                                     uint8_t *__restrict__ out) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nblk) return;
    const uint64_t lo = i * block;
    const uint64_t len = (n - lo < block) ? n - lo : block;
    H hs;
    hash_range(in + lo, len, hs);
    store_digest(hs, out + i * H::kDigest);
}

// The hash-of-hashes is one sequential Merkle-Damgard chain over the digest
// buffer; a single thread runs it.
template <class H>
__global__ void k_root(const uint8_t *__restrict__ digests, uint64_t nbytes,
                       uint8_t *__restrict__ root) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    H hs;
    hash_range(digests, nbytes, hs);
    store_digest(hs, root);
}

template <class H>
__global__ void __launch_bounds__(128) k_hash_chunks(const uint8_t *__restrict__ in, uint64_t n,
                                                     const uint64_t *__restrict__ ends,
                                                     uint64_t nchunk,
                                                     const uint64_t *__restrict__ d_count,
                                                     uint8_t *__restrict__ out, int *err) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t cnt = nchunk;
    if (d_count) cnt = min(cnt, *d_count);
    if (i >= cnt) return;
    const uint64_t lo = i ? ends[i - 1] : 0, hi = ends[i];
    if (hi < lo || hi > n) {
        atomicCAS(err, 0, (int)HG_EINVAL);
        return;
    }
    H hs;
    hash_range(in + lo, hi - lo, hs);
    store_digest(hs, out + i * H::kDigest);
}

}  // namespace

int launch_hash_blocks(int algo, const uint8_t *d_in, uint64_t n, uint64_t block,
                       uint8_t *d_digests, cudaStream_t s, int *) {
    const uint64_t nblk = (n + block - 1) / block;
    if (nblk == 0) return HG_OK;
    const unsigned grid = (unsigned)((nblk + 127) / 128);
    if (algo == HG_MD5) k_hash_blocks<Md5><<<grid, 128, 0, s>>>(d_in, n, block, nblk, d_digests);
    else k_hash_blocks<Sha1><<<grid, 128, 0, s>>>(d_in, n, block, nblk, d_digests);
    return cuda_status(cudaGetLastError());
}

int launch_root(int algo, const uint8_t *d_digests, uint64_t nbytes, uint8_t *d_root,
                cudaStream_t s) {
    if (algo == HG_MD5) k_root<Md5><<<1, 32, 0, s>>>(d_digests, nbytes, d_root);
    else k_root<Sha1><<<1, 32, 0, s>>>(d_digests, nbytes, d_root);
    return cuda_status(cudaGetLastError());
}

int launch_hash_chunks(int algo, const uint8_t *d_in, uint64_t n, const uint64_t *d_ends,
                       uint64_t nchunk, const uint64_t *d_count, uint8_t *d_digests, cudaStream_t s,
                       int *d_err) {
    if (nchunk == 0) return HG_OK;
    const unsigned grid = (unsigned)((nchunk + 127) / 128);
    if (algo == HG_MD5)
        k_hash_chunks<Md5><<<grid, 128, 0, s>>>(d_in, n, d_ends, nchunk, d_count, d_digests, d_err);
    else
        k_hash_chunks<Sha1><<<grid, 128, 0, s>>>(d_in, n, d_ends, nchunk, d_count, d_digests, d_err);
    return cuda_status(cudaGetLastError());
}

}  // namespace hg
