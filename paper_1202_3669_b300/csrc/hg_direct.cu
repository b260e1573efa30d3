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

// One full block of a 16-byte aligned input whose block size is a multiple of
// 64: four aligned 16-byte loads per MD5/SHA-1 block and the padding block as
// constants.
// 32 bytes of global memory into eight registers (one 256-bit load; the
// address must be 32-byte aligned).
__device__ __forceinline__ void ld32(const uint8_t *p, uint32_t *v) {
    asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7])
                 : "l"(p));
}

template <class H>
__device__ __forceinline__ void hash_aligned_block(const uint8_t *__restrict__ in, uint64_t block,
                                                   uint64_t i, uint8_t *__restrict__ out,
                                                   uint32_t one) {
    const uint4 *p = reinterpret_cast<const uint4 *>(in + i * block);
    const uint64_t nb = block >> 6;
    H hs;
    hs.init();
    hs.set_one(one);
    for (uint64_t k = 0; k < nb; k++) {
        const uint4 x0 = __ldg(p + 4 * k), x1 = __ldg(p + 4 * k + 1);
        const uint4 x2 = __ldg(p + 4 * k + 2), x3 = __ldg(p + 4 * k + 3);
        const uint32_t M[16] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w,
                                x2.x, x2.y, x2.z, x2.w, x3.x, x3.y, x3.z, x3.w};
        hs.compress(M);
    }
    uint32_t Z[16] = {0x80u, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    H::put_length(Z, block);
    hs.compress(Z);
    store_digest(hs, out + i * H::kDigest);
}

// Many blocks: the throughput form, one chain per thread, 16-byte loads. MD5
// is capped at 32 registers so 2048 threads fit an SM (occupancy is what hides
// the loads: 4.1 vs 3.3 TB/s at 37 registers) and runs Md5Split with pipe
// policy 1 (the logic op's add on the FMA pipe); a 32-byte aligned input takes
// k_hash_blocks_aligned_x2 instead. SHA-1 runs Sha1Split with pipe policy 3
// (e + W on the FMA pipe) at 12 CTAs per SM (40 registers, no spills): 1 GiB in
// 4 KiB blocks 0.534 -> 0.461 ms; at 16 CTAs per SM the same code spills, and
// 32-byte loads gave it nothing (0.459 ms).
template <class H> struct AlignedForm;
template <> struct AlignedForm<Md5> {
    using Hash = Md5Split<kPolAll1>;
    static constexpr int kMinCtas = 16;
};
template <> struct AlignedForm<Sha1> {
    using Hash = Sha1Split<0xFFFFu>;
    static constexpr int kMinCtas = 12;
};

template <class H>
__global__ void __launch_bounds__(128, AlignedForm<H>::kMinCtas)
    k_hash_blocks_aligned(const uint8_t *__restrict__ in, uint64_t block, uint64_t nfull,
                          uint8_t *__restrict__ out, uint32_t one) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nfull) hash_aligned_block<typename AlignedForm<H>::Hash>(in, block, i, out, one);
}

// MD5 on a 32-byte aligned input: two 256-bit loads per 64-byte block (the
// 16-byte form is bound by L1 tag throughput: each lane's load touches its own
// 128-byte line, so a warp load costs 32 wavefronts for 512 bytes) and two
// blocks per thread, their compressions interleaved (two independent chains,
// 63 registers, 8 CTAs/SM resident). 1 GiB in 4 KiB blocks: 0.248 ms with one
// block per thread and 16-byte loads, 0.239 with 32-byte loads, 0.231 (4.64
// TB/s) with two blocks; an L2 prefetch 2-8 blocks ahead was slower (0.258-0.37
// ms), and the interleave gave SHA-1 nothing. Declared for 6 CTAs/SM: the same
// 63 registers and residency, scheduled ~1.5 % faster than when declared for 8
// (0.2294 vs 0.2315-0.2335 ms with L2 flushed; 4, 5 and 7 equal 6).
template <class H>
__global__ void __launch_bounds__(128, 6) k_hash_blocks_aligned_x2(const uint8_t *__restrict__ in,
                                                                    uint64_t block, uint64_t nfull,
                                                                    uint8_t *__restrict__ out,
                                                                    uint32_t one) {
    const uint64_t i0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * 2;
    if (i0 >= nfull) return;
    const bool two = i0 + 1 < nfull;
    const uint8_t *p0 = in + i0 * block, *p1 = in + (two ? i0 + 1 : i0) * block;
    const uint64_t nb = block >> 6;
    H h0, h1;
    h0.init();
    h0.set_one(one);
    h1.init();
    h1.set_one(one);
    for (uint64_t k = 0; k < nb; k++) {
        uint32_t M0[16], M1[16];
        ld32(p0 + 64 * k, M0);
        ld32(p0 + 64 * k + 32, M0 + 8);
        ld32(p1 + 64 * k, M1);
        ld32(p1 + 64 * k + 32, M1 + 8);
        h0.compress(M0);
        h1.compress(M1);
    }
    uint32_t Z0[16] = {0x80u, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    uint32_t Z1[16] = {0x80u, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    H::put_length(Z0, block);
    H::put_length(Z1, block);
    h0.compress(Z0);
    h1.compress(Z1);
    store_digest(h0, out + i0 * H::kDigest);
    if (two) store_digest(h1, out + (i0 + 1) * H::kDigest);
}

// Few blocks (fewer chains than it takes to fill the integer pipes): each
// block is a latency-bound chain, so the chain form of the step, the message
// staged through shared memory (hash_range_staged), no register cap, and
// half warps in two-warp CTAs when the chains are very few (chain_task).
// With more chains, full warps in four-warp CTAs: one CTA per SM puts one
// warp on each scheduler, where a 32-lane MD5 chain warp keeps the ALU pipe
// ~70 % busy by itself; with two-warp CTAs an SM that received several of
// them ran two or three chain warps per scheduler (1 GiB in 64 KiB blocks:
// 0.52 ms, or 1.03 ms when the CTAs bunched). With one block loaded ahead into
// registers instead of staged: 0.686 ms.
template <class H>
__global__ void __launch_bounds__(128) k_hash_blocks_aligned_few(const uint8_t *__restrict__ in,
                                                                 uint64_t block, uint64_t nfull,
                                                                 uint32_t lanes,
                                                                 uint8_t *__restrict__ out) {
    uint64_t i;
    if (!chain_task(i, lanes) || i >= nfull) return;
    H hs;
    hash_range_staged(in + i * block, block, hs, stage_ring_dyn());
    store_digest(hs, out + i * H::kDigest);
}

// The hash-of-hashes is one sequential Merkle-Damgard chain over the digest
// buffer; a single thread runs it.
template <class H>
__global__ void __launch_bounds__(32) k_root(const uint8_t *__restrict__ digests, uint64_t nbytes,
                                             uint8_t *__restrict__ root) {
    __shared__ __align__(16) uint4 ring[kStageStride];
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    H hs;
    hash_range_staged(digests, nbytes, hs, ring);
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
    hash_range_staged(in + lo, hi - lo, hs, stage_ring_dyn());
    store_digest(hs, out + i * H::kDigest);
}

// All fixed-block requests of a batch in one launch: one thread per block of
// any request (block i of request r is global block reqs[r].first + i).
__global__ void __launch_bounds__(128) k_multi_blocks(const BlkReq *__restrict__ reqs, uint32_t nreq,
                                                      uint64_t total_blocks) {
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total_blocks) return;
    uint32_t lo = 0, hi = nreq;                       // last r with first <= g
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) / 2;
        if (reqs[mid].first <= g) lo = mid; else hi = mid;
    }
    const BlkReq r = reqs[lo];
    const uint64_t i = g - r.first;
    const uint64_t off = i * r.block;
    const uint64_t len = (r.len - off < r.block) ? r.len - off : r.block;
    if (r.algo == HG_MD5) {
        Md5Chain hs;
        hash_range_staged(r.ptr + off, len, hs, stage_ring_dyn());
        store_digest(hs, r.out + i * Md5::kDigest);
    } else {
        Sha1 hs;
        hash_range_staged(r.ptr + off, len, hs, stage_ring_dyn());
        store_digest(hs, r.out + i * Sha1::kDigest);
    }
}

// Hash-of-hashes of every request that asks for one (one thread each); its
// root goes right after its block digests.
__global__ void k_multi_roots(const BlkReq *__restrict__ reqs, uint32_t nreq) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nreq || !reqs[k].root) return;
    const BlkReq r = reqs[k];
    const uint64_t nblk = (r.len + r.block - 1) / r.block;
    if (r.algo == HG_MD5) {
        Md5Chain hs;
        hash_range_staged(r.out, nblk * Md5::kDigest, hs, stage_ring_dyn());
        store_digest(hs, r.out + nblk * Md5::kDigest);
    } else {
        Sha1 hs;
        hash_range_staged(r.out, nblk * Sha1::kDigest, hs, stage_ring_dyn());
        store_digest(hs, r.out + nblk * Sha1::kDigest);
    }
}

}  // namespace

int launch_multi_blocks(const BlkReq *d_reqs, uint32_t nreq, uint64_t total_blocks, cudaStream_t s) {
    if (nreq == 0) return HG_OK;
    const size_t smem = stage_bytes(128);
    if (allow_dyn_smem((const void *)k_multi_blocks, smem) != cudaSuccess ||
        allow_dyn_smem((const void *)k_multi_roots, smem) != cudaSuccess)
        return HG_ECUDA;
    if (total_blocks)
        k_multi_blocks<<<(unsigned)((total_blocks + 127) / 128), 128, smem, s>>>(d_reqs, nreq,
                                                                                 total_blocks);
    k_multi_roots<<<(nreq + 127) / 128, 128, smem, s>>>(d_reqs, nreq);
    return cuda_status(cudaGetLastError());
}

// Below this many chains (about 512 threads per SM) the block kernels are
// latency-bound rather than integer-pipe-bound.
constexpr uint64_t kFewChains = 148ull * 512;

int launch_hash_blocks(int algo, const uint8_t *d_in, uint64_t n, uint64_t block,
                       uint8_t *d_digests, cudaStream_t s, int *) {
    const uint64_t nblk = (n + block - 1) / block;
    if (nblk == 0) return HG_OK;
    const bool aligned = ((reinterpret_cast<uintptr_t>(d_in) & 15) == 0) && (block % 64) == 0;
    if (aligned) {
        // full blocks by the aligned kernel, a short last block (if any) by the generic one
        const uint64_t nfull = n / block;
        if (nfull >= kFewChains) {
            const unsigned grid = (unsigned)((nfull + 127) / 128);
            const bool a32 = (reinterpret_cast<uintptr_t>(d_in) & 31) == 0;
            if (algo == HG_MD5 && a32)
                k_hash_blocks_aligned_x2<Md5Split<kPolAll1>><<<(unsigned)((nfull + 255) / 256), 128, 0, s>>>(
                    d_in, block, nfull, d_digests, 1u);
            else if (algo == HG_MD5)
                k_hash_blocks_aligned<Md5><<<grid, 128, 0, s>>>(d_in, block, nfull, d_digests, 1u);
            else
                k_hash_blocks_aligned<Sha1><<<grid, 128, 0, s>>>(d_in, block, nfull, d_digests, 1u);
        } else if (nfull) {
            const uint32_t lanes = nfull <= kHalfWarpChainsMax ? 16 : 32;
            const unsigned threads = lanes == 16 ? 64 : 128;
            const unsigned grid = chain_grid(nfull, lanes, threads);
            const size_t smem = stage_bytes(threads);
            const void *k = algo == HG_MD5 ? (const void *)k_hash_blocks_aligned_few<Md5Chain>
                                           : (const void *)k_hash_blocks_aligned_few<Sha1>;
            if (allow_dyn_smem(k, smem) != cudaSuccess) return HG_ECUDA;
            if (algo == HG_MD5)
                k_hash_blocks_aligned_few<Md5Chain><<<grid, threads, smem, s>>>(d_in, block, nfull,
                                                                               lanes, d_digests);
            else
                k_hash_blocks_aligned_few<Sha1><<<grid, threads, smem, s>>>(d_in, block, nfull, lanes,
                                                                           d_digests);
        }
        if (nfull < nblk) {
            const uint64_t lo = nfull * block;
            const int dl = algo == HG_MD5 ? 16 : 20;
            if (algo == HG_MD5)
                k_hash_blocks<Md5Chain><<<1, 32, 0, s>>>(d_in + lo, n - lo, block, 1, d_digests + nfull * dl);
            else
                k_hash_blocks<Sha1><<<1, 32, 0, s>>>(d_in + lo, n - lo, block, 1, d_digests + nfull * dl);
        }
        return cuda_status(cudaGetLastError());
    }
    const unsigned grid = (unsigned)((nblk + 127) / 128);
    if (algo == HG_MD5) k_hash_blocks<Md5><<<grid, 128, 0, s>>>(d_in, n, block, nblk, d_digests);
    else k_hash_blocks<Sha1><<<grid, 128, 0, s>>>(d_in, n, block, nblk, d_digests);
    return cuda_status(cudaGetLastError());
}

int launch_root(int algo, const uint8_t *d_digests, uint64_t nbytes, uint8_t *d_root,
                cudaStream_t s) {
    if (algo == HG_MD5) k_root<Md5Chain><<<1, 32, 0, s>>>(d_digests, nbytes, d_root);
    else k_root<Sha1><<<1, 32, 0, s>>>(d_digests, nbytes, d_root);
    return cuda_status(cudaGetLastError());
}

int launch_hash_chunks(int algo, const uint8_t *d_in, uint64_t n, const uint64_t *d_ends,
                       uint64_t nchunk, const uint64_t *d_count, uint8_t *d_digests, cudaStream_t s,
                       int *d_err) {
    if (nchunk == 0) return HG_OK;
    const unsigned grid = (unsigned)((nchunk + 127) / 128);
    const size_t smem = stage_bytes(128);
    if (algo == HG_MD5) {
        if (allow_dyn_smem((const void *)k_hash_chunks<Md5Chain>, smem) != cudaSuccess) return HG_ECUDA;
        k_hash_chunks<Md5Chain><<<grid, 128, smem, s>>>(d_in, n, d_ends, nchunk, d_count, d_digests,
                                                        d_err);
    } else {
        if (allow_dyn_smem((const void *)k_hash_chunks<Sha1>, smem) != cudaSuccess) return HG_ECUDA;
        k_hash_chunks<Sha1><<<grid, 128, smem, s>>>(d_in, n, d_ends, nchunk, d_count, d_digests, d_err);
    }
    return cuda_status(cudaGetLastError());
}

}  // namespace hg
