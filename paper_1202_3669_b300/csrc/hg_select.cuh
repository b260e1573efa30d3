// Exact min/max chunk-boundary selection on the device (Sec. 2.1 content-based
// chunking with minimum and maximum chunk sizes): shared by the single-stream
// and the batched paths.
//
// The greedy rule makes the chunk chain a deterministic function of its
// current start: two chains that ever cut at the same candidate coincide from
// there on. For a block-wide selection the candidates are split into nseg
// segments of K; S_j is the chain that starts with a cut at candidate j*K.
// Phase 1 finds, for every j, the candidate q_j where S_j and S_{j+1} meet
// (two-pointer walk; chains meet within a few cuts because a chunk spans only
// a few candidates), and q_{-1} where the true chain T from the stream start
// meets S_0. With x_0 = q_{-1} and x_{j+1} = max(x_j, q_j), T is the walk from
// the start to x_0 followed by the pieces of S_j from x_j to x_{j+1}; each
// piece is walked twice more, once to count its cuts and once to write them at
// their scanned offsets.
//
// Positions are absolute offsets into the buffer that holds the stream; the
// stream occupies [s0, n) and cuts are written relative to s0.
//
// A limit L < n says only the candidates up to L are known (a stream being
// chunked segment by segment): a cut is emitted only when the candidates up to
// L decide it, and a chain whose next decision needs more stops (returns m)
// without emitting. L >= n means everything is known.
#pragma once
#include <cstdint>

namespace hg {

constexpr int kSelThreads = 1024;
// select_block stages up to kSelStage candidates in shared memory as 32-bit
// offsets from the first one: the chain walks below are chains of dependent
// searches, ~30 cycles a read from shared memory against ~500 from L2
// (64 MiB, ~8 K candidates: k_select_par 41 -> 27 us, k_select_seg 34.5 -> 29.6 us).
constexpr uint32_t kSelStage = 9216;

// Sorted candidate cuts read straight from global memory.
struct CandsGlobal {
    const uint64_t *__restrict__ c;
    __device__ __forceinline__ uint64_t operator[](uint32_t i) const { return __ldg(c + i); }
};
// Sorted candidate cuts staged in shared memory as offsets from base.
struct CandsShared {
    const uint32_t *c;
    uint64_t base;
    __device__ __forceinline__ uint64_t operator[](uint32_t i) const { return base + c[i]; }
};

// First index j >= k with C[j] >= target (m if none); C is sorted.
template <class CA>
__device__ __forceinline__ uint32_t lower_bound_from(const CA &C, uint32_t m, uint32_t k,
                                                     uint64_t target) {
    if (k >= m || C[k] >= target) return k;
    uint32_t lo = k, hi = m, step = 1;                    // C[lo] < target
    while (true) {                                        // gallop
        const uint64_t probe = (uint64_t)lo + step;
        if (probe >= m) break;
        if (C[(uint32_t)probe] >= target) { hi = (uint32_t)probe; break; }
        lo = (uint32_t)probe;
        step <<= 1;
    }
    while (hi - lo > 1) {                                 // C[lo] < target <= C[hi]
        const uint32_t mid = lo + (hi - lo) / 2;
        if (C[mid] >= target) hi = mid; else lo = mid;
    }
    return hi;
}

struct NoEmit {
    __device__ __forceinline__ void operator()(uint64_t) const {}
};
struct CountEmit {
    uint64_t *c;
    __device__ __forceinline__ void operator()(uint64_t) const { ++*c; }
};
struct WriteEmit {
    uint64_t *ends, cap, *idx, base;
    __device__ __forceinline__ void operator()(uint64_t cut) const {
        if (*idx < cap) ends[*idx] = cut - base;
        ++*idx;
    }
};

// One chain step from chunk start s (search for candidates from index k on):
// emits every cut up to and including the next candidate cut and returns that
// candidate's index, or emits the remaining forced cuts and n and returns m,
// or (limit reached) stops and returns m.
template <class CA, class Emit>
__device__ uint32_t chain_next(const CA &C, uint32_t m, uint64_t n, uint64_t L, uint64_t mn,
                               uint64_t mx, uint64_t s, uint32_t k, Emit emit) {
    while (s < n) {
        const uint32_t j = lower_bound_from(C, m, k, s + mn);
        if (j < m && C[j] <= s + mx) {
            emit(C[j]);
            return j;
        }
        if (s + mx > L && L < n) return m;                 // undecided until more is known
        if (s + mx < n) {
            s += mx;                                       // forced cut
            emit(s);
            k = j;
        } else {
            emit(n);                                       // last chunk
            return m;
        }
    }
    return m;
}

template <class CA, class Emit>
__device__ __forceinline__ uint32_t step_from(const CA &C, uint32_t m, uint64_t n, uint64_t L,
                                              uint64_t mn, uint64_t mx, uint32_t node, Emit emit) {
    return chain_next(C, m, n, L, mn, mx, C[node], node + 1, emit);
}

// The whole chain of a stream by one thread (used for streams with few candidates).
template <class Emit>
__device__ void select_thread(const uint64_t *__restrict__ Cg, uint32_t m, uint64_t s0, uint64_t n,
                              uint64_t mn, uint64_t mx, Emit emit) {
    const CandsGlobal C{Cg};
    const uint64_t L = ~0ull;
    uint32_t cur = chain_next(C, m, n, L, mn, mx, s0, 0, emit);
    while (cur != m) cur = step_from(C, m, n, L, mn, mx, cur, emit);
}

// Walk piece p (-1: from s0 to x[0]; j >= 0: from x[j] to x[j+1]).
template <class CA, class Emit>
__device__ void walk_piece(const CA &C, uint32_t m, uint64_t s0, uint64_t n, uint64_t L,
                           uint64_t mn, uint64_t mx, int p, const uint32_t *x, Emit emit) {
    uint32_t cur, to;
    if (p < 0) {
        to = x[0];
        cur = chain_next(C, m, n, L, mn, mx, s0, 0, emit);
    } else {
        cur = x[p];
        to = x[p + 1];
    }
    while (cur != to) cur = step_from(C, m, n, L, mn, mx, cur, emit);
}

// The phases of select_block over candidates C (global or staged).
template <class CA>
__device__ void select_block_run(const CA &C, uint32_t m, uint64_t s0, uint64_t n, uint64_t mn,
                                 uint64_t mx, uint64_t *__restrict__ ends, uint64_t cap,
                                 uint64_t *__restrict__ d_count, uint64_t L, uint64_t out_base,
                                 uint32_t *q, uint32_t *x, uint64_t *warp_tot) {
    const int t = threadIdx.x;
    const uint32_t K = max(16u, (m + kSelThreads - 2) / (kSelThreads - 1));
    const int nseg = (int)((m + K - 1) / K);              // <= kSelThreads - 1
    const int p = t - 1;                                  // piece / chain index of this thread

    // phase 1: meeting points
    if (p >= -1 && p < nseg) {
        uint32_t a, b;
        if (p < 0) {
            a = chain_next(C, m, n, L, mn, mx, s0, 0, NoEmit{});
            b = nseg > 0 ? 0 : m;
        } else {
            a = (uint32_t)p * K;
            b = (p + 1 < nseg) ? (uint32_t)(p + 1) * K : m;
        }
        while (a != b) {
            if (a < b) a = step_from(C, m, n, L, mn, mx, a, NoEmit{});
            else b = step_from(C, m, n, L, mn, mx, b, NoEmit{});
        }
        q[t] = a;
    }
    __syncthreads();
    // phase 2: x[0] = q_{-1}, x[j+1] = max(x[j], q_j): x is the running
    // maximum of q[0..t], a block-wide inclusive max-scan over t <= nseg
    {
        uint32_t v = t <= nseg ? q[t] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, v, d);
            if ((t & 31) >= d) v = max(v, y);
        }
        uint32_t *wmax = reinterpret_cast<uint32_t *>(warp_tot);
        if ((t & 31) == 31) wmax[t >> 5] = v;
        __syncthreads();
        if (t < 32) {
            uint32_t w = wmax[t];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, w, d);
                if (t >= d) w = max(w, y);
            }
            wmax[t] = w;
        }
        __syncthreads();
        if (t <= nseg) x[t] = (t >> 5) ? max(v, wmax[(t >> 5) - 1]) : v;
        __syncthreads();
    }
    // phase 3: count cuts per piece
    uint64_t c = 0;
    if (n > s0 && p >= -1 && p < nseg) walk_piece(C, m, s0, n, L, mn, mx, p, x, CountEmit{&c});
    // phase 4: exclusive scan of counts over the block
    uint64_t v = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, v, d);
        if ((t & 31) >= d) v += y;
    }
    if ((t & 31) == 31) warp_tot[t >> 5] = v;
    __syncthreads();
    if (t < 32) {
        uint64_t w = warp_tot[t];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, w, d);
            if (t >= d) w += y;
        }
        warp_tot[t] = w;
    }
    __syncthreads();
    const uint64_t excl = v - c + ((t >> 5) ? warp_tot[(t >> 5) - 1] : 0);
    if (t == kSelThreads - 1) *d_count = excl + c;
    // phase 5: write
    if (n > s0 && p >= -1 && p < nseg && c) {
        uint64_t idx = excl;
        walk_piece(C, m, s0, n, L, mn, mx, p, x, WriteEmit{ends, cap, &idx, out_base});
    }
}

// Block-wide exact selection (blockDim.x == kSelThreads) of the stream [s0, n)
// whose sorted candidate cuts (all known ones, up to L) are C[0..m). Writes at
// most cap cuts (relative to s0) to ends and the count to *d_count. Up to
// kSelStage candidates spanning less than 4 GiB are first copied to shared
// memory (as offsets from C[0]); the walks then read them there.
static __device__ void select_block(const uint64_t *__restrict__ C, uint32_t m, uint64_t s0,
                                    uint64_t n, uint64_t mn, uint64_t mx,
                                    uint64_t *__restrict__ ends, uint64_t cap,
                                    uint64_t *__restrict__ d_count, uint64_t L = ~0ull,
                                    uint64_t out_base = ~0ull) {
    if (out_base == ~0ull) out_base = s0;
    __shared__ uint32_t q[kSelThreads];          // q[j+1] = meeting candidate of S_j, S_{j+1}
    __shared__ uint32_t x[kSelThreads + 1];      // x[j] = where T joins S_j
    __shared__ uint64_t warp_tot[kSelThreads / 32];
    __shared__ uint32_t sc[kSelStage];           // staged candidates
    const int t = threadIdx.x;
    const uint64_t base = m ? __ldg(C) : 0;
    const bool staged = m <= kSelStage && (m == 0 || __ldg(C + m - 1) - base < (1ull << 32));
    if (staged) {
        for (uint32_t i = t; i < m; i += blockDim.x) sc[i] = (uint32_t)(__ldg(C + i) - base);
        __syncthreads();
        select_block_run(CandsShared{sc, base}, m, s0, n, mn, mx, ends, cap, d_count, L, out_base, q,
                         x, warp_tot);
    } else {
        select_block_run(CandsGlobal{C}, m, s0, n, mn, mx, ends, cap, d_count, L, out_base, q, x,
                         warp_tot);
    }
}

// First window end p in [plo, phi] whose bit is set, by one thread (UINT64_MAX
// if none). Used only when the candidate list overflowed its capacity.
__device__ __forceinline__ uint64_t first_bit_thread(const uint32_t *__restrict__ bitmap,
                                                     uint64_t plo, uint64_t phi) {
    for (uint64_t wi = plo / 32; wi <= phi / 32; wi++) {
        uint32_t w = bitmap[wi];
        if (wi == plo / 32) w &= ~0u << (plo % 32);
        if (wi == phi / 32 && (phi % 32) != 31) w &= (1u << (phi % 32 + 1)) - 1u;
        if (w) return wi * 32 + (__ffs(w) - 1);
    }
    return UINT64_MAX;
}

// Greedy selection of the stream [s0, n) by one thread from the bitmap (bits
// known up to window end L - 1); returns the last cut emitted (s0 if none).
template <class Emit>
__device__ uint64_t select_thread_bitmap(const uint32_t *__restrict__ bitmap, uint64_t s0,
                                         uint64_t n, uint64_t mn, uint64_t mx, Emit emit,
                                         uint64_t L = ~0ull) {
    uint64_t s = s0;
    while (s < n) {
        const uint64_t lo = s + mn, hi = min(min(s + mx, n), L);
        uint64_t cut;
        const uint64_t p = lo <= hi ? first_bit_thread(bitmap, lo - 1, hi - 1) : UINT64_MAX;
        if (p != UINT64_MAX) cut = p + 1;
        else if (s + mx > L && L < n) break;               // undecided until more is known
        else if (s + mx < n) cut = s + mx;
        else cut = n;
        emit(cut);
        s = cut;
    }
    return s;
}

}  // namespace hg
