// Pinned host buffer pool owned by a context: hg_alloc_pinned / hg_free_pinned.
//
// Sec. 3.1 ("One-copy host to device data transfers", "Hiding memory
// allocation overheads"): data the application places in page-locked host
// memory crosses the host link in one DMA copy, and page-locked buffers are
// costly to allocate, so they are allocated once and reused. Sec. 3.2.3: the
// runtime's memory-management module keeps such buffers and hands them out
// again; Sec. 3.2.4: the storage system obtains its buffers through the
// library's allocation call. This pool keeps freed buffers in size classes
// (four per power of two, 64 KiB and up) and serves later requests of a class
// from them without a new host allocation; new allocations count against a
// host budget, and free buffers are released (largest first) when a new one
// would exceed it.
#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "hg_internal.h"

namespace hg {

struct PinnedPool {
    std::mutex mu;
    uint64_t budget = kPinnedDefaultBudget;
    uint64_t held = 0, in_use = 0, host_allocs = 0, reuses = 0;
    std::map<uint64_t, std::vector<void *>> free_lists;       // class bytes -> free buffers
    std::unordered_map<void *, uint64_t> owned;               // every buffer -> its class
    std::unordered_map<void *, bool> busy;                    // handed out and not freed
};

// Size class of a request: 64 KiB, else the next of 2^k * {1, 1.25, 1.5, 1.75}
// at or above it (at most a quarter wasted).
uint64_t pinned_class(uint64_t n) {
    const uint64_t kMin = 64ull << 10;
    if (n <= kMin) return kMin;
    uint64_t p = 1;
    while (p * 2 < n) p *= 2;                                  // p < n <= 2p
    const uint64_t step = p / 4;
    return p + (n - p + step - 1) / step * step;
}

namespace {

// Release free buffers, largest first, until `need` more bytes fit the budget
// (or all free buffers are gone). Caller holds the lock.
void trim_locked(PinnedPool *pp, uint64_t need) {
    while (pp->held + need > pp->budget && !pp->free_lists.empty()) {
        auto it = std::prev(pp->free_lists.end());
        if (it->second.empty()) {
            pp->free_lists.erase(it);
            continue;
        }
        void *p = it->second.back();
        it->second.pop_back();
        cudaFreeHost(p);
        pp->owned.erase(p);
        pp->busy.erase(p);
        pp->held -= it->first;
        if (it->second.empty()) pp->free_lists.erase(it);
    }
}

PinnedPool *pool_of(hg_ctx *c) {
    std::lock_guard<std::mutex> lock(c->pinned_mu);
    if (!c->pinned) c->pinned = new (std::nothrow) PinnedPool();
    return c->pinned;
}

// The pool if it exists (read under the same lock that guards its creation).
PinnedPool *existing_pool(hg_ctx *c) {
    std::lock_guard<std::mutex> lock(c->pinned_mu);
    return c->pinned;
}

}  // namespace

void pinned_destroy(hg_ctx *c) {
    PinnedPool *pp = c->pinned;
    if (!pp) return;
    for (auto &kv : pp->owned) cudaFreeHost(kv.first);
    delete pp;
    c->pinned = nullptr;
}

}  // namespace hg

using namespace hg;

extern "C" {

void *hg_alloc_pinned(hg_ctx *c, size_t bytes) {
    if (!c || bytes == 0) return nullptr;
    PinnedPool *pp = pool_of(c);
    if (!pp) return nullptr;
    const uint64_t cls = pinned_class(bytes);
    std::lock_guard<std::mutex> lock(pp->mu);
    // reuse: the smallest free class that holds the request, up to twice its class
    for (auto it = pp->free_lists.lower_bound(cls); it != pp->free_lists.end() && it->first <= 2 * cls;
         ++it) {
        if (it->second.empty()) continue;
        void *p = it->second.back();
        it->second.pop_back();
        pp->busy[p] = true;
        pp->in_use += it->first;
        pp->reuses++;
        return p;
    }
    trim_locked(pp, cls);
    if (pp->held + cls > pp->budget) return nullptr;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->device) cudaSetDevice(c->device);
    void *p = nullptr;
    const cudaError_t e = cudaHostAlloc(&p, cls, cudaHostAllocPortable | cudaHostAllocMapped);
    if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return nullptr;
    }
    pp->owned[p] = cls;
    pp->busy[p] = true;
    pp->held += cls;
    pp->in_use += cls;
    pp->host_allocs++;
    return p;
}

int hg_free_pinned(hg_ctx *c, void *p) {
    if (!c || !p) return HG_EINVAL;
    PinnedPool *pp = existing_pool(c);
    if (!pp) return HG_EINVAL;
    std::lock_guard<std::mutex> lock(pp->mu);
    auto o = pp->owned.find(p);
    auto b = pp->busy.find(p);
    if (o == pp->owned.end() || b == pp->busy.end() || !b->second) return HG_EINVAL;
    b->second = false;
    pp->in_use -= o->second;
    pp->free_lists[o->second].push_back(p);
    trim_locked(pp, 0);                 // a lowered budget is honoured as buffers come back
    return HG_OK;
}

int hg_pinned_set_budget(hg_ctx *c, uint64_t bytes) {
    if (!c) return HG_EINVAL;
    PinnedPool *pp = pool_of(c);
    if (!pp) return HG_ENOMEM;
    std::lock_guard<std::mutex> lock(pp->mu);
    pp->budget = bytes ? bytes : kPinnedDefaultBudget;
    trim_locked(pp, 0);
    return HG_OK;
}

int hg_pinned_trim(hg_ctx *c) {
    if (!c) return HG_EINVAL;
    PinnedPool *pp = existing_pool(c);
    if (!pp) return HG_OK;
    std::lock_guard<std::mutex> lock(pp->mu);
    const uint64_t keep = pp->budget;
    pp->budget = 0;
    trim_locked(pp, 0);
    pp->budget = keep;
    return HG_OK;
}

int hg_pinned_stats(hg_ctx *c, hg_pinned_info *out) {
    if (!c || !out) return HG_EINVAL;
    *out = hg_pinned_info{};
    PinnedPool *pp = existing_pool(c);
    out->budget_bytes = pp ? pp->budget : kPinnedDefaultBudget;
    if (!pp) return HG_OK;
    std::lock_guard<std::mutex> lock(pp->mu);
    out->held_bytes = pp->held;
    out->in_use_bytes = pp->in_use;
    out->host_allocs = pp->host_allocs;
    out->reuses = pp->reuses;
    out->buffers = pp->owned.size();
    return HG_OK;
}

uint64_t hg_pinned_class(uint64_t bytes) { return bytes ? pinned_class(bytes) : 0; }

}  // extern "C"
