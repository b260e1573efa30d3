// Batch API: many files stored back to back in one device buffer, chunked and
// digested by one job (hg_job.cu) whose launches are captured into a CUDA
// graph on first use, with an autotuner for the job's launch shapes.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include <cstdio>
#include <string>

#include "hg_internal.h"

using namespace hg;

struct hg_batch {
    hg_ctx *ctx = nullptr;
    uint32_t nfile = 0;
    uint64_t total = 0;
    hg_cdc_params p{};
    JobHost host;
    char *mem = nullptr;
    size_t mem_bytes = 0;
    JobDev dev{};
    JobScratch sc{};
    hg_batch_tuning tune{};
    int win_max_per_sm = 8;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void *g_key[5] = {};
    hg_batch_tuning g_tune{};
};

static JobTuning to_job(const hg_batch_tuning &t) {
    return JobTuning{t.window_ctas_per_sm, t.hash_threads, t.hash_ctas_per_sm, t.long_chunk_bytes};
}

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" {

int hg_batch_create(hg_ctx *ctx, const uint64_t *h_file_off, uint32_t nfile,
                    const hg_cdc_params *p, hg_batch **out) {
    if (!ctx || !h_file_off || !p || !out || nfile == 0 || nfile >= (1u << 31)) return HG_EINVAL;
    *out = nullptr;
    if ((p->window_hash != HG_WIN_MD5 && p->window_hash != HG_WIN_RABIN) || p->window < 1 ||
        p->window > (p->window_hash == HG_WIN_RABIN ? 64u : 55u) || p->mask_bits < 1 ||
        p->mask_bits > 32 ||
        (p->mask_bits < 32 && (p->magic >> p->mask_bits)) || p->min_chunk < 1 ||
        p->min_chunk > p->max_chunk)
        return HG_EINVAL;
    if (h_file_off[0] != 0) return HG_EINVAL;
    std::vector<uint64_t> len(nfile);
    for (uint32_t f = 0; f < nfile; f++) {
        if (h_file_off[f + 1] < h_file_off[f]) return HG_EINVAL;
        len[f] = h_file_off[f + 1] - h_file_off[f];
    }
    hg_batch *b = new (std::nothrow) hg_batch();
    if (!b) return HG_ENOMEM;
    b->ctx = ctx;
    b->nfile = nfile;
    b->p = *p;
    b->total = h_file_off[nfile];
    job_plan(len.data(), nfile, p->min_chunk, &b->host);
    const JobHost &h = b->host;
    if (h.ntiles >= (1ull << 32)) { delete b; return HG_EUNSUPPORTED; }
    const uint64_t cand_cap = cand_capacity(b->total);
    const size_t arr = a256((nfile + 1) * 8) * 3 + a256((size_t)nfile * 4 + 4) * 2;
    const size_t scratch = job_scratch_bytes(h.ntiles, cand_cap, h.total_slots);
    b->mem_bytes = arr + scratch;
    if (ctx->held + b->mem_bytes > ctx->budget) { delete b; return HG_ENOMEM; }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    int rc = HG_OK;
    if (cudaMalloc(&b->mem, b->mem_bytes) != cudaSuccess) { cudaGetLastError(); rc = HG_ENOMEM; }
    if (rc == HG_OK) {
        ctx->held += b->mem_bytes;
        char *m = b->mem;
        uint64_t *d_fo = (uint64_t *)m;                     m += a256((nfile + 1) * 8);
        uint64_t *d_ts = (uint64_t *)m;                     m += a256((nfile + 1) * 8);
        uint64_t *d_so = (uint64_t *)m;                     m += a256((nfile + 1) * 8);
        uint32_t *d_small = (uint32_t *)m;                  m += a256((size_t)nfile * 4 + 4);
        uint32_t *d_big = (uint32_t *)m;                    m += a256((size_t)nfile * 4 + 4);
        job_scratch_carve(m, h.ntiles, cand_cap, h.total_slots, &b->sc);
        const size_t fo = (nfile + 1) * 8;
        if (cudaMemcpy(d_fo, h_file_off, fo, cudaMemcpyHostToDevice) ||
            cudaMemcpy(d_ts, h.tile_start.data(), fo, cudaMemcpyHostToDevice) ||
            cudaMemcpy(d_so, h.slot_off.data(), fo, cudaMemcpyHostToDevice) ||
            (!h.small.empty() && cudaMemcpy(d_small, h.small.data(), h.small.size() * 4, cudaMemcpyHostToDevice)) ||
            (!h.big.empty() && cudaMemcpy(d_big, h.big.data(), h.big.size() * 4, cudaMemcpyHostToDevice)) ||
            cudaMemset(b->sc.err, 0, 4) ||
            cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking))
            rc = HG_ECUDA;
        b->dev = JobDev{nullptr, d_fo, nullptr, nullptr, d_ts, d_so, d_small, d_big, nfile,
                        (uint32_t)h.small.size(), (uint32_t)h.big.size(), (uint32_t)h.ntiles};
    }
    if (rc == HG_OK) {
        b->win_max_per_sm = job_window_occupancy(p->window);
        b->tune.window_ctas_per_sm = 0;           // one-warp span CTAs (MD5 window)
        // one warp per scheduler: a SHA-1 warp alone saturates its scheduler's
        // ALU pipe, so long chains run fastest without neighbours
        b->tune.hash_threads = 32;
        b->tune.hash_ctas_per_sm = 4;
        b->tune.long_chunk_bytes = 16384;
    }
    cudaSetDevice(prev);
    if (rc != HG_OK) {
        if (b->mem) { cudaFree(b->mem); ctx->held -= b->mem_bytes; }
        if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
        delete b;
        return rc;
    }
    *out = b;
    return HG_OK;
}

int hg_batch_destroy(hg_batch *b) {
    if (!b) return HG_EINVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->ctx->device);
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->mem) { cudaFree(b->mem); b->ctx->held -= b->mem_bytes; }
    cudaSetDevice(prev);
    delete b;
    return HG_OK;
}

uint64_t hg_batch_slots(const hg_batch *b, uint64_t *h_slot_off) {
    if (!b) return 0;
    if (h_slot_off) std::memcpy(h_slot_off, b->host.slot_off.data(), (b->nfile + 1) * 8);
    return b->host.total_slots;
}

int hg_batch_get_tuning(const hg_batch *b, hg_batch_tuning *t) {
    if (!b || !t) return HG_EINVAL;
    *t = b->tune;
    return HG_OK;
}

int hg_batch_set_tuning(hg_batch *b, const hg_batch_tuning *t) {
    if (!b || !t || t->window_ctas_per_sm < 0 || t->hash_ctas_per_sm < 1 ||
        (t->hash_threads != 32 && t->hash_threads != 64 && t->hash_threads != 128 &&
         t->hash_threads != 256 && t->hash_threads != 512) || t->long_chunk_bytes == 0)
        return HG_EINVAL;
    b->tune = *t;
    if (b->tune.window_ctas_per_sm > b->win_max_per_sm) b->tune.window_ctas_per_sm = b->win_max_per_sm;
    return HG_OK;
}

int hg_batch_cdc_hash(hg_batch *b, int algo, const uint8_t *d_data, uint64_t *d_ends,
                      uint64_t *d_counts, uint8_t *d_digests, void *stream) {
    if (!b || (algo != HG_MD5 && algo != HG_SHA1)) return HG_EINVAL;
    if ((b->total && !d_data) || !d_counts || (b->host.total_slots && (!d_ends || !d_digests)) ||
        (reinterpret_cast<uintptr_t>(d_digests) & 3))
        return HG_EINVAL;
    JobDev j = b->dev;
    j.base = d_data ? d_data : reinterpret_cast<const uint8_t *>(b->mem);   // never read when empty
    return enqueue_cdc_job(j, b->sc, b->p, algo, to_job(b->tune), b->ctx->num_sms, d_ends,
                           d_counts, d_digests, (cudaStream_t)stream);
}

int hg_batch_cdc_hash_graph(hg_batch *b, int algo, const uint8_t *d_data, uint64_t *d_ends,
                            uint64_t *d_counts, uint8_t *d_digests, void *stream) {
    if (!b) return HG_EINVAL;
    const void *key[5] = {d_data, d_ends, d_counts, d_digests, (const void *)(uintptr_t)(algo + 1)};
    const bool same = b->exec && !std::memcmp(key, b->g_key, sizeof key) &&
                      !std::memcmp(&b->tune, &b->g_tune, sizeof b->tune);
    if (!same) {
        if (b->exec) {
            cudaStreamSynchronize((cudaStream_t)stream);
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return HG_ECUDA;
        int r = hg_batch_cdc_hash(b, algo, d_data, d_ends, d_counts, d_digests, b->cap_stream);
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
        if (r) { if (g) cudaGraphDestroy(g); return r; }
        if (e != cudaSuccess) { cudaGetLastError(); return HG_ECUDA; }
        e = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { cudaGetLastError(); b->exec = nullptr; return HG_ECUDA; }
        std::memcpy(b->g_key, key, sizeof key);
        b->g_tune = b->tune;
    }
    return cuda_status(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
}

int hg_batch_sync(hg_batch *b, void *stream) {
    if (!b) return HG_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return HG_ECUDA;
    }
    int err = 0;
    if (cudaMemcpy(&err, b->sc.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return HG_ECUDA;
    if (err) cudaMemset(b->sc.err, 0, sizeof(int));
    return err;
}

int hg_batch_autotune(hg_batch *b, int algo, const uint8_t *d_data, uint64_t *d_ends,
                      uint64_t *d_counts, uint8_t *d_digests, void *stream, hg_batch_tuning *best) {
    if (!b) return HG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) || cudaEventCreate(&e1)) return HG_ECUDA;
    // a candidate's time: the fastest of three runs after one untimed run
    auto time_it = [&](float *ms) -> int {
        int r = hg_batch_cdc_hash(b, algo, d_data, d_ends, d_counts, d_digests, stream);  // warm
        if (r) return r;
        float m = 1e30f;
        for (int k = 0; k < 3; k++) {
            cudaEventRecord(e0, s);
            if ((r = hg_batch_cdc_hash(b, algo, d_data, d_ends, d_counts, d_digests, stream))) return r;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) return HG_ECUDA;
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            m = std::min(m, t);
        }
        *ms = m;
        return HG_OK;
    };
    hg_batch_tuning cur = b->tune, top = cur;
    float best_ms = 1e30f;
    int rc = HG_OK;
    // window persistence first (the dominant kernel), then the chunk-hash shape. The
    // window forms are timed in two passes, each form keeping its faster time: the
    // first pass also brings the clocks up and loads every form's kernel (the forms
    // can be within 2-3 % of each other, and a form timed first from idle lost out).
    const int wm = b->win_max_per_sm;
    const int forms[4] = {0, wm, std::max(1, wm * 3 / 4), std::max(1, wm / 2)};
    float form_ms[4] = {1e30f, 1e30f, 1e30f, 1e30f};
    for (int pass = 0; pass < 2 && rc == HG_OK; pass++)
        for (int i = 0; i < 4; i++) {
            cur = top;
            cur.window_ctas_per_sm = forms[i];
            b->tune = cur;
            float ms;
            if ((rc = time_it(&ms))) break;
            form_ms[i] = std::min(form_ms[i], ms);
        }
    if (rc == HG_OK) {
        int bi = 0;
        for (int i = 1; i < 4; i++)
            if (form_ms[i] < form_ms[bi]) bi = i;
        top.window_ctas_per_sm = forms[bi];
        best_ms = form_ms[bi];
    }
    if (rc == HG_OK) {
        for (int ht : {32, 64, 128})
            for (int hc : {2, 4, 8})
                for (uint64_t lb : {8192ull, 32768ull}) {
                    cur = top;
                    cur.hash_threads = ht;
                    cur.hash_ctas_per_sm = hc;
                    cur.long_chunk_bytes = lb;
                    b->tune = cur;
                    float ms;
                    if ((rc = time_it(&ms))) break;
                    if (ms < best_ms) { best_ms = ms; top = cur; }
                }
    }
    b->tune = top;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best) *best = top;
    return rc;
}

}  // extern "C"

// Autotuner cache (JSON Lines): one line per tuned configuration,
//   {"key": {...}, "tuning": {...}}
// keyed by the GPU (name, SM count), the algorithm, the chunking parameters and
// the batch's shape (file count, log2 of its bytes, files of 1 MiB and up).
static std::string tune_key(const hg_batch *b, int algo) {
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, b->ctx->device);
    const uint32_t big = (uint32_t)b->host.big.size();     // files selected by a whole CTA
    int lg = 0;
    while ((2ull << lg) <= b->total) lg++;
    char buf[512];
    std::snprintf(buf, sizeof buf,
                  "{\"gpu\": \"%s\", \"sms\": %d, \"algo\": %d, \"window\": %u, \"mask_bits\": %u, "
                  "\"magic\": %u, \"window_hash\": %u, \"min_chunk\": %llu, \"max_chunk\": %llu, "
                  "\"nfile\": %u, \"bytes_log2\": %d, \"big_files\": %u}",
                  prop.name, prop.multiProcessorCount, algo, b->p.window, b->p.mask_bits, b->p.magic,
                  b->p.window_hash, (unsigned long long)b->p.min_chunk,
                  (unsigned long long)b->p.max_chunk, b->nfile, lg, big);
    return buf;
}

static bool tune_lookup(const char *path, const std::string &key, hg_batch_tuning *t) {
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[2048];
    const std::string want = "{\"key\": " + key + ", \"tuning\": ";
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        if (std::strncmp(line, want.c_str(), want.size()) != 0) continue;
        int w = 0, ht = 0, hc = 0;
        unsigned long long lb = 0;
        if (std::sscanf(line + want.size(),
                        "{\"window_ctas_per_sm\": %d, \"hash_threads\": %d, \"hash_ctas_per_sm\": %d, "
                        "\"long_chunk_bytes\": %llu}",
                        &w, &ht, &hc, &lb) == 4 &&
            w >= 0 && ht >= 32 && ht <= 512 && hc >= 1) {
            *t = hg_batch_tuning{w, ht, hc, 0, lb};
            found = true;               // the last matching line wins
        }
    }
    std::fclose(f);
    return found;
}

extern "C" {

int hg_batch_autotune_cached(hg_batch *b, int algo, const uint8_t *d_data, uint64_t *d_ends,
                             uint64_t *d_counts, uint8_t *d_digests, void *stream,
                             const char *cache_path, hg_batch_tuning *best, int *from_cache) {
    if (!b || !cache_path) return HG_EINVAL;
    if (from_cache) *from_cache = 0;
    const std::string key = tune_key(b, algo);
    hg_batch_tuning t{};
    if (tune_lookup(cache_path, key, &t)) {
        const int r = hg_batch_set_tuning(b, &t);
        if (r) return r;
        if (best) *best = t;
        if (from_cache) *from_cache = 1;
        return HG_OK;
    }
    const int r = hg_batch_autotune(b, algo, d_data, d_ends, d_counts, d_digests, stream, &t);
    if (r) return r;
    if (best) *best = t;
    FILE *f = std::fopen(cache_path, "a");
    if (!f) return HG_OK;               // tuned; the cache is only an optimisation
    std::fprintf(f,
                 "{\"key\": %s, \"tuning\": {\"window_ctas_per_sm\": %d, \"hash_threads\": %d, "
                 "\"hash_ctas_per_sm\": %d, \"long_chunk_bytes\": %llu}}\n",
                 key.c_str(), t.window_ctas_per_sm, t.hash_threads, t.hash_ctas_per_sm,
                 (unsigned long long)t.long_chunk_bytes);
    std::fclose(f);
    return HG_OK;
}

}  // extern "C"
