// Integer-pipe throughput probe: the measured denominator of the integer
// rooflines. Each thread runs 8 independent chains of one operation class for
// `iters` rounds, so the SM's integer pipes, not dependency latency, set the
// rate; the caller times the launch and divides operations by time x SMs x
// clock. Classes: 3-input logic (lop3), 3-input add, funnel shift, and the
// MD5 operation mix (logic, 3-input add, rotate, add) the hashes are made of.
#include "hg_internal.h"

namespace hg {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

__device__ __forceinline__ uint32_t op_lop3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t r;
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}
__device__ __forceinline__ uint32_t op_add3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t r;
    asm volatile("{\n\t.reg .u32 t;\n\tadd.u32 t, %1, %2;\n\tadd.u32 %0, t, %3;\n\t}"
                 : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}
__device__ __forceinline__ uint32_t op_shf(uint32_t a, uint32_t b) {
    uint32_t r;
    asm volatile("shf.l.wrap.b32 %0, %1, %2, 7;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

// ops per chain per round: 1 (lop3, add3 counted as one 3-input add, shf) or
// 4 (the MD5 mix: logic, 3-input add, rotate, add)
template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) k_int_probe(uint32_t iters, uint32_t seed,
                                                             uint32_t *sink) {
    uint32_t a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; j++) a[j] = seed * (threadIdx.x + 1) + (uint32_t)j * 0x9e3779b9u;
    const uint32_t k = seed ^ 0x5a827999u;
    for (uint32_t i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < kChains; j++) {
            const uint32_t b = a[(j + 1) % kChains];
            if (KIND == 0) a[j] = op_lop3(a[j], b, k);
            else if (KIND == 1) a[j] = op_add3(a[j], b, k);
            else if (KIND == 2) a[j] = op_shf(a[j], b);
            else {
                const uint32_t f = op_lop3(b, a[j], k);
                const uint32_t t = op_add3(a[j], f, k);
                a[j] = op_shf(t, t) + b;
            }
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int j = 0; j < kChains; j++) x ^= a[j];
    if (x == 0x12345678u) sink[0] = x;           // keeps the work observable
}

}  // namespace
}  // namespace hg

using namespace hg;

extern "C" int hg_probe_int_pipe(hg_ctx *ctx, int kind, uint32_t iters, uint32_t ctas_per_sm,
                                 uint64_t *ops_out, void *stream) {
    if (!ctx || kind < 0 || kind > 3 || iters == 0 || ctas_per_sm == 0 || ctas_per_sm > 8 || !ops_out)
        return HG_EINVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    const unsigned grid = (unsigned)ctx->num_sms * ctas_per_sm;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *sink = reinterpret_cast<uint32_t *>(ctx->d_err) + 8;   // unused words of the error block
    switch (kind) {
        case 0: k_int_probe<0><<<grid, kProbeThreads, 0, s>>>(iters, 0x1234567u, sink); break;
        case 1: k_int_probe<1><<<grid, kProbeThreads, 0, s>>>(iters, 0x1234567u, sink); break;
        case 2: k_int_probe<2><<<grid, kProbeThreads, 0, s>>>(iters, 0x1234567u, sink); break;
        default: k_int_probe<3><<<grid, kProbeThreads, 0, s>>>(iters, 0x1234567u, sink); break;
    }
    const int r = cuda_status(cudaGetLastError());
    cudaSetDevice(prev);
    *ops_out = (uint64_t)grid * kProbeThreads * kChains * iters * (kind == 3 ? 4u : 1u);
    return r;
}
