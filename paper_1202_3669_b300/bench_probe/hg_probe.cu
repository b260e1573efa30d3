// Integer-pipe throughput probe (a measurement tool of the benchmark, built
// into its own library, libhgprobe.so, not into the hashing library): the
// measured denominators of the integer rooflines. Each thread runs 8
// independent chains of one operation class for `iters` rounds, so the SM's
// integer pipes, not dependency latency, set the rate; the caller times the
// launch and divides operations by time x SMs x clock. Classes: 3-input logic
// (lop3), 3-input add, funnel shift, the MD5 operation mix (logic, 3-input
// add, rotate, add), and an add written as a multiply-add by a run-time 1
// (the FMA-pipe add of the split hash steps).
#include <cstdint>
#include <cuda_runtime.h>

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
__device__ __forceinline__ uint32_t op_mad1(uint32_t a, uint32_t one, uint32_t c) {
    uint32_t r;
    asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(one), "r"(c));
    return r;
}
__device__ __forceinline__ uint32_t op_shf(uint32_t a, uint32_t b) {
    uint32_t r;
    asm volatile("shf.l.wrap.b32 %0, %1, %2, 7;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

// ops per chain per round: 1 (lop3, add3 counted as one 3-input add, shf,
// multiply-add by 1) or 4 (the MD5 mix: logic, 3-input add, rotate, add)
template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) k_int_probe(uint32_t iters, uint32_t seed,
                                                             uint32_t one, uint32_t *sink) {
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
            else if (KIND == 4) a[j] = op_mad1(a[j], one, b);
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

__device__ uint32_t g_sink[4];

}  // namespace
}  // namespace hg

using namespace hg;

extern "C" int hgp_probe_int_pipe(int device, int kind, uint32_t iters, uint32_t ctas_per_sm,
                                  uint64_t *ops_out, void *stream) {
    if (kind < 0 || kind > 4 || iters == 0 || ctas_per_sm == 0 || ctas_per_sm > 8 || !ops_out)
        return -1;
    int prev = 0, sms = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    uint32_t *sink = nullptr;
    cudaGetSymbolAddress((void **)&sink, g_sink);
    const unsigned grid = (unsigned)sms * ctas_per_sm;
    cudaStream_t s = (cudaStream_t)stream;
    switch (kind) {
        case 0: k_int_probe<0><<<grid, kProbeThreads, 0, s>>>(iters, 0x1234567u, 1u, sink); break;
        case 1: k_int_probe<1><<<grid, kProbeThreads, 0, s>>>(iters, 0x1234567u, 1u, sink); break;
        case 2: k_int_probe<2><<<grid, kProbeThreads, 0, s>>>(iters, 0x1234567u, 1u, sink); break;
        case 3: k_int_probe<3><<<grid, kProbeThreads, 0, s>>>(iters, 0x1234567u, 1u, sink); break;
        default: k_int_probe<4><<<grid, kProbeThreads, 0, s>>>(iters, 0x1234567u, 1u, sink); break;
    }
    const int r = cudaGetLastError() == cudaSuccess ? 0 : -5;
    cudaSetDevice(prev);
    *ops_out = (uint64_t)grid * kProbeThreads * kChains * iters * (kind == 3 ? 4u : 1u);
    return r;
}
