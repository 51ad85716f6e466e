// k_probe.cu -- issue-rate probes that measure the denominators of the
// dedispersion roofline on the running GPU: integer adds per second, ALU-pipe
// byte permutes per second, and shared-memory load bandwidth.
//
// Dedispersion here is shift-and-add on integers (Sec. "Dedispersion"); its
// kernels are bound by integer issue and by shared-memory reads, not by HBM
// or tensor cores, so the roofline needs those two peaks.  Each probe runs
// many independent dependency chains per thread at full occupancy, so the
// measured rate is a throughput limit, not a latency.
//   kind 0: a = a + b + c chains (two 32-bit adds per operation; the compiler
//           forms three-input adds), counted as adds;
//   kind 1: byte-permute chains (an ALU-pipe-only operation), counted as
//           operations;
//   kind 2: conflict-free 32-bit shared-memory loads (one add each to keep
//           them live), counted as bytes loaded;
//   kind 3: chains of a = a * b + c (32-bit multiply-add, the FMA pipe's
//           integer operation), counted as adds (one per operation);
//   kind 4: three-input add chains and multiply-add chains interleaved one to
//           one, counted as adds (two and one per operation): the add rate
//           of the ALU and FMA pipes together.
#include "fdd_plan_impl.h"

namespace fdd {
namespace {

constexpr int kChains = 16;
constexpr int kRepeat = 4;  // chain rounds per loop iteration (keeps the loop counter's share small)

__global__ void __launch_bounds__(256) k_probe_add(int64_t iters, uint32_t seed, uint32_t* sink) {
    uint32_t a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = seed * (threadIdx.x + 1u) + static_cast<uint32_t>(k) * 0x9E3779B9u;
#pragma unroll 1
    for (int64_t it = 0; it < iters; it++) {
#pragma unroll
        for (int r = 0; r < kRepeat; r++)
#pragma unroll
            for (int k = 0; k < kChains; k++) a[k] = a[k] + a[(k + 1) % kChains] + a[(k + 5) % kChains];
    }
    uint32_t x = 0;
#pragma unroll
    for (int k = 0; k < kChains; k++) x ^= a[k];
    if (x == 0x12345678u) atomicXor(sink, x);  // keeps the chains live; practically never taken
}

__global__ void __launch_bounds__(256) k_probe_prmt(int64_t iters, uint32_t seed, uint32_t* sink) {
    uint32_t a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = seed * (threadIdx.x + 1u) + static_cast<uint32_t>(k) * 0x9E3779B9u;
    constexpr uint32_t sel[4] = {0x5410u, 0x7632u, 0x3276u, 0x1054u};
#pragma unroll 1
    for (int64_t it = 0; it < iters; it++) {
#pragma unroll
        for (int r = 0; r < kRepeat; r++)
#pragma unroll
            for (int k = 0; k < kChains; k++) a[k] = __byte_perm(a[k], a[(k + 1) % kChains], sel[(k + r) & 3]);
    }
    uint32_t x = 0;
#pragma unroll
    for (int k = 0; k < kChains; k++) x ^= a[k];
    if (x == 0x12345678u) atomicXor(sink, x);
}

__global__ void __launch_bounds__(256) k_probe_lds(int64_t iters, uint32_t seed, uint32_t* sink) {
    __shared__ uint32_t buf[32 * 32];
    for (int k = threadIdx.x; k < 32 * 32; k += blockDim.x) buf[k] = seed ^ static_cast<uint32_t>(k);
    __syncthreads();
    const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(buf)) + 4u * (threadIdx.x & 31u);
    uint32_t acc[4] = {0u, 0u, 0u, 0u};
#pragma unroll 1
    for (int64_t it = 0; it < iters; it++) {
        const uint32_t row = static_cast<uint32_t>(it) & 7u;
#pragma unroll
        for (int k = 0; k < 8 * kRepeat; k++) {
            uint32_t v;
            // lanes read consecutive words of one 128-byte row (no bank conflicts); the 32 loads of an
            // iteration read 32 different rows, so none can be merged with another
            asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(base + 128u * ((row + k) & 31u)));
            acc[k & 3] += v;
        }
    }
    const uint32_t x = acc[0] ^ acc[1] ^ acc[2] ^ acc[3];
    if (x == 0x12345678u) atomicXor(sink, x);
}

__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__global__ void __launch_bounds__(256) k_probe_imad(int64_t iters, uint32_t seed, uint32_t* sink) {
    uint32_t a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = seed * (threadIdx.x + 1u) + static_cast<uint32_t>(k) * 0x9E3779B9u;
    const uint32_t m = seed | 1u;  // a run-time odd multiplier
#pragma unroll 1
    for (int64_t it = 0; it < iters; it++) {
#pragma unroll
        for (int r = 0; r < kRepeat; r++)
#pragma unroll
            for (int k = 0; k < kChains; k++) a[k] = imad(a[k], m, a[(k + 1) % kChains]);
    }
    uint32_t x = 0;
#pragma unroll
    for (int k = 0; k < kChains; k++) x ^= a[k];
    if (x == 0x12345678u) atomicXor(sink, x);
}

__global__ void __launch_bounds__(256) k_probe_mix(int64_t iters, uint32_t seed, uint32_t* sink) {
    uint32_t a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = seed * (threadIdx.x + 1u) + static_cast<uint32_t>(k) * 0x9E3779B9u;
    const uint32_t m = seed | 1u;
#pragma unroll 1
    for (int64_t it = 0; it < iters; it++) {
#pragma unroll
        for (int r = 0; r < kRepeat; r++)
#pragma unroll
            for (int k = 0; k < kChains; k++)
                a[k] = (k & 1) ? imad(a[k], m, a[(k + 1) % kChains])
                               : a[k] + a[(k + 1) % kChains] + a[(k + 5) % kChains];
    }
    uint32_t x = 0;
#pragma unroll
    for (int k = 0; k < kChains; k++) x ^= a[k];
    if (x == 0x12345678u) atomicXor(sink, x);
}

}  // namespace
}  // namespace fdd

extern "C" int fdd_probe_issue_rate(int32_t kind, int32_t blocks_per_sm, int64_t iters, double* per_second,
                                    float* ms, int32_t* n_sm) {
    using fdd::host::cuda_fail;
    using fdd::host::fail;
    if (kind < 0 || kind > 4 || blocks_per_sm < 1 || blocks_per_sm > 8 || iters < 1 || iters > (int64_t(1) << 30) ||
        !per_second || !ms)
        return fail(FDD_ERR_INVALID_ARG, "bad probe argument");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    uint32_t* sink = nullptr;
    if ((e = cudaMalloc(&sink, sizeof(uint32_t))) != cudaSuccess) return cuda_fail(e, "cudaMalloc(probe sink)");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int threads = 256;
    const dim3 grid(static_cast<unsigned>(sms * blocks_per_sm));
    auto launch = [&](int64_t n) {
        switch (kind) {
            case 0: fdd::k_probe_add<<<grid, threads>>>(n, 0x2545F491u, sink); break;
            case 1: fdd::k_probe_prmt<<<grid, threads>>>(n, 0x2545F491u, sink); break;
            case 2: fdd::k_probe_lds<<<grid, threads>>>(n, 0x2545F491u, sink); break;
            case 3: fdd::k_probe_imad<<<grid, threads>>>(n, 0x2545F491u, sink); break;
            default: fdd::k_probe_mix<<<grid, threads>>>(n, 0x2545F491u, sink); break;
        }
    };
    launch(iters / 8 + 1);  // warm-up (clocks, module load)
    cudaEventRecord(e0);
    launch(iters);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return cuda_fail(e, "issue-rate probe");
    const double threads_total = static_cast<double>(grid.x) * threads;
    // per loop iteration and thread: kind 0 kRepeat x 16 three-input adds (2 adds each); kind 1
    // kRepeat x 16 permutes; kind 2 kRepeat x 8 loads of 4 bytes; kind 3 kRepeat x 16 multiply-adds
    // (1 add each); kind 4 kRepeat x (8 three-input adds + 8 multiply-adds)
    const double per_iter = kind == 0   ? 2.0 * fdd::kChains * fdd::kRepeat
                            : kind == 1 ? 1.0 * fdd::kChains * fdd::kRepeat
                            : kind == 2 ? 8.0 * fdd::kRepeat * 4.0
                            : kind == 3 ? 1.0 * fdd::kChains * fdd::kRepeat
                                        : 1.5 * fdd::kChains * fdd::kRepeat;
    *ms = t;
    *per_second = threads_total * static_cast<double>(iters) * per_iter / (static_cast<double>(t) * 1e-3);
    if (n_sm) *n_sm = sms;
    return FDD_OK;
}
