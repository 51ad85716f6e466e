// tma.cuh -- mbarrier and TMA tensor-copy helpers (inline PTX, sm_100+).
//
// A kernel stages a tile with one cp.async.bulk.tensor per box, completion
// counted in bytes on an mbarrier (arrive.expect_tx by the issuing thread).
// Every wait is bounded: mbar_wait_bounded gives up after kSpinLimit polls
// (about a second with the back-off), so a copy that never lands ends in an
// error status the host can read instead of a hung GPU.
#pragma once

#include <cstdint>
#include <cuda.h>

namespace fdd {
namespace tma {

constexpr int kSpinLimit = 1 << 22;  // polls of one wait; each after the first 64 sleeps ~256 ns

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// Make barrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0u;
}
// Wait for phase `parity` of the barrier to complete; false if `limit` polls pass first.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int limit = kSpinLimit) {
    for (int it = 0; it < limit; it++) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it >= 64) __nanosleep(256);
    }
    return false;
}
__device__ __forceinline__ void load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void load_4d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, int w,
                                        uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
        : "memory");
}

}  // namespace tma
}  // namespace fdd
