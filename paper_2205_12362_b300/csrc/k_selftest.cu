// k_selftest.cu -- self-test of the bounded mbarrier wait (tma.cuh) that the
// TMA-staged kernels use: one block initialises an mbarrier that nothing
// ever arrives on and waits for it with a small poll limit.  The wait must
// give up and the block must return normally, reporting that it did; no
// copy is issued, so nothing is left in flight.
#include "fdd_plan_impl.h"
#include "tma.cuh"

namespace fdd {
namespace {

__global__ void k_wait_selftest(int limit, int32_t* gave_up) {
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = static_cast<uint32_t>(__cvta_generic_to_shared(&bar));
    if (threadIdx.x == 0) {
        tma::mbar_init(b, 1);
        tma::mbar_init_fence();
    }
    __syncthreads();
    const bool ok = tma::mbar_wait_bounded(b, 0u, limit);  // phase 0 never completes
    if (__syncthreads_or(!ok) && threadIdx.x == 0) *gave_up = 1;
}

}  // namespace
}  // namespace fdd

extern "C" int fdd_selftest_bounded_wait(int32_t polls, int32_t* gave_up) {
    if (!gave_up || polls < 1 || polls > fdd::tma::kSpinLimit) return fdd::host::fail(FDD_ERR_INVALID_ARG, "bad argument");
    int32_t* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(int32_t));
    if (e != cudaSuccess) return fdd::host::cuda_fail(e, "cudaMalloc(self-test flag)");
    int32_t h = 0;
    if ((e = cudaMemset(d, 0, sizeof(int32_t))) == cudaSuccess) {
        fdd::k_wait_selftest<<<1, 64>>>(polls, d);
        if ((e = cudaGetLastError()) == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int32_t), cudaMemcpyDeviceToHost);
    }
    cudaFree(d);
    if (e != cudaSuccess) return fdd::host::cuda_fail(e, "bounded-wait self-test");
    *gave_up = h;
    return FDD_OK;
}
