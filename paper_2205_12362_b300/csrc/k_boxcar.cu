// k_boxcar.cu -- per-range launch of the S/N stage: one block per series
// running boxcar_series (see boxcar_series.cuh for the method and numerics).
#include "boxcar_series.cuh"

namespace fdd {

namespace {

__global__ void __launch_bounds__(detail::kThreads) k_boxcar(const BoxcarArgs a) {
    detail::boxcar_series(a, blockIdx.x);
}

}  // namespace

cudaError_t launch_boxcar(const BoxcarArgs& a, cudaStream_t s) {
    if (a.n_sb == 0 || a.n_dm == 0 || a.n_out == 0) return cudaSuccess;
    const size_t smem = detail::boxcar_smem_bytes(a.wmax);
    const long long blocks = static_cast<long long>(a.n_sb) * a.n_dm;
    k_boxcar<<<static_cast<unsigned>(blocks), detail::kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace fdd
