// k_boxcar.cu -- per-range launch of the S/N stage: one warp per series
// (boxcar_warp.cuh) when every width fits its 512-sample chunks, otherwise
// one block per series (boxcar_series.cuh); both use the same method and
// numerics.
#include "boxcar_series.cuh"
#include "boxcar_warp.cuh"

namespace fdd {

namespace {

__global__ void __launch_bounds__(detail::kThreads) k_boxcar(const BoxcarArgs a) {
    detail::boxcar_series(a, blockIdx.x);
}

template <int NWB>
__global__ void __launch_bounds__(detail::kBoxWarps * 32) k_boxcar_warp(const __grid_constant__ BoxcarArgs a) {
    __shared__ uint32_t ring[detail::kBoxWarps][detail::kWarpRing];
    const int warp = threadIdx.x >> 5;
    const int64_t q = static_cast<int64_t>(blockIdx.x) * detail::kBoxWarps + warp;
    if (q >= static_cast<int64_t>(a.n_sb) * a.n_dm) return;  // warp-uniform
    const int i = static_cast<int>(q % a.n_dm);
    detail::BoxSeries v;
    v.S = a.series + q * a.n_out;
    v.stat = a.stat + 2 * q;
    v.widths = a.widths;
    v.cands = a.cands;
    v.count = a.count;
    v.cap = a.cap;
    v.t_offset = a.t_offset;
    v.dm = a.dm0 + static_cast<double>(i) * a.ddm;
    v.n = a.n_emit;
    v.n_width = a.n_width;
    v.sb = static_cast<int>(q / a.n_dm);
    v.dm_index = a.dm_index0 + i;
    v.D = a.D;
    v.thr = a.thr;
    detail::boxcar_series_warp<NWB>(v, ring[warp]);
}

}  // namespace

cudaError_t launch_boxcar(const BoxcarArgs& a, cudaStream_t s) {
    if (a.n_sb == 0 || a.n_dm == 0 || a.n_emit <= 0) return cudaSuccess;
    const long long series = static_cast<long long>(a.n_sb) * a.n_dm;
    if (a.wmax <= detail::kWarpCS) {
        const unsigned blocks = static_cast<unsigned>((series + detail::kBoxWarps - 1) / detail::kBoxWarps);
        if (a.n_width <= 4)
            k_boxcar_warp<4><<<blocks, detail::kBoxWarps * 32, 0, s>>>(a);
        else if (a.n_width <= 8)
            k_boxcar_warp<8><<<blocks, detail::kBoxWarps * 32, 0, s>>>(a);
        else
            k_boxcar_warp<16><<<blocks, detail::kBoxWarps * 32, 0, s>>>(a);
        return cudaGetLastError();
    }
    const size_t smem = detail::boxcar_smem_bytes(a.wmax);
    k_boxcar<<<static_cast<unsigned>(series), detail::kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace fdd
