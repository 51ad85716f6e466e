// k_downsample.cu -- time downsampling of 8-bit filterbank rows.
//
// Paper Sec. "Downsampling": reduce the time resolution before dedispersion,
// used for high-DM ranges where intra-channel smearing already exceeds the
// native sampling time.  out[r][j] = sum_{k<D} in[r][j*D + k] for
// j < floor((n_in - offset) / D); exact uint16 sums (D <= 257), bins starting
// at input sample `offset` (0, or the phase of a window whose bins are aligned
// to its stream).  Done on the TABs, before the SB gather: gather and time sums
// commute, and there are fewer TAB rows than SB rows.
//
// HBM-bound: each thread reads 8*D consecutive bytes with 16-byte (or 8-byte
// for D = 1) vector loads and writes 8 uint16 with one 16-byte store; rows
// ride on gridDim.y.  Ragged tails and D not dividing 16 take a scalar path.
#include "downsample_chunk.cuh"

namespace fdd {

namespace {

template <int D>
__global__ void __launch_bounds__(256) k_downsample(const uint8_t* __restrict__ in, int64_t in_pitch, int64_t n_in,
                                                    int runtime_d, uint16_t* __restrict__ out, int64_t out_pitch,
                                                    int64_t offset) {
    const int64_t row = blockIdx.y;
    const int dd = (D > 0) ? D : runtime_d;
    const int64_t n_y = (n_in - offset) / dd;
    const int64_t j0 = 8 * (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x);
    if (j0 >= n_y) return;
    const uint8_t* src = in + row * in_pitch + offset;
    uint16_t* dst = out + row * out_pitch;
    if constexpr (D > 0) {
        if (j0 + 8 <= n_y) {
            if ((offset & 15) == 0)
                detail::sum8_vec<D>(src + j0 * D, dst + j0);
            else
                detail::sum8_shifted<D>(src + j0 * D, dst + j0);
            return;
        }
    }
    const int64_t jn = min(j0 + 8, n_y);
    for (int64_t j = j0; j < jn; j++) {
        uint32_t acc = 0;
        for (int k = 0; k < dd; k++) acc += src[j * dd + k];
        dst[j] = static_cast<uint16_t>(acc);
    }
}

}  // namespace

cudaError_t launch_downsample(const uint8_t* in, int64_t n_rows, int64_t n_in, int64_t in_pitch, int D,
                              uint16_t* out, int64_t out_pitch, cudaStream_t s, int64_t offset) {
    if (offset < 0 || offset > n_in) return cudaErrorInvalidValue;
    const int64_t n_y = (n_in - offset) / D;
    if (n_rows == 0 || n_y == 0) return cudaSuccess;
    const int threads = 256;
    const int64_t per_block = 8LL * threads;
    const int64_t kMaxRows = 65535;  // gridDim.y limit
    for (int64_t r0 = 0; r0 < n_rows; r0 += kMaxRows) {
        const int64_t nr = n_rows - r0 < kMaxRows ? n_rows - r0 : kMaxRows;
        const uint8_t* src = in + r0 * in_pitch;
        uint16_t* dst = out + r0 * out_pitch;
        dim3 grid(static_cast<unsigned>((n_y + per_block - 1) / per_block), static_cast<unsigned>(nr));
        switch (D) {
            case 1: k_downsample<1><<<grid, threads, 0, s>>>(src, in_pitch, n_in, D, dst, out_pitch, offset); break;
            case 2: k_downsample<2><<<grid, threads, 0, s>>>(src, in_pitch, n_in, D, dst, out_pitch, offset); break;
            case 4: k_downsample<4><<<grid, threads, 0, s>>>(src, in_pitch, n_in, D, dst, out_pitch, offset); break;
            case 8: k_downsample<8><<<grid, threads, 0, s>>>(src, in_pitch, n_in, D, dst, out_pitch, offset); break;
            case 16: k_downsample<16><<<grid, threads, 0, s>>>(src, in_pitch, n_in, D, dst, out_pitch, offset); break;
            default: k_downsample<0><<<grid, threads, 0, s>>>(src, in_pitch, n_in, D, dst, out_pitch, offset); break;
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace fdd
