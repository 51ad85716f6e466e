// downsample_chunk.cuh -- 8-output chunk of the time downsampler, shared by
// the per-plan launch (k_downsample.cu) and the batched launch (k_batch.cu).
// out[j] = sum_{k<D} in[j*D + k] for j in [j0, min(j0 + 8, n_y)), exact uint16;
// `in` may start at any byte (windows whose bins are aligned to the stream).
#pragma once

#include "fdd_internal.cuh"

namespace fdd {
namespace detail {

// Sums of 8 consecutive bins of D bytes held in 2*D little-endian words.
template <int D>
__device__ __forceinline__ void sum8_words(const uint32_t* w, uint16_t* dst) {
    uint32_t s[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        uint32_t acc = 0;
#pragma unroll
        for (int k = 0; k < D; k++) {
            const int b = j * D + k;
            acc += (w[b >> 2] >> (8 * (b & 3))) & 0xFFu;
        }
        s[j] = acc;
    }
    uint4 o;
    o.x = s[0] | (s[1] << 16);
    o.y = s[2] | (s[3] << 16);
    o.z = s[4] | (s[5] << 16);
    o.w = s[6] | (s[7] << 16);
    *reinterpret_cast<uint4*>(dst) = o;
}

// src 16-byte aligned (8-byte for D = 1): vector loads.
template <int D>
__device__ __forceinline__ void sum8_vec(const uint8_t* src, uint16_t* dst) {
    uint32_t w[2 * D];
    if constexpr (D == 1) {
        const uint2 v = *reinterpret_cast<const uint2*>(src);
        w[0] = v.x;
        w[1] = v.y;
    } else {
#pragma unroll
        for (int v = 0; v < D / 2; v++) {
            const uint4 x = *reinterpret_cast<const uint4*>(src + 16 * v);
            w[4 * v + 0] = x.x; w[4 * v + 1] = x.y; w[4 * v + 2] = x.z; w[4 * v + 3] = x.w;
        }
    }
    sum8_words<D>(w, dst);
}

// src at any byte address (the bins of a window start at a phase inside a
// row): aligned 32-bit loads of the words covering the 8*D bytes, funnel-
// shifted by the misalignment.  The extra word is read only when the bytes
// reach into it, so no byte past the last needed word is touched.
template <int D>
__device__ __forceinline__ void sum8_shifted(const uint8_t* src, uint16_t* dst) {
    const uintptr_t addr = reinterpret_cast<uintptr_t>(src);
    const uint32_t* wp = reinterpret_cast<const uint32_t*>(addr & ~static_cast<uintptr_t>(3));
    const uint32_t sh = 8u * static_cast<uint32_t>(addr & 3u);
    uint32_t raw[2 * D + 1];
#pragma unroll
    for (int k = 0; k < 2 * D; k++) raw[k] = wp[k];
    raw[2 * D] = sh ? wp[2 * D] : 0u;
    uint32_t w[2 * D];
#pragma unroll
    for (int k = 0; k < 2 * D; k++) w[k] = __funnelshift_r(raw[k], raw[k + 1], sh);
    sum8_words<D>(w, dst);
}

// Chunk [j0, j0+8) of one row; vector path for D in {1, 2, 4, 8, 16} when the
// chunk is complete, scalar otherwise.
__device__ __forceinline__ void downsample_chunk(const uint8_t* __restrict__ src, uint16_t* __restrict__ dst,
                                                 int64_t n_y, int D, int64_t j0) {
    if (j0 + 8 <= n_y) {
        if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
            switch (D) {
                case 1: sum8_vec<1>(src + j0, dst + j0); return;
                case 2: sum8_vec<2>(src + j0 * 2, dst + j0); return;
                case 4: sum8_vec<4>(src + j0 * 4, dst + j0); return;
                case 8: sum8_vec<8>(src + j0 * 8, dst + j0); return;
                case 16: sum8_vec<16>(src + j0 * 16, dst + j0); return;
                default: break;
            }
        } else {
            switch (D) {
                case 1: sum8_shifted<1>(src + j0, dst + j0); return;
                case 2: sum8_shifted<2>(src + j0 * 2, dst + j0); return;
                case 4: sum8_shifted<4>(src + j0 * 4, dst + j0); return;
                case 8: sum8_shifted<8>(src + j0 * 8, dst + j0); return;
                case 16: sum8_shifted<16>(src + j0 * 16, dst + j0); return;
                default: break;
            }
        }
    }
    const int64_t jn = min(j0 + 8, n_y);
    for (int64_t j = j0; j < jn; j++) {
        uint32_t acc = 0;
        for (int k = 0; k < D; k++) acc += src[j * D + k];
        dst[j] = static_cast<uint16_t>(acc);
    }
}

}  // namespace detail
}  // namespace fdd
