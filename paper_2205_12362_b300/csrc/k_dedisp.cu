// k_dedisp.cu -- fused synthesized-beam gather + brute-force dedispersion.
//
// Computes, for one DM range (paper Sec. "Dedispersion"; SB formation of
// Sec. "Hierarchical beam forming"),
//     S[s][i][t] = sum_c X[sb_map[s][c]][c][t + d[i][c]],   t < n_out,
// with exact integer sums, and accumulates per-series sum S and sum S^2 for
// the S/N stage.
//
// Design (B300): the work is shift-and-add, not a contraction, so no tensor
// cores.  Every output costs one byte read from shared memory and one add;
// both the LDS bandwidth and the integer pipe are the limits.  To reach them:
//   * A block owns BD = WARPS*DPW consecutive DM trials and T output samples
//     of one SB.  Channels are streamed in stages of CC; for each channel the
//     input bytes covering [t0 + min_i d, t0 + max_i d + T) of the TAB that
//     the SB selects (the gather is free: it only picks the source row) are
//     staged in shared memory in 4/E copies, copy q shifted by q*E bytes, so
//     that every trial's 4-byte word is an aligned LDS.32 whatever its delay.
//   * A warp reads 32 consecutive words per (trial, channel): conflict-free.
//   * SWAR accumulation for uint8 samples: acc_all += x (mod 2^32) and
//     acc_odd += bytes 1,3 of x in 16-bit lanes.  Bytes 0,2 are recovered as
//     acc_all - (acc_odd << 8).  Lanes hold <= 256 channels of 255, so they
//     are flushed into int32 totals every 256 channels.  For uint16 samples
//     (downsampled ranges) acc_all += x and acc_hi += x >> 16 are exact
//     without flushing.  That is 2 integer ops per 4 (or 2) channel-adds.
//   * Per-trial staged offsets (copy, word) are precomputed on the host into
//     a table, so the inner loop is LDS + PRMT/SHF + IADD only.
#include "fdd_internal.cuh"

namespace fdd {

namespace {

// Staged row layout in shared memory, per channel slot:
//   copy q (q < NC) occupies Lw words; word j of copy q holds the 4 bytes at
//   byte offset 4*j + q*E of the global row segment starting at the block's
//   aligned base sample.
template <int E>
__device__ __forceinline__ void stage_channels(const DedispArgs& a, uint8_t* s_rows, int slot_bytes,
                                               int c0, int ncc, int sb, int blk, int t0) {
    constexpr int NC = 4 / E;
    const int chunks = a.Lw >> 2;  // 16-byte chunks per copy row
    const int items = ncc * chunks;
    const int64_t limit = a.n_valid * E;  // valid bytes per row
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int cc = it / chunks;
        const int m = it - cc * chunks;
        const int c = c0 + cc;
        const int tab = a.sb_map[(int64_t)sb * a.n_chan + c];
        const uint8_t* row = a.in + ((int64_t)tab * a.n_chan + c) * a.pitch_bytes;
        const int64_t b0 = (int64_t)(t0 + a.base[(int64_t)blk * a.n_chan + c]) * E + 16 * (int64_t)m;
        uint32_t g[5];
        if (b0 + 20 <= limit) {
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(row + b0));
            g[0] = v.x; g[1] = v.y; g[2] = v.z; g[3] = v.w;
            g[4] = __ldg(reinterpret_cast<const uint32_t*>(row + b0 + 16));
        } else {
#pragma unroll
            for (int k = 0; k < 5; k++) {
                uint32_t w = 0;
#pragma unroll
                for (int b = 0; b < 4; b++) {
                    const int64_t p = b0 + 4 * k + b;
                    const uint32_t byte = (p < limit) ? (uint32_t)row[p] : 0u;
                    w |= byte << (8 * b);
                }
                g[k] = w;
            }
        }
        uint8_t* dst = s_rows + cc * slot_bytes + 16 * m;
#pragma unroll
        for (int q = 0; q < NC; q++) {
            uint4 o;
            o.x = __funnelshift_r(g[0], g[1], 8 * q * E);
            o.y = __funnelshift_r(g[1], g[2], 8 * q * E);
            o.z = __funnelshift_r(g[2], g[3], 8 * q * E);
            o.w = __funnelshift_r(g[3], g[4], 8 * q * E);
            *reinterpret_cast<uint4*>(dst + q * a.Lw * 4) = o;
        }
    }
}

template <int E, int NW, int DPW, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_dedisp(const DedispArgs a) {
    constexpr int NC = 4 / E;
    constexpr int SPW = 4 / E;
    constexpr int BD = WARPS * DPW;
    constexpr int T = 32 * NW * SPW;
    extern __shared__ __align__(16) uint8_t smem[];

    const int CC = a.CC;
    const int slot_bytes = NC * a.Lw * 4;
    uint8_t* s_rows = smem;
    int32_t* s_off = reinterpret_cast<int32_t*>(smem + CC * slot_bytes);  // [CC][BD]

    const int tile = blockIdx.x, blk = blockIdx.y, sb = blockIdx.z;
    const int t0 = tile * T;
    const int i0 = blk * BD;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    uint32_t acc_a[DPW][NW], acc_b[DPW][NW];
    uint32_t tot[DPW][NW][SPW];
#pragma unroll
    for (int j = 0; j < DPW; j++)
#pragma unroll
        for (int k = 0; k < NW; k++) {
            acc_a[j][k] = 0u;
            acc_b[j][k] = 0u;
#pragma unroll
            for (int e = 0; e < SPW; e++) tot[j][k][e] = 0u;
        }

    // E == 1: fold the 16-bit SWAR lanes into the int32 totals (must happen
    // before a lane holds more than 257 channels of <= 255).
    auto flush = [&]() {
        if constexpr (E == 1) {
#pragma unroll
            for (int j = 0; j < DPW; j++)
#pragma unroll
                for (int k = 0; k < NW; k++) {
                    const uint32_t odd = acc_b[j][k];                  // bytes 1,3
                    const uint32_t even = acc_a[j][k] - (odd << 8);    // bytes 0,2
                    tot[j][k][0] += even & 0xFFFFu;
                    tot[j][k][1] += odd & 0xFFFFu;
                    tot[j][k][2] += even >> 16;
                    tot[j][k][3] += odd >> 16;
                    acc_a[j][k] = 0u;
                    acc_b[j][k] = 0u;
                }
        }
    };

    const uint8_t* s_lane = s_rows + 4 * lane;
    int since_flush = 0;  // channels held in the 16-bit lanes (E == 1)
    for (int c0 = 0; c0 < a.n_chan; c0 += CC) {
        const int ncc = min(CC, a.n_chan - c0);
        __syncthreads();  // previous stage fully consumed
        stage_channels<E>(a, s_rows, slot_bytes, c0, ncc, sb, blk, t0);
        for (int idx = threadIdx.x; idx < ncc * BD; idx += blockDim.x) {
            const int cc = idx / BD, jj = idx - cc * BD;
            const int i = min(i0 + jj, a.n_dm - 1);
            s_off[idx] = a.off[(int64_t)i * a.n_chan + c0 + cc] + cc * slot_bytes;
        }
        __syncthreads();

        if (E == 1) {
            if (since_flush + ncc > 256) {
                flush();
                since_flush = 0;
            }
            since_flush += ncc;
        }
#pragma unroll 2
        for (int cc = 0; cc < ncc; cc++) {
            const uint32_t* p[DPW];
#pragma unroll
            for (int j = 0; j < DPW; j++)
                p[j] = reinterpret_cast<const uint32_t*>(s_lane + s_off[cc * BD + warp * DPW + j]);
#pragma unroll
            for (int j = 0; j < DPW; j++)
#pragma unroll
                for (int k = 0; k < NW; k++) {
                    const uint32_t x = p[j][32 * k];
                    acc_a[j][k] += x;
                    if constexpr (E == 1)
                        acc_b[j][k] += __byte_perm(x, 0u, 0x4341);  // bytes 1,3 -> 16-bit lanes
                    else
                        acc_b[j][k] += x >> 16;                     // high uint16 sample
                }
        }
    }
    if constexpr (E == 1) {
        flush();
    } else {
#pragma unroll
        for (int j = 0; j < DPW; j++)
#pragma unroll
            for (int k = 0; k < NW; k++) {
                tot[j][k][1] = acc_b[j][k];
                tot[j][k][0] = acc_a[j][k] - (acc_b[j][k] << 16);
            }
    }

    // Epilogue: write the series and fold per-series moments.
#pragma unroll
    for (int j = 0; j < DPW; j++) {
        const int i = i0 + warp * DPW + j;
        if (i >= a.n_dm) continue;  // warp-uniform
        const int64_t q = (int64_t)sb * a.n_dm + i;
        int32_t* row = a.series + q * a.n_out;
        long long s1 = 0;
        unsigned long long s2 = 0;
#pragma unroll
        for (int k = 0; k < NW; k++)
#pragma unroll
            for (int e = 0; e < SPW; e++) {
                const int t = t0 + (lane + 32 * k) * SPW + e;
                if (t < a.n_out) {
                    const uint32_t v = tot[j][k][e];
                    row[t] = static_cast<int32_t>(v);
                    s1 += v;
                    s2 += static_cast<unsigned long long>(v) * v;
                }
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) {
            atomicAdd(a.stat + 2 * q, static_cast<unsigned long long>(s1));
            atomicAdd(a.stat + 2 * q + 1, s2);
        }
    }
}

using KernelFn = void (*)(const DedispArgs);

struct Entry {
    DedispVariant v;
    KernelFn fn;
};

#define FDD_V(E, NW, DPW, WARPS) {{E, NW, DPW, WARPS}, k_dedisp<E, NW, DPW, WARPS>}
const Entry kEntries[] = {
    FDD_V(1, 4, 2, 8),  FDD_V(1, 4, 2, 16), FDD_V(1, 4, 4, 8), FDD_V(1, 8, 1, 16), FDD_V(1, 8, 2, 8),
    FDD_V(1, 2, 4, 8),
    FDD_V(2, 4, 2, 8),  FDD_V(2, 4, 2, 16), FDD_V(2, 4, 4, 8), FDD_V(2, 8, 2, 8),  FDD_V(2, 8, 1, 16),
};
#undef FDD_V

}  // namespace

int num_dedisp_variants() { return static_cast<int>(sizeof(kEntries) / sizeof(kEntries[0])); }

const DedispVariant& dedisp_variant(int idx) { return kEntries[idx].v; }

size_t dedisp_smem_bytes(const DedispVariant& v, int Lw, int CC) {
    return static_cast<size_t>(CC) * (4 / v.E) * Lw * 4 + static_cast<size_t>(CC) * v.bd() * 4;
}

cudaError_t launch_dedisp(int variant, const DedispArgs& a, cudaStream_t s) {
    const Entry& e = kEntries[variant];
    const size_t smem = dedisp_smem_bytes(e.v, a.Lw, a.CC);
    cudaError_t err = cudaFuncSetAttribute(e.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    const int T = e.v.tile(), BD = e.v.bd();
    dim3 grid((a.n_out + T - 1) / T, (a.n_dm + BD - 1) / BD, a.n_sb);
    e.fn<<<grid, e.v.threads(), smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace fdd
