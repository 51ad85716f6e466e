// dedisp_tile.cuh -- the dedispersion block-tile shared by the per-range
// kernels (k_dedisp.cu) and the batched persistent kernel (k_batch.cu).
//
// Computes, for one DM range (paper Sec. "Dedispersion"; SB formation of
// Sec. "Hierarchical beam forming"),
//     S[s][i][t] = sum_c X[sb_map[s][c]][c][t + d[i][c]],   t < n_out,
// with exact integer sums, and accumulates per-series sum S and sum S^2 for
// the S/N stage.
//
// Design (B300): the work is shift-and-add, not a contraction, so no tensor
// cores.  Every channel-add needs its input byte from shared memory, so the
// LDS bandwidth and the integer issue rate are the limits.  To approach them:
//   * A block owns BD = WARPS*DPW consecutive DM trials and T output samples
//     of one SB.  Channels are streamed in stages of CC.  For each channel the
//     input bytes covering [t0 + min_i d, t0 + max_i d + T) of the TAB the SB
//     selects (the gather only picks the source row) are staged in shared
//     memory as 4/E copies, copy q shifted by q*E bytes, so every trial's
//     4-byte word is one aligned, conflict-free LDS.32 whatever its delay.
//   * Staging is software-pipelined: the global loads of stage k+1 are issued
//     into registers before stage k is computed and written to shared memory
//     after it, so L2 latency hides behind the adds.
//   * SWAR accumulation for uint8 samples: acc_a += x (mod 2^32) and acc_b +=
//     bytes 1,3 of x in 16-bit lanes (one PRMT); bytes 0,2 are recovered as
//     acc_a - (acc_b << 8).  Lanes hold <= 256 channels of 255 and are folded
//     into int32 totals every 256 channels.  uint16 samples (downsampled
//     ranges) use acc_a += x, acc_b += x >> 16, exact without folding.
//     Channels are taken in groups of four: every accumulator update is one
//     IADD3 over two channels, the group's loads are all issued before its
//     adds, and the next group's offsets are fetched ahead.
//   * Per-trial staged offsets come from a host table laid out
//     [DM block][channel][trial], so a stage's offsets are one coalesced read.
#pragma once

#include "fdd_internal.cuh"

namespace fdd {
namespace detail {

template <int N>
__device__ __forceinline__ void load_offsets(const int32_t* p, int32_t (&o)[N]) {
    if constexpr (N == 1) {
        o[0] = p[0];
    } else if constexpr (N == 2) {
        const int2 v = *reinterpret_cast<const int2*>(p);
        o[0] = v.x;
        o[1] = v.y;
    } else {
        static_assert(N == 4, "DPW must be 1, 2 or 4");
        const int4 v = *reinterpret_cast<const int4*>(p);
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    }
}

// 32-bit shared-window load (keeps address arithmetic in 32 bits).
__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

// One block-tile of dedispersion: DM block `blk` (BD trials), time tile
// `tile_x` (T output samples) of SB `sb`.  Must be called by all WARPS*32
// threads of the block; uses the block's dynamic shared memory
// (dedisp_smem_bytes(v, a.Lw, a.CC)) and ends with no shared-memory reads
// pending, so a caller may run tiles back to back after a __syncthreads().
template <int E, int NW, int DPW, int WARPS, int MAXIT>
__device__ __forceinline__ void dedisp_tile(const DedispArgs& a, int tile_x, int blk, int sb) {
    constexpr int NC = 4 / E;       // byte-shifted copies of each staged row
    constexpr int SPW = 4 / E;      // samples per 32-bit word
    constexpr int BD = WARPS * DPW; // DM trials per block
    constexpr int T = 32 * NW * SPW;
    constexpr int NT = WARPS * 32;
    static_assert(BD % 4 == 0, "BD must be a multiple of 4");
    extern __shared__ __align__(16) uint8_t smem[];

    const int CC = a.CC;
    const int Lw = a.Lw;
    const int chunks = Lw >> 2;  // 16-byte chunks per copy row
    const int slot_bytes = NC * Lw * 4;
    uint8_t* s_rows = smem;
    int32_t* s_off = reinterpret_cast<int32_t*>(smem + CC * slot_bytes);  // [CC][BD]

    const int t0 = tile_x * T;
    const int i0 = blk * BD;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t limit = a.n_valid * E;  // valid bytes per input row
    const int16_t* sbm = a.sb_map + (int64_t)sb * a.n_chan;
    const int32_t* base_blk = a.base + (int64_t)blk * a.n_chan;
    const uint8_t* in_blk = a.in + (a.blk_per_coarse > 0 ? (int64_t)(blk / a.blk_per_coarse) * a.coarse_stride : 0);
    const int32_t* off_blk = a.off + (int64_t)blk * a.n_chan * BD;

    // ---- staging registers (one stage in flight)
    uint4 pv[MAXIT];
    uint32_t pn[MAXIT];
    int4 po = make_int4(0, 0, 0, 0);

    auto stage_load = [&](int c0, int ncc) {
        const int items = ncc * chunks;
#pragma unroll
        for (int u = 0; u < MAXIT; u++) {
            const int it = threadIdx.x + u * NT;
            if (it < items) {
                const int cc = it / chunks;
                const int m = it - cc * chunks;
                const int c = c0 + cc;
                const uint8_t* row = in_blk + ((int64_t)sbm[c] * a.n_chan + c) * a.pitch_bytes;
                const int64_t b0 = (int64_t)(t0 + base_blk[c]) * E + 16 * (int64_t)m;
                if (b0 + 20 <= limit) {
                    pv[u] = __ldg(reinterpret_cast<const uint4*>(row + b0));
                    pn[u] = __ldg(reinterpret_cast<const uint32_t*>(row + b0 + 16));
                } else {
                    uint32_t g[5];
#pragma unroll
                    for (int k = 0; k < 5; k++) {
                        uint32_t w = 0;
#pragma unroll
                        for (int b = 0; b < 4; b++) {
                            const int64_t p = b0 + 4 * k + b;
                            w |= ((p < limit) ? (uint32_t)row[p] : 0u) << (8 * b);
                        }
                        g[k] = w;
                    }
                    pv[u] = make_uint4(g[0], g[1], g[2], g[3]);
                    pn[u] = g[4];
                }
            }
        }
        if (threadIdx.x < ncc * (BD / 4))
            po = __ldg(reinterpret_cast<const int4*>(off_blk + (int64_t)c0 * BD) + threadIdx.x);
    };

    auto stage_store = [&](int ncc) {
        const int items = ncc * chunks;
#pragma unroll
        for (int u = 0; u < MAXIT; u++) {
            const int it = threadIdx.x + u * NT;
            if (it < items) {
                const int cc = it / chunks;
                const int m = it - cc * chunks;
                uint8_t* dst = s_rows + cc * slot_bytes + 16 * m;
                const uint32_t g0 = pv[u].x, g1 = pv[u].y, g2 = pv[u].z, g3 = pv[u].w, g4 = pn[u];
#pragma unroll
                for (int q = 0; q < NC; q++) {
                    uint4 o;
                    o.x = __funnelshift_r(g0, g1, 8 * q * E);
                    o.y = __funnelshift_r(g1, g2, 8 * q * E);
                    o.z = __funnelshift_r(g2, g3, 8 * q * E);
                    o.w = __funnelshift_r(g3, g4, 8 * q * E);
                    *reinterpret_cast<uint4*>(dst + q * Lw * 4) = o;
                }
            }
        }
        if (threadIdx.x < ncc * (BD / 4)) {
            const int cc = (threadIdx.x * 4) / BD;
            const int add = cc * slot_bytes;
            reinterpret_cast<int4*>(s_off)[threadIdx.x] =
                make_int4(po.x + add, po.y + add, po.z + add, po.w + add);
        }
    };

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

    // E == 1: fold the 16-bit SWAR lanes into the int32 totals.
    auto flush = [&]() {
        if constexpr (E == 1) {
#pragma unroll
            for (int j = 0; j < DPW; j++)
#pragma unroll
                for (int k = 0; k < NW; k++) {
                    const uint32_t odd = acc_b[j][k];                // bytes 1,3
                    const uint32_t even = acc_a[j][k] - (odd << 8);  // bytes 0,2
                    tot[j][k][0] += even & 0xFFFFu;
                    tot[j][k][1] += odd & 0xFFFFu;
                    tot[j][k][2] += even >> 16;
                    tot[j][k][3] += odd >> 16;
                    acc_a[j][k] = 0u;
                    acc_b[j][k] = 0u;
                }
        }
    };
    auto split = [](uint32_t x) -> uint32_t {
        if constexpr (E == 1)
            return __byte_perm(x, 0u, 0x4341);  // bytes 1,3 -> 16-bit lanes
        else
            return x >> 16;                     // high uint16 sample
    };

    const uint32_t s_lane32 = static_cast<uint32_t>(__cvta_generic_to_shared(s_rows)) + 4u * lane;
    const int32_t* s_off_w = s_off + warp * DPW;

    int ncc = min(CC, a.n_chan);
    stage_load(0, ncc);
    stage_store(ncc);
    __syncthreads();

    int since_flush = 0;
    for (int c0 = 0; c0 < a.n_chan; c0 += CC) {
        const int c1 = c0 + CC;
        const int ncc_next = (c1 < a.n_chan) ? min(CC, a.n_chan - c1) : 0;
        if (ncc_next) stage_load(c1, ncc_next);  // in flight during the adds below

        if constexpr (E == 1) {
            if (since_flush + ncc > 256) {
                flush();
                since_flush = 0;
            }
            since_flush += ncc;
        }
        // Channels in groups of four: offsets of the next group are fetched
        // before this group's 4*DPW*NW loads, and all loads of a group are
        // issued before its adds, so LDS latency overlaps within a warp.
        int cc = 0;
        int32_t og[4][DPW];
        if (ncc >= 4) {
#pragma unroll
            for (int u = 0; u < 4; u++) load_offsets<DPW>(s_off_w + u * BD, og[u]);
        }
#pragma unroll 1
        for (; cc + 3 < ncc; cc += 4) {
            int32_t on[4][DPW];
            const bool more = cc + 7 < ncc;
            if (more) {
#pragma unroll
                for (int u = 0; u < 4; u++) load_offsets<DPW>(s_off_w + (cc + 4 + u) * BD, on[u]);
            }
            uint32_t x[4][DPW][NW];
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int j = 0; j < DPW; j++) {
                    const uint32_t ad = s_lane32 + static_cast<uint32_t>(og[u][j]);
#pragma unroll
                    for (int k = 0; k < NW; k++) x[u][j][k] = lds32(ad + 128u * k);
                }
#pragma unroll
            for (int j = 0; j < DPW; j++)
#pragma unroll
                for (int k = 0; k < NW; k++) {
                    acc_a[j][k] = acc_a[j][k] + x[0][j][k] + x[1][j][k];
                    acc_b[j][k] = acc_b[j][k] + split(x[0][j][k]) + split(x[1][j][k]);
                    acc_a[j][k] = acc_a[j][k] + x[2][j][k] + x[3][j][k];
                    acc_b[j][k] = acc_b[j][k] + split(x[2][j][k]) + split(x[3][j][k]);
                }
            if (more) {
#pragma unroll
                for (int u = 0; u < 4; u++)
#pragma unroll
                    for (int j = 0; j < DPW; j++) og[u][j] = on[u][j];
            }
        }
#pragma unroll 1
        for (; cc < ncc; cc++) {  // remainder (n_chan not a multiple of 4)
            int32_t o0[DPW];
            load_offsets<DPW>(s_off_w + cc * BD, o0);
#pragma unroll
            for (int j = 0; j < DPW; j++)
#pragma unroll
                for (int k = 0; k < NW; k++) {
                    const uint32_t x0 = lds32(s_lane32 + static_cast<uint32_t>(o0[j]) + 128u * k);
                    acc_a[j][k] += x0;
                    acc_b[j][k] += split(x0);
                }
        }
        __syncthreads();  // stage fully consumed
        if (ncc_next) {
            stage_store(ncc_next);
            __syncthreads();
        }
        ncc = ncc_next;
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
                if (t < a.n_emit) {
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

}  // namespace detail
}  // namespace fdd
