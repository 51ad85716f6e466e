// boxcar_series.cuh -- per-series statistics, boxcar S/N and ballot
// compaction, shared by the per-range kernel (k_boxcar.cu) and the batched
// kernel (k_batch.cu).
//
// Paper Sec. "Integration": each dedispersed series is convolved with boxcars
// of the user's widths; Sec. "S/N evaluation": S/N of every sample of the
// integrated series; Sec. "Candidate selection": keep what exceeds the
// threshold.  The S/N method is left open by the paper; this library uses
//     snr(t, w) = (B_w(t) - w * mu) / (sigma * sqrt(w)),
//     B_w(t) = sum_{k<w} S[t + k],  t in [0, n - w],
// with mu, sigma the mean and population standard deviation of the series.
//
// Numerics: mu and sigma come from the exact integer moments accumulated by
// the dedispersion kernel (sum S and sum S^2), finalised in FP64 with a
// 128-bit integer numerator n*sum S^2 - (sum S)^2.  Box sums are exact:
// S is centred on m0 = round(mu) and prefix-summed in wrapping uint32, so
// B_w(t) - w*m0 = P[t+w] - P[t] exactly.  Only the final
// (Bc - w*(mu - m0)) * 1/(sigma sqrt(w)) is FP32.
//
// One block per series; tiles of 4096 outputs plus a (wmax-1) halo are
// staged in shared memory and prefix-summed with warp shuffles.  Every
// (t, w) is first tested in integers, Bc > tau_w, with tau_w a bound a little
// below the exact threshold crossing (thr / scale_w + offs_w, lowered by a
// margin far larger than FP32 rounding), so almost every sample costs one
// shared load, one subtraction and one compare per width.  Only warps where
// some lane passes evaluate the FP32 S/N -- the same expression as always --
// and the exact snr > thr, so the candidates are unchanged by the filter.
// Lanes of a warp hold consecutive t for one width, so __ballot_sync + __popc
// give each warp one atomicAdd on the global counter per width with any
// candidate.
#pragma once

#include "fdd_internal.cuh"

namespace fdd {
namespace detail {

constexpr int kThreads = 256;
constexpr int kTile = 4096;
constexpr int kMaxSeg = (kTile + FDD_MAX_WIDTH - 1 + kThreads - 1) / kThreads;  // 20

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < kThreads / 32) ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kThreads / 32) s_warp[lane] = wi - w;  // exclusive warp offsets
        if (lane == kThreads / 32 - 1) *total = wi;
    }
    __syncthreads();
    return s_warp[warp] + incl - v;
}

// Statistics, boxcar S/N and compaction of series q (0 <= q < n_sb*n_dm) of
// one DM range.  Called by all kThreads threads of a block; uses
// boxcar_smem_bytes(a.wmax) of dynamic shared memory.
__device__ __forceinline__ void boxcar_series(const BoxcarArgs& a, const int64_t q) {
    extern __shared__ uint32_t sP[];  // exclusive prefix sums, seg*kThreads + 1 entries
    __shared__ float s_scale[FDD_MAX_WIDTHS];
    __shared__ float s_offs[FDD_MAX_WIDTHS];
    __shared__ int32_t s_tau[FDD_MAX_WIDTHS];  // integer pre-filter: Bc <= tau never exceeds thr
    __shared__ int32_t s_m0;
    __shared__ int32_t s_ok;
    __shared__ uint32_t s_warp[kThreads / 32];
    __shared__ uint32_t s_total;

    const int n = a.n_emit;  // samples searched; rows are a.n_out apart
    if (threadIdx.x == 0) {
        const long long sum = static_cast<long long>(a.stat[2 * q]);
        const unsigned long long sq = a.stat[2 * q + 1];
        const __int128 num = (__int128)n * (__int128)sq - (__int128)sum * (__int128)sum;
        const int ok = (n > 0) && (num > 0);
        s_ok = ok;
        if (ok) {
            const double mu = (double)sum / (double)n;
            const double var = (double)num / ((double)n * (double)n);
            const double sigma = sqrt(var);
            const long long m0 = llrint(mu);
            const double delta = mu - (double)m0;
            s_m0 = static_cast<int32_t>(m0);
            for (int k = 0; k < a.n_width; k++) {
                const double w = (double)a.widths[k];
                s_scale[k] = (float)(1.0 / (sigma * sqrt(w)));
                s_offs[k] = (float)(w * delta);
                // exact crossing thr * sigma * sqrt(w) + w * delta, lowered by 1e-5 relative + 2
                const double cross = (double)a.thr * sigma * sqrt(w) + w * delta;
                const double lo = floor(cross - (1e-5 * fabs(cross) + 2.0));
                s_tau[k] = lo < -2147483647.0 ? -2147483647 : (lo > 2147483646.0 ? 2147483646 : (int32_t)lo);
            }
        }
    }
    __syncthreads();
    if (!s_ok) return;

    const int s = static_cast<int>(q / a.n_dm), i = static_cast<int>(q % a.n_dm);
    const int32_t* S = a.series + q * a.n_out;
    const int32_t m0 = s_m0;
    const int seg = (kTile + a.wmax - 1 + kThreads - 1) / kThreads;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;

    for (int t0 = 0; t0 < n; t0 += kTile) {
        const int need = min(kTile + a.wmax - 1, n - t0);  // centred samples this tile can use
        uint32_t loc[kMaxSeg];
        uint32_t tsum = 0;
        const int start = threadIdx.x * seg;
#pragma unroll
        for (int k = 0; k < kMaxSeg; k++) {
            uint32_t v = 0;
            if (k < seg && start + k < need) v = static_cast<uint32_t>(S[t0 + start + k] - m0);
            loc[k] = v;
            tsum += v;
        }
        uint32_t run = block_exclusive_scan(tsum, s_warp, &s_total);
#pragma unroll
        for (int k = 0; k < kMaxSeg; k++) {
            if (k < seg) {
                sP[start + k] = run;
                run += loc[k];
            }
        }
        if (threadIdx.x == 0) sP[seg * kThreads] = s_total;
        __syncthreads();

        const int nw = a.n_width;
#pragma unroll 1
        for (int e = 0; e < kTile / kThreads; e++) {
            const int tl = e * kThreads + threadIdx.x;
            const int t = t0 + tl;
            if (t0 + e * kThreads >= n) break;  // block-uniform
            // integer pre-filter over every width
            bool any = false;
            if (t < n) {
                const uint32_t p0 = sP[tl];
                for (int wi = 0; wi < nw; wi++) {
                    const int w = a.widths[wi];
                    if (t + w <= n) any |= static_cast<int32_t>(sP[tl + w] - p0) > s_tau[wi];
                }
            }
            if (!__any_sync(0xffffffffu, any)) continue;
            for (int wi = 0; wi < nw; wi++) {
                const int w = a.widths[wi];
                bool pred = false;
                float snr = 0.f;
                if (t + w <= n) {
                    const int32_t bc = static_cast<int32_t>(sP[tl + w] - sP[tl]);
                    snr = (static_cast<float>(bc) - s_offs[wi]) * s_scale[wi];
                    pred = snr > a.thr;
                }
                const unsigned mask = __ballot_sync(0xffffffffu, pred);
                if (mask) {
                    const int leader = __ffs(mask) - 1;
                    unsigned long long base = 0;
                    if (lane == leader) base = atomicAdd(a.count, static_cast<unsigned long long>(__popc(mask)));
                    base = __shfl_sync(0xffffffffu, base, leader);
                    if (pred) {
                        const unsigned long long idx = base + __popc(mask & lt_mask);
                        if (idx < static_cast<unsigned long long>(a.cap)) {
                            fdd_candidate c;
                            c.sb = s;
                            c.dm_index = a.dm_index0 + i;
                            c.downsamp = a.D;
                            c.width_native = w * a.D;
                            c.t_native = static_cast<int64_t>(t) * a.D + a.t_offset;
                            c.dm = static_cast<float>(a.dm0 + static_cast<double>(i) * a.ddm);
                            c.snr = snr;
                            a.cands[idx] = c;
                        }
                    }
                }
            }
        }
        __syncthreads();  // sP reused by the next tile
    }
}

inline size_t boxcar_smem_bytes(int wmax) {
    const int seg = (kTile + wmax - 1 + kThreads - 1) / kThreads;
    return (static_cast<size_t>(seg) * kThreads + 1) * sizeof(uint32_t);
}

}  // namespace detail
}  // namespace fdd
