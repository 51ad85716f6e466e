// boxcar_warp.cuh -- boxcar S/N and compaction with one WARP per series, no
// block barriers (used when every width is at most kWarpCS samples; the
// block-per-series form in boxcar_series.cuh serves wider boxcars).
//
// Same method and numerics as boxcar_series.cuh (paper Sec. "Integration",
// "S/N evaluation", "Candidate selection"): exact integer moments finalised
// in FP64, series centred on m0 = round(mu), wrapping-uint32 prefix sums so
// B_w(t) - w*m0 = P[t+w] - P[t] exactly, the integer pre-filter
// Bc > tau_w, and for survivors snr = (Bc - w*(mu - m0)) * 1/(sigma sqrt w)
// in FP32 against thr.
//
// Per warp, the series is walked in chunks of kWarpCS = 512 samples, lane l
// holding samples 32*m + l (m < 16) so every global load and shared access
// is coalesced / conflict-free.  The exclusive prefix of a chunk is one warp
// scan per row of 32 plus a running carry; it goes to slot c mod 3 of a
// per-warp shared ring (slot 0 is mirrored past slot 2 for the first wmax
// entries), and chunk c-1 is evaluated once chunk c is in, so P[t + w] for
// w <= 512 is always one contiguous read.
#pragma once

#include "fdd_internal.cuh"

namespace fdd {
namespace detail {

constexpr int kWarpCS = 512;                      // samples per chunk
constexpr int kWarpRows = kWarpCS / 32;           // rows of 32 per chunk
constexpr int kSlotWords = kWarpCS + kWarpCS / 32;  // one slot, one padding word per 32 entries
constexpr int kWarpRing = 4 * kSlotWords;            // three slots + mirror of slot 0, uint32 words
constexpr int kBoxWarps = 4;                      // warps (series) per block
constexpr int kBoundWmax = 128;                   // widest width of the chunk pre-check

constexpr int kBoundRows = kWarpRows + (kBoundWmax - 1 + 31) / 32;  // pre-check rows at most

// 32-bit shared load at a compile-time byte offset from a per-lane address.
template <int OFF>
__device__ __forceinline__ uint32_t lds_at(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(a), "n"(OFF));
    return v;
}

// Pre-check of a chunk, rows M .. rows-1: lane l of row m takes start j = 32 m + l, whose prefix
// entries j, j + 8 (and j + 64) sit at the lane's base addresses + 132 m bytes in the padded ring
// (entry J at word J + J / 32, and (32 m + l + k) / 32 = m + (l + k) / 32).  (The 1-sample maxima
// come from the samples themselves, in registers.)
template <int M, bool B64>
struct PrecheckRows {
    __device__ static __forceinline__ void run(uint32_t a0, uint32_t a8, uint32_t a64, int rows, int32_t& mx1,
                                               int32_t& mx2) {
        if constexpr (M < kBoundRows) {
            if (M >= kWarpRows && M >= rows) return;
            const uint32_t p0 = lds_at<132 * M>(a0);
            const uint32_t p8 = lds_at<132 * M>(a8);
            mx1 = max(mx1, static_cast<int32_t>(p8 - p0));
            if constexpr (B64) {
                const uint32_t p64 = lds_at<132 * M>(a64);
                mx2 = max(mx2, static_cast<int32_t>(p64 - p0));
            }
            PrecheckRows<M + 1, B64>::run(a0, a8, a64, rows, mx1, mx2);
        }
    }
};

// One series as the warp needs it.
struct BoxSeries {
    const int32_t* S;                    // [n]
    const unsigned long long* stat;      // [2]: sum S, sum S^2
    const int32_t* widths;               // [n_width]
    fdd_candidate* cands;
    unsigned long long* count;
    int64_t cap;
    int64_t t_offset;
    double dm;
    int32_t n, n_width, sb, dm_index, D;
    float thr;
};

// All 32 lanes of the warp call this with the same series; ring is the
// warp's kWarpRing-entry shared buffer.  NWB >= n_width (compile-time bound).
template <int NWB>
__device__ __forceinline__ void boxcar_series_warp(const BoxSeries& v, uint32_t* ring) {
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int n = v.n;

    // statistics on lane 0 (exact integer moments, FP64 finalisation)
    double mu = 0.0, sigma = 0.0;
    int ok = 0;
    if (lane == 0) {
        const long long sum = static_cast<long long>(v.stat[0]);
        const unsigned long long sq = v.stat[1];
        const __int128 num = (__int128)n * (__int128)sq - (__int128)sum * (__int128)sum;
        ok = (n > 0) && (num > 0);
        if (ok) {
            mu = (double)sum / (double)n;
            sigma = sqrt((double)num / ((double)n * (double)n));
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) return;
    mu = __shfl_sync(0xffffffffu, mu, 0);
    sigma = __shfl_sync(0xffffffffu, sigma, 0);
    const long long m0 = llrint(mu);
    const double delta = mu - (double)m0;
    // width k's constants on lane k
    int32_t w_l = 0, tau_l = 0x7fffffff;
    float scale_l = 0.f, offs_l = 0.f;
    if (lane < v.n_width) {
        w_l = v.widths[lane];
        const double w = (double)w_l;
        scale_l = (float)(1.0 / (sigma * sqrt(w)));
        offs_l = (float)(w * delta);
        // exact crossing thr * sigma * sqrt(w) + w * delta, lowered by 1e-5 relative + 2
        const double cross = (double)v.thr * sigma * sqrt(w) + w * delta;
        const double lo = floor(cross - (1e-5 * fabs(cross) + 2.0));
        tau_l = lo < -2147483647.0 ? -2147483647 : (lo > 2147483646.0 ? 2147483646 : (int32_t)lo);
    }
    int32_t wk[NWB], tk[NWB];
    uint32_t wb[NWB];  // byte offsets 4 * w
    int wmax = 0;
#pragma unroll
    for (int k = 0; k < NWB; k++) {
        wk[k] = __shfl_sync(0xffffffffu, w_l, k);
        tk[k] = __shfl_sync(0xffffffffu, tau_l, k);  // lanes >= n_width hold "never"
        wb[k] = 4u * static_cast<uint32_t>(wk[k]);
        wmax = max(wmax, wk[k]);
    }
    const uint32_t m0u = static_cast<uint32_t>(m0);
    const uint32_t negm0 = 0u - m0u, neg16m0 = 0u - 16u * m0u;
    // Virtual index vv = t + mis, mis = the row's misalignment in samples, so that chunk c
    // (vv in [512 c, 512 c + 512)) starts on a 16-byte boundary of the series and lane l's 16
    // consecutive samples vv = 512 c + 16 l + k come in as four aligned 16-byte loads.
    const int mis = static_cast<int>((reinterpret_cast<uintptr_t>(v.S) >> 2) & 3u);
    const int32_t* Sa = v.S - mis;  // 16-byte aligned; element vv is sample vv - mis
    const int nv = n + mis;          // prefix entries vv = 0 .. nv
    const int n_chunks = nv / kWarpCS + 1;
    const uint32_t ring_s = static_cast<uint32_t>(__cvta_generic_to_shared(ring));
    uint32_t carry = 0;
    // Chunk pre-check (widths <= kBoundWmax): for bases b in {1, 8, 64}, M_b >= max of B_b(s) over s in
    // [chunk start, chunk end + wmax - 1].  A width w with base b (the largest base dividing it) has
    // B_w(t) = sum_{j < w/b} B_b(t + j b) <= (w/b) M_b for every t of the chunk, so a chunk where
    // (w/b) M_b <= tau_w for every width holds no candidate and is skipped; any other chunk is
    // evaluated exactly below.
    const bool bound = wmax <= kBoundWmax;
    int32_t bmul[NWB];  // w / b
    int bsel[NWB];      // base index of width k
#pragma unroll
    for (int k = 0; k < NWB; k++) {
        const int w = wk[k];
        bsel[k] = (w >= 64 && w % 64 == 0) ? 2 : ((w >= 8 && w % 8 == 0) ? 1 : 0);
        bmul[k] = w / (bsel[k] == 2 ? 64 : (bsel[k] == 1 ? 8 : 1));
    }
    // (w/b) M_b > tau_w  <=>  M_b > floor(tau_w / (w/b)): per base, the smallest such threshold over
    // its widths (widths k >= n_width have w = 0 and never pass)
    int32_t thb0 = 2147483647, thb1 = 2147483647, thb2 = 2147483647;
#pragma unroll
    for (int k = 0; k < NWB; k++) {
        if (bmul[k] > 0) {
            int32_t q = tk[k] / bmul[k];
            if (tk[k] % bmul[k] != 0 && tk[k] < 0) q -= 1;  // floor
            if (bsel[k] == 0) thb0 = min(thb0, q);
            if (bsel[k] == 1) thb1 = min(thb1, q);
            if (bsel[k] == 2) thb2 = min(thb2, q);
        }
    }
    // the ring's mirror of slot 0 must cover every read past the end of slot 2
    const int mirror = bound ? min(kWarpCS, 2 * wmax + 64) : wmax;

    // raw samples of chunk c for lane l: 16 consecutive ones, m0 outside the series (centred 0)
    auto fetch = [&](int c, uint32_t (&dst)[16]) {
        const int v0 = c * kWarpCS + 16 * lane;
        const int t0 = v0 - mis;
        if (t0 >= 0 && t0 + 16 <= n) {
            const int4* src = reinterpret_cast<const int4*>(Sa + v0);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int4 a = __ldg(src + q);
                dst[4 * q + 0] = static_cast<uint32_t>(a.x);
                dst[4 * q + 1] = static_cast<uint32_t>(a.y);
                dst[4 * q + 2] = static_cast<uint32_t>(a.z);
                dst[4 * q + 3] = static_cast<uint32_t>(a.w);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 16; k++) {
                const int t = t0 + k;
                dst[k] = (t >= 0 && t < n) ? static_cast<uint32_t>(__ldg(v.S + t)) : m0u;
            }
        }
    };
    uint32_t nx[16];  // the next chunk's samples, loaded a chunk ahead
    fetch(0, nx);
    // the lane's largest sample of chunk c - 1 and of chunk c (raw values; m0 stands in outside the
    // series): the 1-sample pre-check maximum of chunk e = c - 1 is bounded by the larger of the two
    int32_t lmax_prev = -2147483647 - 1, lmax_cur = lmax_prev;

    // Chunk c = n_chunks lies wholly past the series: its flat prefix entries are written too, so
    // every chunk's pre-check can read its successor's first entries.
    for (int c = 0; c <= n_chunks; c++) {
        {
            uint32_t xs[16];
#pragma unroll
            for (int k = 0; k < 16; k++) xs[k] = nx[k];
            if (c < n_chunks) fetch(c + 1, nx);  // in flight while this chunk is scanned and the last one evaluated
            lmax_prev = lmax_cur;
            lmax_cur = static_cast<int32_t>(xs[0]);
#pragma unroll
            for (int k = 1; k < 16; k++) lmax_cur = max(lmax_cur, static_cast<int32_t>(xs[k]));
            // lane total of the centred samples, then one warp scan of the lane totals
            uint32_t lane_tot = neg16m0;
#pragma unroll
            for (int k = 0; k < 16; k += 2) lane_tot = lane_tot + xs[k] + xs[k + 1];
            uint32_t incl = lane_tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            // exclusive prefix entries of the lane's 16 samples
            uint32_t pv = carry + incl - lane_tot;
            carry += __shfl_sync(0xffffffffu, incl, 31);
#pragma unroll
            for (int k = 0; k < 16; k++) {
                const uint32_t x = xs[k];
                xs[k] = pv;
                pv = pv + x + negm0;
            }
            // padded ring layout: entry j of a slot at word j + j / 32 (conflict-free for these
            // 16-consecutive-per-lane stores and for lane-consecutive reads); slots are kSlotWords apart
            const int slot = c % 3;
            const uint32_t at = ring_s + 4u * static_cast<uint32_t>(slot * kSlotWords + 16 * lane + (lane >> 1));
            const bool mir = slot == 0 && 16 * lane < mirror;
            const uint32_t am = ring_s + 4u * static_cast<uint32_t>(3 * kSlotWords + 16 * lane + (lane >> 1));
#pragma unroll
            for (int k = 0; k < 16; k++)
                asm volatile("st.shared.u32 [%0], %1;" ::"r"(at + 4u * k), "r"(xs[k]) : "memory");
            if (mir) {
#pragma unroll
                for (int k = 0; k < 16; k++)
                    asm volatile("st.shared.u32 [%0], %1;" ::"r"(am + 4u * k), "r"(xs[k]) : "memory");
            }
            __syncwarp();
        }
        if (c == 0) continue;
        // evaluate chunk e = c - 1: vv = e*CS + 32*m + lane, sample t = vv - mis
        const int e = c - 1;
        const int ebase = e * kWarpCS;
        if (ebase >= nv) break;
        const uint32_t s_slot = ring_s + 4u * static_cast<uint32_t>((e % 3) * kSlotWords);
        // word address of chunk-relative prefix entry j (j may run past this slot into the next one,
        // which the padding keeps contiguous: slot size = padded 512)
        auto addr = [&](int j) { return s_slot + 4u * static_cast<uint32_t>(j + (j >> 5)); };
        const bool interior = ebase - mis >= 0 && ebase + kWarpCS + wmax <= nv;  // every window inside
        if (bound) {
            // Every entry the pre-check reads is written (chunk c follows chunk e in the ring), and a
            // start outside the series only adds windows of the zero-padded series to the maxima,
            // which keeps them upper bounds.
            int32_t mx1 = -2147483647 - 1, mx2 = mx1;
            const int rows = kWarpRows + (wmax - 1 + 31) / 32;
            const uint32_t a0 = s_slot + 4u * static_cast<uint32_t>(lane);
            const uint32_t a8 = s_slot + 4u * static_cast<uint32_t>(lane + 8 + ((lane + 8) >> 5));
            const uint32_t a64 = s_slot + 4u * static_cast<uint32_t>(lane + 66);
            if (wmax >= 64)
                PrecheckRows<0, true>::run(a0, a8, a64, rows, mx1, mx2);
            else
                PrecheckRows<0, false>::run(a0, a8, a64, rows, mx1, mx2);
            // 1-sample boxes: every start of the pre-check lies in chunk e or e + 1 (rows <= 2 chunks)
            const int32_t mx0 = static_cast<int32_t>(static_cast<uint32_t>(max(lmax_prev, lmax_cur)) - m0u);
            if (!__any_sync(0xffffffffu, mx0 > thb0 || mx1 > thb1 || mx2 > thb2)) {
                __syncwarp();  // slot e % 3 may be rewritten by chunk c + 2
                continue;
            }
        }
#pragma unroll 2
        for (int m = 0; m < kWarpRows; m++) {
            const int j = 32 * m + lane;
            const int t = ebase + j - mis;
            uint32_t p0;
            asm volatile("ld.shared.u32 %0, [%1];" : "=r"(p0) : "r"(addr(j)));
            bool any = false;
            if (interior) {
#pragma unroll
                for (int k = 0; k < NWB; k++) {
                    uint32_t pw;
                    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(pw) : "r"(addr(j + wk[k])));
                    any |= static_cast<int32_t>(pw - p0) > tk[k];
                }
            } else if (t >= 0) {
#pragma unroll
                for (int k = 0; k < NWB; k++) {
                    uint32_t pw;
                    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(pw) : "r"(addr(j + wk[k])));
                    any |= (t + wk[k] <= n) && (static_cast<int32_t>(pw - p0) > tk[k]);
                }
            }
            if (!__any_sync(0xffffffffu, any)) continue;
            // exact FP32 S/N for this row, width by width
            for (int k = 0; k < v.n_width; k++) {
                const int w = __shfl_sync(0xffffffffu, w_l, k);
                const float scale = __shfl_sync(0xffffffffu, scale_l, k);
                const float offs = __shfl_sync(0xffffffffu, offs_l, k);
                bool pred = false;
                float snr = 0.f;
                if (t >= 0 && t + w <= n) {
                    uint32_t pw;
                    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(pw) : "r"(addr(j + w)));
                    const int32_t bc = static_cast<int32_t>(pw - p0);
                    snr = (static_cast<float>(bc) - offs) * scale;
                    pred = snr > v.thr;
                }
                const unsigned mask = __ballot_sync(0xffffffffu, pred);
                if (mask) {
                    const int leader = __ffs(mask) - 1;
                    unsigned long long b0 = 0;
                    if (lane == leader) b0 = atomicAdd(v.count, static_cast<unsigned long long>(__popc(mask)));
                    b0 = __shfl_sync(0xffffffffu, b0, leader);
                    if (pred) {
                        const unsigned long long idx = b0 + __popc(mask & lt_mask);
                        if (idx < static_cast<unsigned long long>(v.cap)) {
                            fdd_candidate cd;
                            cd.sb = v.sb;
                            cd.dm_index = v.dm_index;
                            cd.downsamp = v.D;
                            cd.width_native = w * v.D;
                            cd.t_native = static_cast<int64_t>(t) * v.D + v.t_offset;
                            cd.dm = static_cast<float>(v.dm);
                            cd.snr = snr;
                            v.cands[idx] = cd;
                        }
                    }
                }
            }
        }
        __syncwarp();  // slot e % 3 may be rewritten by chunk c + 2
    }
}

}  // namespace detail
}  // namespace fdd
