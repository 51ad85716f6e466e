// sbf_part.cuh -- the part tile of the SB-factored dedispersion (partial
// sums P[tab][segment][trial][t] of one TAB over channel segments), shared by
// the per-slab part kernel (k_sbf.cu) and the persistent SB-factored batch
// kernel (k_sbf_persist.cu).
#pragma once

#include "dedisp_tile.cuh"

namespace fdd {

namespace detail {

// One part tile: TAB `tab`, DM block a.i0 / BD + blk_rel, output samples
// [tile * T, (tile + 1) * T); smem holds sbf_smem_bytes of the variant.
// Called by every thread of the block (the standalone part kernel and the
// persistent SB-factored kernel).
template <int E, int NW, int DPW, int WARPS, int MAXIT>
__device__ __forceinline__ void sbf_part_tile(const SbfPartArgs& a, const int tile, const int blk_rel, const int tab,
                                              uint8_t* smem) {
    constexpr int NC = 4 / E;
    constexpr int SPW = 4 / E;
    constexpr int BD = WARPS * DPW;
    constexpr int T = 32 * NW * SPW;
    constexpr int NT = WARPS * 32;

    const int blk = a.i0 / BD + blk_rel;
    const int Lw = a.Lw;
    const int chunks = Lw >> 2;
    const int slot_bytes = NC * Lw * 4;
    uint8_t* s_rows = smem;
    int32_t* s_off = reinterpret_cast<int32_t*>(smem + a.CC * slot_bytes);  // [CC][BD]

    const int t0 = tile * T;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t limit = a.n_valid * E;
    const uint8_t* tab_rows = a.in + static_cast<int64_t>(tab) * a.n_chan * a.pitch_bytes;
    const int32_t* base_blk = a.base + (int64_t)blk * a.n_chan;
    const int32_t* off_blk = a.off + (int64_t)blk * a.n_chan * BD;

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
                const uint8_t* row = tab_rows + (int64_t)c * a.pitch_bytes;
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
            reinterpret_cast<int4*>(s_off)[threadIdx.x] = make_int4(po.x + add, po.y + add, po.z + add, po.w + add);
        }
    };

    auto split = [](uint32_t x) -> uint32_t {
        if constexpr (E == 1)
            return __byte_perm(x, 0u, 0x4341);  // bytes 1,3 -> 16-bit lanes
        else
            return 0u;                          // uint16 lanes accumulate directly in acc_a
    };

    uint32_t acc_a[DPW][NW], acc_b[DPW][NW];
#pragma unroll
    for (int j = 0; j < DPW; j++)
#pragma unroll
        for (int k = 0; k < NW; k++) acc_a[j][k] = acc_b[j][k] = 0u;

    const uint32_t s_lane32 = static_cast<uint32_t>(__cvta_generic_to_shared(s_rows)) + 4u * lane;
    const int32_t* s_off_w = s_off + warp * DPW;

    // Store the 16-bit sums of segment g and restart the accumulators.
    auto store_segment = [&](int g) {
#pragma unroll
        for (int j = 0; j < DPW; j++) {
            const int i = blk * BD + warp * DPW + j;
            const bool valid = i < a.n_dm && i < a.i0 + a.n_slab;  // warp-uniform
            uint16_t* row = a.P + tab * a.tab_stride + g * a.seg_stride + (int64_t)(i - a.i0) * a.Np;
#pragma unroll
            for (int k = 0; k < NW; k++) {
                const int t = t0 + (lane + 32 * k) * SPW;
                if (valid) {
                    if constexpr (E == 1) {
                        const uint32_t odd = acc_b[j][k];                // samples 1, 3
                        const uint32_t even = acc_a[j][k] - (odd << 8);  // samples 0, 2
                        *reinterpret_cast<uint2*>(row + t) =
                            make_uint2(__byte_perm(even, odd, 0x5410), __byte_perm(even, odd, 0x7632));
                    } else {
                        *reinterpret_cast<uint32_t*>(row + t) = acc_a[j][k];
                    }
                }
                acc_a[j][k] = 0u;
                acc_b[j][k] = 0u;
            }
        }
    };

    int4 sd = __ldg(&a.stages[0]);  // first channel, channels, first segment, segments
    stage_load(sd.x, sd.y);
    stage_store(sd.y);
    __syncthreads();

    for (int st = 0; st < a.n_stages; st++) {
        const int4 cur = sd;
        const bool has_next = st + 1 < a.n_stages;
        int4 nxt = cur;
        if (has_next) {
            nxt = __ldg(&a.stages[st + 1]);
            stage_load(nxt.x, nxt.y);  // in flight during the adds below
        }
        for (int g = cur.z; g < cur.z + cur.w; g++) {
            const int2 sg = __ldg(&a.segs[g]);
            int cc = sg.x - cur.x;
            const int cc_end = cc + sg.y;
#pragma unroll 1
            for (; cc + 3 < cc_end; cc += 4) {
                int32_t og[4][DPW];
#pragma unroll
                for (int u = 0; u < 4; u++) detail::load_offsets<DPW>(s_off_w + (cc + u) * BD, og[u]);
                uint32_t x[4][DPW][NW];
#pragma unroll
                for (int u = 0; u < 4; u++)
#pragma unroll
                    for (int j = 0; j < DPW; j++) {
                        const uint32_t ad = s_lane32 + static_cast<uint32_t>(og[u][j]);
#pragma unroll
                        for (int k = 0; k < NW; k++) x[u][j][k] = detail::lds32(ad + 128u * k);
                    }
#pragma unroll
                for (int j = 0; j < DPW; j++)
#pragma unroll
                    for (int k = 0; k < NW; k++) {
                        acc_a[j][k] = acc_a[j][k] + x[0][j][k] + x[1][j][k];
                        acc_a[j][k] = acc_a[j][k] + x[2][j][k] + x[3][j][k];
                        if constexpr (E == 1) {
                            acc_b[j][k] = acc_b[j][k] + split(x[0][j][k]) + split(x[1][j][k]);
                            acc_b[j][k] = acc_b[j][k] + split(x[2][j][k]) + split(x[3][j][k]);
                        }
                    }
            }
#pragma unroll 1
            for (; cc < cc_end; cc++) {
                int32_t o0[DPW];
                detail::load_offsets<DPW>(s_off_w + cc * BD, o0);
#pragma unroll
                for (int j = 0; j < DPW; j++)
#pragma unroll
                    for (int k = 0; k < NW; k++) {
                        const uint32_t x0 = detail::lds32(s_lane32 + static_cast<uint32_t>(o0[j]) + 128u * k);
                        acc_a[j][k] += x0;
                        if constexpr (E == 1) acc_b[j][k] += split(x0);
                    }
            }
            store_segment(g);
        }
        __syncthreads();  // stage fully consumed
        if (has_next) {
            stage_store(nxt.y);
            __syncthreads();
            sd = nxt;
        }
    }
}

}  // namespace detail

}  // namespace fdd
