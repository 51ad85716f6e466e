// k_dedisp_fact.cu -- pattern-factored exact dedispersion (native-rate
// ranges).  Same result as k_dedisp, bit for bit; fewer shared-memory reads
// per channel-add.  See fdd_fact.cu for the factorisation and its tables.
//
// Block = BD trials x T = 64*NW output samples of one SB.  Per channel stage:
//   1. staging: TMA tensor copies (one to four boxes per channel) bring the
//      SB's TAB row (Lw words from a 16-byte-aligned start, zero past the
//      row's valid words) into shared memory, unshifted; raw rows are double-buffered
//      and the copies of stage s+2 are issued as soon as stage s's builds
//      are done, so the loads run behind two stages of work and no register
//      holds them;
//   2. build: each warp takes pattern rows of the stage's channel groups
//      (descriptors staged in shared memory); a lane forms 4 consecutive
//      samples of R_p(tau) = sum_k X_k(tau + rel_k) from two aligned LDS.32
//      per channel joined by a funnel shift (rows start at any byte), odd
//      bytes split off with one PRMT, even bytes recovered by subtraction,
//      and stores them as two copies of 16-bit pairs, the second shifted by
//      one sample (the neighbouring lane's first sample comes by shuffle), so
//      every trial's offset is an aligned LDS.32;
//   3. accumulate: each trial adds, per group, one word of two 16-bit
//      partials into 16-bit lanes (two groups per IADD3), folded into 32-bit
//      totals before a lane holds more than 256 channels.
// The raw rows are read only by the builds (a few pattern rows per group),
// not by every trial, which is why one unshifted TMA copy beats the four
// byte-shifted copies the brute-force kernel stages.
#include "fdd_internal.cuh"
#include "tma.cuh"

namespace fdd {

namespace {

__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ void sts32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ void sts64(uint32_t addr, uint32_t a, uint32_t b) {
    asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
}

template <int N>
__device__ __forceinline__ void load_offsets(const int32_t* p, int32_t (&o)[N]) {
    if constexpr (N == 1) {
        o[0] = p[0];
    } else if constexpr (N == 2) {
        const int2 v = *reinterpret_cast<const int2*>(p);
        o[0] = v.x;
        o[1] = v.y;
    } else if constexpr (N == 4) {
        const int4 v = *reinterpret_cast<const int4*>(p);
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    } else {
        static_assert(N == 8, "DPW must be 1, 2, 4 or 8");
        const int4 v = *reinterpret_cast<const int4*>(p);
        const int4 w = *reinterpret_cast<const int4*>(p + 4);
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
        o[4] = w.x;
        o[5] = w.y;
        o[6] = w.z;
        o[7] = w.w;
    }
}

// Pattern-row builds (whole warp).  A row descriptor in shared memory is
// {dst0, dst1, nw4, src[G]}: copy-0 and copy-1 destinations, units of 4
// samples, and the shared-memory byte address of unit 0 of each channel's
// raw row (any alignment: a lane reads the aligned words around it and
// funnel-shifts).  Per lane and unit: acc_a = sum of the G raw words (bytes
// overlap), acc_b = sum of bytes 1,3 in 16-bit lanes (one PRMT per word);
// samples 0,2 are acc_a - (acc_b << 8) (lanes hold <= 257 * 255).  Copy 0
// stores [R0,R1],[R2,R3]; copy 1 stores [R1,R2],[R3,R4], R4 being the next
// lane's R0 (shuffle; across a 32-unit step it comes from lane 0 of the next
// step).
// E = bytes per input sample: 1 (raw 8-bit rows, byte lanes split into even and odd samples) or 2
// (downsampled 16-bit rows: a unit's four samples are two words, summed in 16-bit lanes directly).
template <int G, int E>
struct RowState {
    uint32_t dst0, dst1, src[G], sh[G];
    int nw4;
    uint32_t pend_b;

    __device__ __forceinline__ void load(uint32_t d, uint32_t s0) {
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(dst0), "=r"(dst1), "=r"(nw4), "=r"(src[0])
                     : "r"(d));
#pragma unroll
        for (int k = 1; k < G; k++) src[k] = lds32(d + 4u * (3 + k));
#pragma unroll
        for (int k = 0; k < G; k++) {
            sh[k] = src[k] << 3;             // funnel shift uses the low 5 bits: 8 * (byte & 3)
            src[k] = (s0 + src[k]) & ~3u;    // aligned word holding the row's first byte (s0 is 128-aligned)
        }
        dst0 += s0;
        dst1 += s0;
        pend_b = 0;
    }

    // One 32-unit step starting at unit jb (jb < nw4 or the row is done).
    __device__ __forceinline__ void step(int jb, int lane) {
        if (jb >= nw4) return;  // warp-uniform
        const int j = jb + lane;
        uint32_t A, B, C;  // [R0, R1], [R2, R3], [R1, R2]
        if constexpr (E == 1) {
            uint32_t acc_a = 0, acc_b = 0;
            if (j < nw4) {
#pragma unroll
                for (int k = 0; k < G; k += 2) {
                    const uint32_t a0 = src[k] + 4u * j, a1 = src[k + 1] + 4u * j;
                    const uint32_t x0 = __funnelshift_r(lds32(a0), lds32(a0 + 4u), sh[k]);
                    const uint32_t x1 = __funnelshift_r(lds32(a1), lds32(a1 + 4u), sh[k + 1]);
                    acc_a = acc_a + x0 + x1;
                    acc_b = acc_b + __byte_perm(x0, 0u, 0x4341) + __byte_perm(x1, 0u, 0x4341);
                }
            }
            const uint32_t od = acc_b;                 // [R1, R3]
            const uint32_t ev = acc_a - (acc_b << 8);  // [R0, R2]
            A = __byte_perm(ev, od, 0x5410);
            B = __byte_perm(ev, od, 0x7632);
            C = __byte_perm(od, ev, 0x7610);
        } else {
            // 16-bit samples: unit j is bytes [8 j, 8 j + 8) of each channel's row (sums of G samples of
            // at most 255 D each stay below 2^16)
            uint32_t acc0 = 0, acc1 = 0;
            if (j < nw4) {
#pragma unroll
                for (int k = 0; k < G; k++) {
                    const uint32_t a0 = src[k] + 8u * j;
                    const uint32_t w0 = lds32(a0), w1 = lds32(a0 + 4u), w2 = lds32(a0 + 8u);
                    acc0 += __funnelshift_r(w0, w1, sh[k]);
                    acc1 += __funnelshift_r(w1, w2, sh[k]);
                }
            }
            A = acc0;
            B = acc1;
            C = __byte_perm(acc0, acc1, 0x5432);
        }
        const uint32_t next_a = __shfl_down_sync(0xffffffffu, A, 1);
        const uint32_t first_a = __shfl_sync(0xffffffffu, A, 0);
        if (j < nw4) {
            sts64(dst0 + 8u * j, A, B);
            sts32(dst1 + 8u * j, C);
            if (lane < 31) sts32(dst1 + 8u * j + 4u, __byte_perm(B, next_a, 0x5432));  // [R3, R4]
        }
        if (lane == 31 && jb > 0) sts32(dst1 + 8u * (jb - 1) + 4u, __byte_perm(pend_b, first_a, 0x5432));
        pend_b = B;
    }

    __device__ __forceinline__ void finish(int lane) {
        if (lane == 31 && nw4 > 0 && (nw4 & 31) == 0)
            sts32(dst1 + 8u * (nw4 - 1) + 4u, __byte_perm(pend_b, 0u, 0x5432));
    }
};

// Rows d0 and d1 (d1 == 0xffffffff: none) interleaved step by step, so a
// lane has two independent build chains in flight.
template <int G, int E>
__device__ __forceinline__ void build_rows(uint32_t d0, uint32_t d1, uint32_t s0, int lane) {
    RowState<G, E> a, b;
    a.load(d0, s0);
    const bool two = d1 != 0xffffffffu;
    if (two) {
        b.load(d1, s0);
    } else {
        b.nw4 = 0;
        b.pend_b = 0;
    }
    const int n = max(a.nw4, b.nw4);
    for (int jb = 0; jb < n; jb += 32) {
        a.step(jb, lane);
        b.step(jb, lane);
    }
    a.finish(lane);
    if (two) b.finish(lane);
}

// PB = 1: per stage, build its pattern rows, barrier, accumulate, barrier.
// PB = 2: two pattern-row buffers; one interval between barriers builds
// stage s + 1 and accumulates stage s, so a warp that finishes its builds
// goes straight on to its adds (the build rounds differ between warps) and
// a stage costs one barrier.  Stage offsets then rotate over three buffers
// (stage s + 2's are stored while stage s's are read) and descriptors over two.
// PART: the block's z index is a TAB, every channel row comes from that TAB, and each channel
// segment's 16-bit sums are stored to P when its last group is added (the SB-factored part step;
// segments are whole groups), instead of accumulating all channels into a series.
template <int G, int NW, int DPW, int WARPS, int PB, bool PART, int E>
__global__ void __launch_bounds__(WARPS * 32, (WARPS <= 8) ? 2 : 1)
    k_dedisp_fact(const __grid_constant__ FactArgs a) {
    constexpr int BD = WARPS * DPW;
    constexpr int T = 64 * NW;
    constexpr int DI = (3 + G + 3) / 4 * 4;
    constexpr int NGB = PB + 1;  // stage-offset buffers
    static_assert(BD % 4 == 0, "BD must be a multiple of 4");
    static_assert(PB == 1 || PB == 2, "one or two pattern-row buffers");
    extern __shared__ __align__(16) uint8_t smem_raw[];

    const int Lw = a.Lw, CC = a.CC;
    const int gps = CC / G;
    // every offset below is from the 128-byte-aligned base (TMA destinations)
    const uint32_t s_unal = static_cast<uint32_t>(__cvta_generic_to_shared(smem_raw));
    const uint32_t s0 = (s_unal + 127u) & ~127u;
    uint8_t* smem = smem_raw + (s0 - s_unal);
    int32_t* s_goff = reinterpret_cast<int32_t*>(smem + a.pat_off + PB * a.pat_bytes);  // [NGB][gps][BD]
    int32_t* s_desc = s_goff + NGB * gps * BD;  // [PB][max_desc][DI]: descriptors of the stage(s) to build
    const uint32_t s_desc32 = static_cast<uint32_t>(__cvta_generic_to_shared(s_desc));
    const uint32_t s_bar = s0 + static_cast<uint32_t>(a.bar_off);  // two 8-byte mbarriers (raw buffers 0, 1)

    // DM block of the range (in part mode the grid covers the slab starting at trial a.i0)
    const int blk = PART ? a.i0 / BD + static_cast<int>(blockIdx.y) : static_cast<int>(blockIdx.y);
    const int sb = blockIdx.z;  // SB, or the TAB in part mode
    const int t0 = blockIdx.x * T;
    const int i0 = blk * BD;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int16_t* sbm = PART ? nullptr : a.sb_map + (int64_t)sb * a.n_chan;
    const int32_t* base_blk = a.base + (int64_t)blk * a.n_chan;
    const int32_t* goff_blk = a.goff + (int64_t)blk * a.n_groups * BD;
    const int32_t* pd_blk = a.pd_idx + (int64_t)blk * a.n_stages * 2;

    for (int i = threadIdx.x; i < Lw + 4; i += WARPS * 32)
        reinterpret_cast<uint32_t*>(smem + a.zero_off)[i] = 0u;  // zero row (missing channels)
    if (threadIdx.x == 0) {
        tma::mbar_init(s_bar, 1);
        tma::mbar_init(s_bar + 8u, 1);
        tma::mbar_init_fence();
    }
    __syncthreads();

    // Raw rows of stage s into buffer s & 1 (warp 0): Lw words per channel
    // (fact_boxes(Lw) boxes), from word (t0 + base) / 4 of row (TAB, c).
    // coords(s) loads each lane's channels' coordinates (channel lane and
    // lane + 32; CC <= 64) a stage before fire(s) needs them, so the global
    // loads' latency is not in front of a barrier; fire(s) arms the buffer's
    // barrier with the stage's byte count (lane 0) and issues the copies.
    // With channel boxes (R = a.box_rows > 1) lane q < ceil(ncc / R) copies channels R q .. R q + R - 1
    // of the stage as one box of rb / 4 words from the box's least start (bbase); their rows land in
    // their own slots (the box row pitch is the slot size).
    const int R = a.box_rows;
    const int32_t* bbase_blk = a.bbase + (int64_t)blk * ((a.n_chan + R - 1) / R);
    int cx[2] = {0, 0}, cy[2] = {0, 0};
    auto coords = [&](int s) {
        const int c0 = s * CC;
        const int ncc = min(CC, a.n_chan - c0);
        if (R > 1) {
            if (R * lane < ncc) {
                const int c = c0 + R * lane;
                cx[0] = ((t0 + bbase_blk[c / R]) * E) >> 2;
                cy[0] = (PART ? sb : sbm[c]) * a.n_chan + c;
            }
            return;
        }
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int cc = lane + 32 * q;
            if (cc < ncc) {
                const int c = c0 + cc;
                cx[q] = ((t0 + base_blk[c]) * E) >> 2;  // word of the row's first staged sample
                cy[q] = (PART ? sb : sbm[c]) * a.n_chan + c;
            }
        }
    };
    auto fire = [&](int s) {
        const int c0 = s * CC;
        const int ncc = min(CC, a.n_chan - c0);
        const uint32_t bar = s_bar + 8u * (s & 1);
        const uint32_t dst = s0 + static_cast<uint32_t>(a.raw_off + (s & 1) * CC * a.rb);
        if (R > 1) {
            const int nbox = (ncc + R - 1) / R;
            if (lane == 0)
                tma::mbar_expect_tx(bar, static_cast<uint32_t>(nbox * R) * static_cast<uint32_t>(a.rb));
            __syncwarp();
            if (lane < nbox) tma::load_2d(dst + static_cast<uint32_t>(R * lane * a.rb), &a.tmap, cx[0], cy[0], bar);
            return;
        }
        if (lane == 0) tma::mbar_expect_tx(bar, static_cast<uint32_t>(ncc) * static_cast<uint32_t>(Lw) * 4u);
        __syncwarp();
        const int nb = fact_boxes(Lw), bw = Lw / nb;
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int cc = lane + 32 * q;
            if (cc < ncc)
                for (int k = 0; k < nb; k++)
                    tma::load_2d(dst + static_cast<uint32_t>(cc * a.rb + 4 * k * bw), &a.tmap, cx[q] + k * bw, cy[q],
                                 bar);
        }
    };

    int4 po = make_int4(0, 0, 0, 0);
    int4 pdv = make_int4(0, 0, 0, 0);
    int n_desc_next = 0;

    // stage offsets and descriptors of stage s into registers, then shared memory
    auto small_load = [&](int s) {
        const int ncc = min(CC, a.n_chan - s * CC);
        const int ngs = (ncc + G - 1) / G;
        if (threadIdx.x < ngs * (BD / 4))
            po = __ldg(reinterpret_cast<const int4*>(goff_blk + (int64_t)(s * gps) * BD) + threadIdx.x);
        const int first = pd_blk[2 * s];
        n_desc_next = pd_blk[2 * s + 1];
        if (threadIdx.x < n_desc_next * (DI / 4))
            pdv = __ldg(reinterpret_cast<const int4*>(a.pdesc + (int64_t)first * DI) + threadIdx.x);
    };
    auto small_store = [&](int s, int buf, int dbuf) {
        const int ncc = min(CC, a.n_chan - s * CC);
        const int ngs = (ncc + G - 1) / G;
        if (threadIdx.x < ngs * (BD / 4)) reinterpret_cast<int4*>(s_goff + buf * gps * BD)[threadIdx.x] = po;
        if (threadIdx.x < n_desc_next * (DI / 4))
            reinterpret_cast<int4*>(reinterpret_cast<uint8_t*>(s_desc) + dbuf * a.desc_bytes)[threadIdx.x] = pdv;
    };
    // every pattern row of one stage: warp w builds rows w, w + WARPS, w + 2 WARPS, ..., two at a
    // time (two build chains per lane), so the counts differ by at most one
    auto build_stage = [&](int n_desc, int dbuf) {
        const uint32_t sd = s_desc32 + static_cast<uint32_t>(dbuf * a.desc_bytes);
        for (int d = warp; d < n_desc; d += 2 * WARPS)
            build_rows<G, E>(sd + 4u * DI * d, d + WARPS < n_desc ? sd + 4u * DI * (d + WARPS) : 0xffffffffu, s0,
                             lane);
    };

    // Per output word: acc = two 16-bit partial sums (samples 2m, 2m+1); a
    // lane gains <= G*255 per group, so lanes are folded into the 32-bit
    // totals before they hold more than 256 channels.
    uint32_t acc[DPW][NW], tot_lo[DPW][NW], tot_hi[DPW][NW];
#pragma unroll
    for (int j = 0; j < DPW; j++)
#pragma unroll
        for (int k = 0; k < NW; k++) {
            acc[j][k] = 0u;
            tot_lo[j][k] = 0u;
            tot_hi[j][k] = 0u;
        }
    auto fold = [&]() {
#pragma unroll
        for (int j = 0; j < DPW; j++)
#pragma unroll
            for (int k = 0; k < NW; k++) {
                tot_lo[j][k] += acc[j][k] & 0xFFFFu;
                tot_hi[j][k] += acc[j][k] >> 16;
                acc[j][k] = 0u;
            }
    };

    const uint32_t s_lane = s0 + 4u * lane;
    int since_fold = 0;  // channels held in the 16-bit lanes
    // part mode: the 16-bit sums of segment seg to P (two samples per word), lanes restarted
    auto store_segment = [&](int seg) {
#pragma unroll
        for (int j = 0; j < DPW; j++) {
            const int i = i0 + warp * DPW + j;
            const bool valid = i < a.n_dm && i - a.i0 < a.n_slab;  // warp-uniform
            uint32_t* row = reinterpret_cast<uint32_t*>(a.P + sb * a.tab_stride + seg * a.seg_stride +
                                                        static_cast<int64_t>(i - a.i0) * a.Np + t0) + lane;
#pragma unroll
            for (int k = 0; k < NW; k++) {
                if (valid) row[32 * k] = acc[j][k];
                acc[j][k] = 0u;
            }
        }
    };
    // adds of stage s: every trial, one 16-bit pattern partial per group, offsets from buffer gbuf
    auto accumulate = [&](int s, int gbuf) {
        const int ncc = min(CC, a.n_chan - s * CC);
        const int ngs = (ncc + G - 1) / G;
        if constexpr (!PART) {
            if (since_fold + ncc > a.fold_ch) {
                fold();
                since_fold = 0;
            }
            since_fold += ncc;
        }
        int2 ss = make_int2(0, 0);  // part mode: segment-closing groups of the stage, first segment
        if constexpr (PART) ss = __ldg(&a.sseg[s]);
        int seg = ss.y;
        const int32_t* go = s_goff + gbuf * gps * BD + warp * DPW;
        int gl = 0;
#pragma unroll 1
        while (gl < ngs) {
            // two groups at a time unless the first closes a segment (part mode)
            if (gl + 1 >= ngs || (PART && ((ss.x >> gl) & 1))) {
                int32_t o0[DPW];
                load_offsets<DPW>(go + gl * BD, o0);
#pragma unroll
                for (int j = 0; j < DPW; j++)
#pragma unroll
                    for (int k = 0; k < NW; k++) acc[j][k] += lds32(s_lane + static_cast<uint32_t>(o0[j]) + 128u * k);
                gl += 1;
            } else {
            int32_t o0[DPW], o1[DPW];
            load_offsets<DPW>(go + gl * BD, o0);
            load_offsets<DPW>(go + (gl + 1) * BD, o1);
            uint32_t x[2][DPW][NW];
#pragma unroll
            for (int j = 0; j < DPW; j++)
#pragma unroll
                for (int k = 0; k < NW; k++) {
                    x[0][j][k] = lds32(s_lane + static_cast<uint32_t>(o0[j]) + 128u * k);
                    x[1][j][k] = lds32(s_lane + static_cast<uint32_t>(o1[j]) + 128u * k);
                }
#pragma unroll
            for (int j = 0; j < DPW; j++)
#pragma unroll
                for (int k = 0; k < NW; k++) acc[j][k] = acc[j][k] + x[0][j][k] + x[1][j][k];
                gl += 2;
            }
            if constexpr (PART) {
                if ((ss.x >> (gl - 1)) & 1) store_segment(seg++);
            }
        }
    };
    // a raw-row copy did not land: flag it, let thread 0 wait (bounded) for the copies of stages
    // s1 and s2 (s2 < 0: none) still in flight, then the block stops
    auto drain = [&](int s1, int s2) {
        if (threadIdx.x == 0) {
            atomicOr(a.status, 1u);
            tma::mbar_wait_bounded(s_bar + 8u * (s1 & 1), static_cast<uint32_t>(s1 >> 1) & 1u);
            if (s2 >= 0) tma::mbar_wait_bounded(s_bar + 8u * (s2 & 1), static_cast<uint32_t>(s2 >> 1) & 1u);
        }
    };

    if (warp == 0) {
        coords(0);
        fire(0);
        if (a.n_stages > 1) {
            coords(1);
            fire(1);
        }
        if (a.n_stages > 2) coords(2);
    }
    small_load(0);
    small_store(0, 0, 0);
    if constexpr (PB == 1) {
        __syncthreads();
        for (int s = 0; s < a.n_stages; s++) {
            const int buf = s & 1;
            const bool next = s + 1 < a.n_stages;
            const int n_desc = n_desc_next;
            if (next) small_load(s + 1);
            const bool ok = tma::mbar_wait_bounded(s_bar + 8u * buf, static_cast<uint32_t>(s >> 1) & 1u);
            if (ok) build_stage(n_desc, 0);
            // pattern rows complete; raw buffer buf and the descriptors free
            if (__syncthreads_or(!ok)) {
                drain(s, next ? s + 1 : -1);
                return;
            }
            if (warp == 0 && s + 2 < a.n_stages) {
                fire(s + 2);                                    // into buffer buf, behind two stages of work
                if (s + 3 < a.n_stages) coords(s + 3);
            }
            if (next) small_store(s + 1, buf ^ 1, 0);
            accumulate(s, buf);
            __syncthreads();  // pattern rows consumed; next stage's offsets and descriptors visible
        }
    } else {
        // prologue: stage 1's offsets and descriptors stored, stage 0 built
        int nd_build = n_desc_next;  // pattern rows of the stage built next
        int nd_next = 0;
        if (a.n_stages > 1) {
            small_load(1);
            small_store(1, 1, 1);
            nd_next = n_desc_next;
        }
        __syncthreads();
        {
            const bool ok = tma::mbar_wait_bounded(s_bar, 0u);
            if (ok) build_stage(nd_build, 0);
            if (__syncthreads_or(!ok)) {
                drain(0, a.n_stages > 1 ? 1 : -1);
                return;
            }
        }
        nd_build = nd_next;
        if (warp == 0 && a.n_stages > 2) {
            fire(2);  // raw buffer 0: stage 0 is built
            if (a.n_stages > 3) coords(3);
        }
        for (int s = 0; s < a.n_stages; s++) {
            const bool next = s + 1 < a.n_stages;
            const bool next2 = s + 2 < a.n_stages;
            if (next2) small_load(s + 2);
            bool ok = true;
            if (next) {
                ok = tma::mbar_wait_bounded(s_bar + 8u * ((s + 1) & 1), static_cast<uint32_t>((s + 1) >> 1) & 1u);
                if (ok) build_stage(nd_build, (s + 1) & 1);  // into pattern buffer (s + 1) & 1
            }
            accumulate(s, s % 3);
            // stage s + 2's offsets: buffer (s + 2) % 3, last read by stage s - 1's adds; its
            // descriptors: buffer s & 1, last read by stage s's builds (previous interval)
            if (next2) small_store(s + 2, (s + 2) % 3, s & 1);
            if (__syncthreads_or(!ok)) {
                drain(s + 1, next2 ? s + 2 : -1);
                return;
            }
            nd_build = n_desc_next;
            if (warp == 0 && s + 3 < a.n_stages) {
                fire(s + 3);  // raw buffer (s + 1) & 1: stage s + 1 is built
                if (s + 4 < a.n_stages) coords(s + 4);
            }
        }
    }
    if constexpr (PART) return;  // every segment is stored
    fold();

    // Epilogue: two samples per word; write the series and fold the moments.
#pragma unroll
    for (int j = 0; j < DPW; j++) {
        const int i = i0 + warp * DPW + j;
        if (i >= a.n_dm) continue;  // warp-uniform
        const int64_t q = (int64_t)sb * a.n_dm + i;
        int32_t* row = a.series + q * a.n_out;
        long long s1 = 0;
        unsigned long long s2 = 0;
#pragma unroll
        for (int k = 0; k < NW; k++) {
            const uint32_t hi = tot_hi[j][k];
            const uint32_t lo = tot_lo[j][k];
            const int t = t0 + 2 * (lane + 32 * k);
            if (t < a.n_emit) {
                row[t] = static_cast<int32_t>(lo);
                s1 += lo;
                s2 += static_cast<unsigned long long>(lo) * lo;
            }
            if (t + 1 < a.n_emit) {
                row[t + 1] = static_cast<int32_t>(hi);
                s1 += hi;
                s2 += static_cast<unsigned long long>(hi) * hi;
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

using FactFn = void (*)(const FactArgs);

struct FEntry {
    FactVariant v;
    FactFn fn[2];    // by bytes per sample (E = 1, 2); nullptr: not built for that width
    FactFn part[2];  // part mode (the SB-factored partial sums), or nullptr
};

#define FDD_F(G, NW, DPW, WARPS) \
    {{G, NW, DPW, WARPS, 1}, {k_dedisp_fact<G, NW, DPW, WARPS, 1, false, 1>, nullptr}, {nullptr, nullptr}}
#define FDD_FP(G, NW, DPW, WARPS)                                                                              \
    {{G, NW, DPW, WARPS, 1},                                                                                   \
     {k_dedisp_fact<G, NW, DPW, WARPS, 1, false, 1>, k_dedisp_fact<G, NW, DPW, WARPS, 1, false, 2>},        \
     {k_dedisp_fact<G, NW, DPW, WARPS, 1, true, 1>, k_dedisp_fact<G, NW, DPW, WARPS, 1, true, 2>}}
#define FDD_F2(G, NW, DPW, WARPS) \
    {{G, NW, DPW, WARPS, 2}, {k_dedisp_fact<G, NW, DPW, WARPS, 2, false, 1>, nullptr}, {nullptr, nullptr}}
#define FDD_F2P(G, NW, DPW, WARPS)                                                                             \
    {{G, NW, DPW, WARPS, 2},                                                                                   \
     {k_dedisp_fact<G, NW, DPW, WARPS, 2, false, 1>, nullptr},                                                \
     {k_dedisp_fact<G, NW, DPW, WARPS, 2, true, 1>, k_dedisp_fact<G, NW, DPW, WARPS, 2, true, 2>}}
const FEntry kFEntries[] = {
    FDD_FP(8, 4, 4, 16),  // G 8, BD 64, T 256, 512 threads
    FDD_F(8, 4, 2, 16),  // G 8, BD 32, T 256
    FDD_FP(4, 4, 4, 16),  // G 4, BD 64, T 256
    FDD_F(8, 2, 4, 16),  // G 8, BD 64, T 128
    FDD_F(8, 8, 2, 16),  // G 8, BD 32, T 512
    FDD_F(4, 8, 2, 16),  // G 4, BD 32, T 512
    FDD_F(4, 2, 8, 8),   // G 4, BD 64, T 128, 256 threads (two blocks per SM)
    FDD_FP(4, 4, 4, 8),   // G 4, BD 32, T 256, 256 threads
    FDD_F2(4, 4, 4, 16),  // two pattern-row buffers: G 4, BD 64, T 256, 512 threads
    FDD_F2P(4, 4, 4, 8),  // two pattern-row buffers: G 4, BD 32, T 256, 256 threads (also in part mode)
    FDD_F2(8, 4, 4, 16),  // two pattern-row buffers: G 8, BD 64, T 256, 512 threads
    FDD_F(4, 3, 4, 16),  // G 4, BD 64, T 192: pattern rows of ~53 units fill 2 warp steps (83 % of lanes)
};
#undef FDD_F
#undef FDD_FP
#undef FDD_F2
#undef FDD_F2P

}  // namespace

int num_fact_variants() { return static_cast<int>(sizeof(kFEntries) / sizeof(kFEntries[0])); }

const FactVariant& fact_variant(int idx) { return kFEntries[idx].v; }

bool fact_cc_ok(const FactVariant& v, int Lw, int CC, int max_desc) {
    if (CC < v.G || CC % v.G != 0 || CC > 64) return false;  // two channels per lane of the copy-issuing warp
    if (Lw < 4 || Lw > kFactMaxLw || Lw % fact_lw_align(Lw) != 0) return false;  // whole, aligned boxes
    if (max_desc * (v.desc_ints() / 4) > v.threads()) return false;
    if ((CC / v.G) * (v.bd() / 4) > v.threads()) return false;
    return true;
}

// The input rows as a 2-D uint32 tensor: dim 0 = words of a row (the valid
// bytes rounded up to a word; TMA fills zeros past it), dim 1 = rows
// (TAB, channel); box = Lw / fact_boxes(Lw) words of one row.  Rounding up may bring in up to
// three bytes past the valid ones (inside the row pitch), which reach only
// output samples at or beyond n_out.
cudaError_t encode_fact_map(FactArgs& a, int64_t n_rows) {
    const EncodeTiledFn enc = encode_tiled_fn();
    if (!enc) return cudaErrorNotSupported;
    const int64_t words = (a.n_valid * a.E + 3) / 4;
    if (a.Lw < 4 || a.Lw > kFactMaxLw || a.Lw % fact_lw_align(a.Lw) != 0 ||
        (a.box_rows > 1 && (a.rb / 4 > 256 || a.rb % 128 != 0 || !a.bbase || a.CC % a.box_rows != 0)) ||
        (a.box_rows != 8 && a.box_rows != 4 && a.box_rows != 1) ||
        (reinterpret_cast<uintptr_t>(a.in) & 15u) != 0 || a.pitch_bytes % 16 != 0 || words * 4 > a.pitch_bytes ||
        n_rows < 1)
        return cudaErrorInvalidValue;
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(words), static_cast<cuuint64_t>(n_rows)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(a.pitch_bytes)};
    // a box of box_rows channel rows of rb / 4 words, or one row's piece of Lw / fact_boxes(Lw) words
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(a.box_rows > 1 ? a.rb / 4 : a.Lw / fact_boxes(a.Lw)),
                               static_cast<cuuint32_t>(a.box_rows)};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(&a.tmap, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<uint8_t*>(a.in), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

bool fact_has_width(int variant, int E, bool part) {
    if (variant < 0 || variant >= num_fact_variants() || (E != 1 && E != 2)) return false;
    return (part ? kFEntries[variant].part[E - 1] : kFEntries[variant].fn[E - 1]) != nullptr;
}

cudaError_t launch_dedisp_fact(int variant, const FactArgs& a, size_t smem, cudaStream_t s) {
    if (!fact_has_width(variant, a.E, false)) return cudaErrorInvalidValue;
    const FEntry& e = kFEntries[variant];
    const FactFn fn = e.fn[a.E - 1];
    cudaError_t err = allow_dynamic_smem(reinterpret_cast<const void*>(fn), smem);
    if (err != cudaSuccess) return err;
    const int T = e.v.tile(), BD = e.v.bd();
    dim3 grid((a.n_out + T - 1) / T, (a.n_dm + BD - 1) / BD, a.n_sb);
    fn<<<grid, e.v.threads(), smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sbf_part_fact(int variant, const FactArgs& a, size_t smem, int n_tab, cudaStream_t s) {
    if (!fact_has_width(variant, a.E, true)) return cudaErrorInvalidValue;
    const FEntry& e = kFEntries[variant];
    const FactFn fn = e.part[a.E - 1];
    const int T = e.v.tile(), BD = e.v.bd();
    if (a.i0 % BD != 0 || a.n_slab <= 0 || !a.P || !a.sseg) return cudaErrorInvalidValue;
    cudaError_t err = allow_dynamic_smem(reinterpret_cast<const void*>(fn), smem);
    if (err != cudaSuccess) return err;
    dim3 grid((a.n_out + T - 1) / T, (a.n_slab + BD - 1) / BD, n_tab);
    fn<<<grid, e.v.threads(), smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace fdd
