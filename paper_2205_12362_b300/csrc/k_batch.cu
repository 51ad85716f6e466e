// k_batch.cu -- kernels of the batched search: many chunks ("jobs") of one
// plan and all of its DM ranges in four launches (prep, downsample, one
// persistent dedispersion launch, boxcar).  Jobs arrive as kernel parameters
// (BatchParams), so the whole sequence can be captured in a CUDA graph.
//
// The persistent dedispersion kernels keep every SM busy across ranges of
// uneven length: resident blocks pull work items (job, range, SB, DM block,
// time tile) from an atomic counter.  One persistent launch serves all raw
// (uint8) ranges and one all downsampled (uint16) ranges, so each keeps the
// register budget of its own sample width.  Items of one
// (job, range, SB, time tile) differ only in DM block and are consecutive, so
// blocks running at the same time share staged input rows in L2.  Each item
// runs the same dedisp_tile as the per-range kernel, instantiated for raw
// (uint8) and downsampled (uint16) samples.
#include <algorithm>

#include "boxcar_series.cuh"
#include "boxcar_warp.cuh"
#include "dedisp_tile.cuh"
#include "downsample_chunk.cuh"

namespace fdd {

namespace {

__global__ void __launch_bounds__(256) k_batch_prep(const __grid_constant__ BatchParams p) {
    const BatchJob& J = p.jobs[blockIdx.y];
    const int64_t words = 2 * p.series_per_job;
    for (int64_t i = blockIdx.x * 256LL + threadIdx.x; i < words; i += 256LL * gridDim.x) J.stat[i] = 0ULL;
    if (p.sp_done) {  // task counters of the persistent SB-factored launch, this job's part
        const int64_t n = 2LL * p.sp_n_groups;
        unsigned int* d = p.sp_done + blockIdx.y * n;
        for (int64_t i = blockIdx.x * 256LL + threadIdx.x; i < n; i += 256LL * gridDim.x) d[i] = 0u;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *J.count = 0ULL;
        if (blockIdx.y == 0) {
            p.counter[0] = 0ULL;  // work items, raw ranges
            p.counter[1] = 0ULL;  // work items, downsampled ranges
            p.counter[2] = 0ULL;  // persistent SB-factored tasks
            p.counter[3] = 0ULL;  // persistent SB-factored abort flag
        }
    }
}

__global__ void __launch_bounds__(256) k_batch_downsample(const __grid_constant__ BatchParams p, int64_t rows) {
    const int job = blockIdx.z / p.n_ds, k = blockIdx.z - job * p.n_ds;
    const BatchJob& J = p.jobs[job];
    const int D = p.ds_factor[k];
    const int phase = J.ds_phase[k];
    const int64_t n_y = (J.n_in - phase) / D;
    const int64_t j0 = 8 * (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x);
    if (j0 >= n_y) return;
    for (int64_t row = blockIdx.y; row < rows; row += gridDim.y)
        detail::downsample_chunk(J.tabs + row * J.tab_pitch + phase, J.ds[k] + row * J.ds_pitch[k], n_y, D, j0);
}

// Every factor in {2, 4, 8} and every bin starting at the first input sample: one pass over the
// input.  Thread q reads bytes [8 DMAX q, 8 DMAX (q + 1)) of a row and writes every factor's bins
// in them: the D=2 sums as 16-bit lanes of one word per input word, each coarser factor from
// pairs of the next finer sums.
template <int DMAX>
__global__ void __launch_bounds__(256) k_batch_downsample_pow2(const __grid_constant__ BatchParams p, int64_t rows) {
    constexpr int NB = 8 * DMAX;  // input bytes per thread
    const BatchJob& J = p.jobs[blockIdx.z];
    const int64_t b0 = NB * (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x);
    if (b0 >= J.n_in) return;
    int k2 = -1, k4 = -1, k8 = -1;
    for (int k = 0; k < p.n_ds; k++) {
        if (p.ds_factor[k] == 2) k2 = k;
        if (p.ds_factor[k] == 4) k4 = k;
        if (p.ds_factor[k] == 8) k8 = k;
    }
    for (int64_t row = blockIdx.y; row < rows; row += gridDim.y) {
        const uint8_t* src = J.tabs + row * J.tab_pitch + b0;
        if (b0 + NB <= J.n_in) {
            uint32_t u2[2 * DMAX];  // D=2 sums, two per word
#pragma unroll
            for (int v = 0; v < DMAX / 2; v++) {
                const uint4 x = __ldg(reinterpret_cast<const uint4*>(src) + v);
                const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int e = 0; e < 4; e++) u2[4 * v + e] = (w[e] & 0x00FF00FFu) + ((w[e] >> 8) & 0x00FF00FFu);
            }
            if (k2 >= 0) {
                uint4* dst = reinterpret_cast<uint4*>(J.ds[k2] + row * J.ds_pitch[k2] + b0 / 2);
#pragma unroll
                for (int v = 0; v < DMAX / 2; v++)
                    dst[v] = make_uint4(u2[4 * v], u2[4 * v + 1], u2[4 * v + 2], u2[4 * v + 3]);
            }
            if constexpr (DMAX >= 4) {
                uint32_t u4[DMAX];
#pragma unroll
                for (int i = 0; i < DMAX; i++)
                    u4[i] = __byte_perm(u2[2 * i], u2[2 * i + 1], 0x5410) + __byte_perm(u2[2 * i], u2[2 * i + 1], 0x7632);
                if (k4 >= 0) {
                    uint4* dst = reinterpret_cast<uint4*>(J.ds[k4] + row * J.ds_pitch[k4] + b0 / 4);
#pragma unroll
                    for (int v = 0; v < DMAX / 4; v++)
                        dst[v] = make_uint4(u4[4 * v], u4[4 * v + 1], u4[4 * v + 2], u4[4 * v + 3]);
                }
                if constexpr (DMAX >= 8) {
                    uint32_t u8[DMAX / 2];
#pragma unroll
                    for (int i = 0; i < DMAX / 2; i++)
                        u8[i] = __byte_perm(u4[2 * i], u4[2 * i + 1], 0x5410) +
                                __byte_perm(u4[2 * i], u4[2 * i + 1], 0x7632);
                    if (k8 >= 0)
                        *reinterpret_cast<uint4*>(J.ds[k8] + row * J.ds_pitch[k8] + b0 / 8) =
                            make_uint4(u8[0], u8[1], u8[2], u8[3]);
                }
            }
        } else {
            // ragged end of the row: the complete bins of each factor, one by one
            for (int k = 0; k < p.n_ds; k++) {
                const int D = p.ds_factor[k];
                const int64_t n_y = J.n_in / D;
                uint16_t* dst = J.ds[k] + row * J.ds_pitch[k];
                for (int64_t j = b0 / D; j < (b0 + NB) / D && j < n_y; j++) {
                    uint32_t acc = 0;
                    for (int e = 0; e < D; e++) acc += src[j * D - b0 + e];
                    dst[j] = static_cast<uint16_t>(acc);
                }
            }
        }
    }
}

template <int E, int NW, int DPW, int WARPS, int MAXIT>
__global__ void __launch_bounds__(WARPS * 32) k_dedisp_persistent(const __grid_constant__ BatchParams p) {
    __shared__ unsigned long long s_item;
    const int64_t per_job = p.items_per_job_e[E - 1];
    const unsigned long long total = static_cast<unsigned long long>(per_job) * p.n_jobs;
    unsigned long long* counter = p.counter + (E - 1);
    for (;;) {
        __syncthreads();  // previous item's shared-memory reads are done
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1ULL);
        __syncthreads();
        const unsigned long long it = s_item;
        if (it >= total) break;
        const int job = static_cast<int>(it / per_job);
        int64_t rest = static_cast<int64_t>(it - static_cast<unsigned long long>(job) * per_job);
        int r = -1;  // last range of this sample width whose first item is <= rest
        for (int k = 0; k < p.n_range; k++)
            if (p.ranges[k].E == E && p.ranges[k].item_off <= rest) r = k;
        const BatchRange& R = p.ranges[r];
        rest -= R.item_off;
        const int blk = static_cast<int>(rest % R.n_blk);
        rest /= R.n_blk;
        const int tile = static_cast<int>(rest % R.n_tiles);
        const int sb = static_cast<int>(rest / R.n_tiles);
        const BatchJob& J = p.jobs[job];
        DedispArgs a;
        a.blk_per_coarse = 0;
        a.coarse_stride = 0;
        if (R.ds_index < 0) {
            a.in = J.tabs;
            a.pitch_bytes = J.tab_pitch;
        } else {
            a.in = reinterpret_cast<const uint8_t*>(J.ds[R.ds_index]);
            a.pitch_bytes = J.ds_pitch[R.ds_index] * 2;
        }
        a.n_valid = (J.n_in - (R.ds_index < 0 ? 0 : J.ds_phase[R.ds_index])) / R.D;
        a.sb_map = p.sb_map;
        a.base = R.base;
        a.off = R.off;
        a.series = J.series + R.series_elem_off;
        a.stat = J.stat + 2 * R.series_off;
        a.n_chan = p.n_chan;
        a.n_dm = R.n_dm;
        a.n_out = R.n_out;
        a.n_emit = J.emit[r];
        a.n_sb = p.n_sb;
        a.Lw = R.Lw;
        a.CC = R.CC;
        detail::dedisp_tile<E, NW, DPW, WARPS, MAXIT>(a, tile, blk, sb);
    }
}

__global__ void __launch_bounds__(detail::kThreads) k_boxcar_batch(const __grid_constant__ BatchParams p, const float thr) {
    const int64_t gq = blockIdx.x;
    const int job = static_cast<int>(gq / p.series_per_job);
    int64_t q = gq - static_cast<int64_t>(job) * p.series_per_job;
    int r = 0;
    while (r + 1 < p.n_range && q >= p.ranges[r + 1].series_off) r++;
    const BatchRange& R = p.ranges[r];
    q -= R.series_off;
    if (R.n_out == 0) return;
    const BatchJob& J = p.jobs[job];
    if (J.emit[r] <= 0) return;
    BoxcarArgs a;
    a.series = J.series + R.series_elem_off;
    a.stat = J.stat + 2 * R.series_off;
    a.cands = J.cands;
    a.count = J.count;
    a.cap = J.cap;
    a.t_offset = J.t_offset + (R.ds_index < 0 ? 0 : J.ds_phase[R.ds_index]);
    a.dm0 = R.dm0;
    a.ddm = R.ddm;
    a.n_sb = p.n_sb;
    a.n_dm = R.n_dm;
    a.n_out = R.n_out;
    a.n_emit = J.emit[r];
    a.dm_index0 = R.dm_index0;
    a.D = R.D;
    a.n_width = R.n_width;
    a.wmax = R.wmax;
    a.thr = thr;
    for (int k = 0; k < FDD_MAX_WIDTHS; k++) {
        a.widths[k] = R.widths[k];
        a.inv_sqrt_w[k] = R.inv_sqrt_w[k];
    }
    detail::boxcar_series(a, q);
}

// Warp-per-series boxcar over every series of every job (all widths <= 512).
template <int NWB>
__global__ void __launch_bounds__(detail::kBoxWarps * 32)
    k_boxcar_batch_warp(const __grid_constant__ BatchParams p, const float thr) {
    __shared__ uint32_t ring[detail::kBoxWarps][detail::kWarpRing];
    const int warp = threadIdx.x >> 5;
    const int64_t gq = static_cast<int64_t>(blockIdx.x) * detail::kBoxWarps + warp;
    if (gq >= static_cast<int64_t>(p.n_jobs) * p.series_per_job) return;  // warp-uniform
    const int job = static_cast<int>(gq / p.series_per_job);
    int64_t q = gq - static_cast<int64_t>(job) * p.series_per_job;
    int r = 0;
    while (r + 1 < p.n_range && q >= p.ranges[r + 1].series_off) r++;
    const BatchRange& R = p.ranges[r];
    q -= R.series_off;
    if (R.n_out == 0) return;
    const BatchJob& J = p.jobs[job];
    if (J.emit[r] <= 0) return;  // warp-uniform
    const int i = static_cast<int>(q % R.n_dm);
    detail::BoxSeries v;
    v.S = J.series + R.series_elem_off + q * R.n_out;
    v.stat = J.stat + 2 * (R.series_off + q);
    v.widths = R.widths;
    v.cands = J.cands;
    v.count = J.count;
    v.cap = J.cap;
    v.t_offset = J.t_offset + (R.ds_index < 0 ? 0 : J.ds_phase[R.ds_index]);
    v.dm = R.dm0 + static_cast<double>(i) * R.ddm;
    v.n = J.emit[r];
    v.n_width = R.n_width;
    v.sb = static_cast<int>(q / R.n_dm);
    v.dm_index = R.dm_index0 + i;
    v.D = R.D;
    v.thr = thr;
    detail::boxcar_series_warp<NWB>(v, ring[warp]);
}

using PersistentFn = void (*)(const BatchParams);

struct PEntry {
    PersistentVariant v;
    PersistentFn fn[2];  // raw (uint8) and downsampled (uint16) work items
};

#define FDD_P(NW, DPW, WARPS, MAXIT) \
    {{NW, DPW, WARPS, MAXIT}, {k_dedisp_persistent<1, NW, DPW, WARPS, MAXIT>, k_dedisp_persistent<2, NW, DPW, WARPS, MAXIT>}}
const PEntry kPEntries[] = {
    FDD_P(4, 2, 16, 4),  // BD 32, T 512 (uint8) / 256 (uint16), 512 threads
    FDD_P(2, 4, 16, 4),  // BD 64, T 256 / 128, 512 threads
    FDD_P(4, 2, 8, 4),   // BD 16, T 512 / 256, 256 threads
    FDD_P(2, 4, 8, 4),   // BD 32, T 256 / 128, 256 threads
    FDD_P(4, 1, 16, 4),  // BD 16, T 512 / 256, 512 threads
};
#undef FDD_P

}  // namespace

int num_persistent_variants() { return static_cast<int>(sizeof(kPEntries) / sizeof(kPEntries[0])); }

const PersistentVariant& persistent_variant(int idx) { return kPEntries[idx].v; }

cudaError_t persistent_occupancy(int idx, int E, size_t smem, int* blocks_per_sm) {
    const PEntry& e = kPEntries[idx];
    cudaError_t err = allow_dynamic_smem(reinterpret_cast<const void*>(e.fn[E - 1]), smem);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, e.fn[E - 1], e.v.threads(), smem);
}

cudaError_t launch_batch_prep(const BatchParams& p, cudaStream_t s) {
    const int64_t words = 2 * p.series_per_job;
    const int gx = static_cast<int>(std::min<int64_t>(1024, std::max<int64_t>(1, (words + 4095) / 4096)));
    k_batch_prep<<<dim3(gx, p.n_jobs), 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_batch_downsample(const BatchParams& p, cudaStream_t s) {
    if (p.n_ds == 0) return cudaSuccess;
    int64_t n_in_max = 0;
    int d_min = 1 << 30;
    for (int j = 0; j < p.n_jobs; j++) n_in_max = std::max<int64_t>(n_in_max, p.jobs[j].n_in);
    for (int k = 0; k < p.n_ds; k++) d_min = std::min(d_min, p.ds_factor[k]);
    const int64_t n_y = n_in_max / d_min;
    if (n_y == 0) return cudaSuccess;
    const int64_t rows = static_cast<int64_t>(p.n_tab) * p.n_chan;
    // one pass for factors in {2, 4, 8} with bins from the first sample and 16-byte aligned rows
    bool pow2 = true;
    int d_max = 0;
    for (int k = 0; k < p.n_ds; k++) {
        const int D = p.ds_factor[k];
        pow2 = pow2 && (D == 2 || D == 4 || D == 8);
        d_max = std::max(d_max, D);
        for (int j = 0; j < p.n_jobs && pow2; j++)
            pow2 = p.jobs[j].ds_phase[k] == 0 && p.jobs[j].ds_pitch[k] % 8 == 0 && p.jobs[j].tab_pitch % 16 == 0 &&
                   (reinterpret_cast<uintptr_t>(p.jobs[j].ds[k]) & 15u) == 0 &&
                   (reinterpret_cast<uintptr_t>(p.jobs[j].tabs) & 15u) == 0;
    }
    if (pow2) {
        const unsigned gy = static_cast<unsigned>(std::min<int64_t>(rows, 65535));
        const int64_t per_block = 8LL * d_max * 256;
        dim3 grid(static_cast<unsigned>((n_in_max + per_block - 1) / per_block), gy, static_cast<unsigned>(p.n_jobs));
        if (d_max == 2)
            k_batch_downsample_pow2<2><<<grid, 256, 0, s>>>(p, rows);
        else if (d_max == 4)
            k_batch_downsample_pow2<4><<<grid, 256, 0, s>>>(p, rows);
        else
            k_batch_downsample_pow2<8><<<grid, 256, 0, s>>>(p, rows);
        return cudaGetLastError();
    }
    dim3 grid(static_cast<unsigned>((n_y + 8 * 256 - 1) / (8 * 256)),
              static_cast<unsigned>(std::min<int64_t>(rows, 65535)), static_cast<unsigned>(p.n_jobs * p.n_ds));
    k_batch_downsample<<<grid, 256, 0, s>>>(p, rows);
    return cudaGetLastError();
}

cudaError_t launch_dedisp_persistent(int idx, int E, const BatchParams& p, int grid, size_t smem, cudaStream_t s) {
    const PEntry& e = kPEntries[idx];
    cudaError_t err = allow_dynamic_smem(reinterpret_cast<const void*>(e.fn[E - 1]), smem);
    if (err != cudaSuccess) return err;
    e.fn[E - 1]<<<grid, e.v.threads(), smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_boxcar_batch(const BatchParams& p, int wmax_all, int n_width_max, float thr, cudaStream_t s) {
    const long long blocks = static_cast<long long>(p.n_jobs) * p.series_per_job;
    if (blocks == 0) return cudaSuccess;
    if (wmax_all <= detail::kWarpCS) {
        const unsigned wb = static_cast<unsigned>((blocks + detail::kBoxWarps - 1) / detail::kBoxWarps);
        if (n_width_max <= 4)
            k_boxcar_batch_warp<4><<<wb, detail::kBoxWarps * 32, 0, s>>>(p, thr);
        else if (n_width_max <= 8)
            k_boxcar_batch_warp<8><<<wb, detail::kBoxWarps * 32, 0, s>>>(p, thr);
        else
            k_boxcar_batch_warp<16><<<wb, detail::kBoxWarps * 32, 0, s>>>(p, thr);
        return cudaGetLastError();
    }
    const size_t smem = detail::boxcar_smem_bytes(wmax_all);
    k_boxcar_batch<<<static_cast<unsigned>(blocks), detail::kThreads, smem, s>>>(p, thr);
    return cudaGetLastError();
}

}  // namespace fdd
