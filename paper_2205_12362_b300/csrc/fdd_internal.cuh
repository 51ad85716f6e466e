// fdd_internal.cuh -- declarations shared by the library's own .cu files.
// Not installed; the public interface is include/fdd.h.
#pragma once

#include <cstdint>
#include <string>
#include <cuda.h>  // CUtensorMap (the tensor-map encoder is reached through the runtime's entry-point query)
#include <cuda_runtime.h>

#include "fdd.h"

namespace fdd {

// Raise a kernel's dynamic shared-memory limit to at least smem bytes; never lowers it.  One kernel
// launched with different sizes (one instantiation serves several DM ranges) keeps a limit that covers
// every size asked so far, so a CUDA graph node captured with a larger request than a later launch's
// still passes the launch check when it is launched again on its own.
cudaError_t allow_dynamic_smem(const void* fn, size_t smem);

// Workspace bytes of a plain (not batched) search: fdd_workspace_size without the second lane of
// SB-factored scratch that batched searches use.
size_t plain_workspace_bytes(const fdd_plan* plan, int64_t n_in, int64_t n_out, bool with_series);

// ---------------------------------------------------------------------------
// Dedispersion kernel variants (template instantiations of k_dedisp).
//   E     bytes per input sample: 1 = raw uint8 filterbank, 2 = uint16 sums
//         written by the downsampler
//   NW    32-bit words per lane per DM trial (a lane covers NW * 4/E samples)
//   DPW   DM trials per warp
//   WARPS warps per block; the block covers BD = WARPS * DPW trials and
//         T = 32 * NW * (4/E) output samples
//   MAXIT 16-byte staging chunks per thread per channel stage (register
//         budget of the software pipeline)
struct DedispVariant {
    int E, NW, DPW, WARPS, MAXIT;
    int bd() const { return WARPS * DPW; }
    int tile() const { return 32 * NW * (4 / E); }
    int threads() const { return WARPS * 32; }
};

int num_dedisp_variants();
const DedispVariant& dedisp_variant(int idx);

struct DedispArgs {
    const uint8_t* in;          // row (tab, c) starts at in + (tab * n_chan + c) * pitch_bytes
    int64_t pitch_bytes;        // multiple of 16
    int64_t n_valid;            // valid samples per row (elements of E bytes)
    const int16_t* sb_map;      // [n_sb][n_chan]
    const int32_t* base;        // [n_blk][n_chan]: first staged sample of (DM block, channel), aligned to 16/E
    const int32_t* off;         // [n_blk][n_chan][BD]: byte offset of trial (i, c) inside its channel slot
    int32_t* series;            // [n_sb][n_dm][n_out]
    unsigned long long* stat;   // [n_sb * n_dm][2]: sum S, sum S^2
    int32_t n_chan;
    int32_t n_dm;
    int32_t n_out;              // outputs per series row (the row stride)
    int32_t n_emit;             // outputs written and counted in the moments: t < n_emit <= n_out
    int32_t n_sb;
    int32_t Lw;                 // 32-bit words per staged copy row
    int32_t CC;                 // channels per smem stage (divides 256 when E == 1)
    // two-step subband mode, second step: DM block blk reads its rows coarse_stride bytes further per
    // coarse block (blk / blk_per_coarse); 0 = off
    int32_t blk_per_coarse;
    int64_t coarse_stride;
};

// Shared-memory bytes of one dedispersion block.
size_t dedisp_smem_bytes(const DedispVariant& v, int Lw, int CC);
// Whether channel-stage size CC fits variant v's staging registers, offset
// prefetch and the shared-memory budget for rows of Lw words.
bool dedisp_cc_ok(const DedispVariant& v, int Lw, int CC, size_t smem_budget);
cudaError_t launch_dedisp(int variant, const DedispArgs& a, cudaStream_t s);

// ---------------------------------------------------------------------------
// Pattern-factored dedispersion (k_dedisp_fact.cu; tables from fdd_fact.cu).
//   G     channels per group; NW, DPW, WARPS as above; samples per word are
//         16-bit pattern partials, so T = 64 * NW.  Raw rows are staged by
//         TMA (one unshifted copy per channel, double-buffered), so there is
//         no staging-register budget.
struct FactVariant {
    int G, NW, DPW, WARPS;
    int PB = 1;  // pattern-row buffers: 2 = stage s+1's rows are built while stage s accumulates
                 // (one block barrier per stage instead of two)
    int bd() const { return WARPS * DPW; }
    int tile() const { return 64 * NW; }
    int threads() const { return WARPS * 32; }
    int desc_ints() const { return (3 + G + 3) / 4 * 4; }
};
// Staged raw rows (32-bit words) travel as fact_boxes(Lw) TMA boxes of
// Lw / fact_boxes(Lw) words (at most 256); the table builder rounds Lw to a
// multiple of fact_lw_align(Lw) so every box is whole and starts on a
// 16-byte global and a 128-byte shared-memory boundary.
constexpr int kFactMaxLw = 1024;
__host__ __device__ inline int fact_boxes(int Lw) { return (Lw + 255) / 256; }
__host__ __device__ inline int fact_lw_align(int Lw) { return fact_boxes(Lw) == 1 ? 4 : 32 * fact_boxes(Lw); }

struct FactArgs {
    CUtensorMap tmap;           // the input as a 2-D uint32 tensor (words of a row, rows); encode_fact_map
    unsigned int* status;       // device status word: bit 0 set if a tile wait gave up
    const uint8_t* in;          // raw uint8 rows (tab, c) at in + (tab * n_chan + c) * pitch_bytes
    int64_t pitch_bytes;
    int64_t n_valid;            // valid samples per row
    int32_t E;                  // bytes per sample: 1 (raw rows) or 2 (downsampled rows)
    int32_t fold_ch;            // channels summed in the 16-bit lanes between folds (256 / D)
    const int16_t* sb_map;      // [n_sb][n_chan]
    const int32_t* base;        // [n_blk][n_chan]
    const int32_t* goff;        // [n_blk][n_groups][BD]
    const int32_t* pdesc;       // pattern-row descriptors
    const int32_t* pd_idx;      // [n_blk][n_stages][2]
    const int32_t* bbase;       // [n_blk][ceil(n_chan / box_rows)] first staged sample of each box
    int32_t box_rows;           // channels per TMA copy: 8 or 4 (bbase used, rows of rb / 4 words) or 1
    int32_t* series;            // [n_sb][n_dm][n_out]
    unsigned long long* stat;   // [n_sb * n_dm][2]
    int32_t n_chan, n_dm, n_out, n_sb;
    int32_t n_emit;             // outputs written and counted (<= n_out, the row stride)
    int32_t Lw, CC, n_stages, n_groups, pat_bytes;
    int32_t zero_off;           // shared-memory layout (bytes from the 128-aligned base): zero row,
    int32_t raw_off, rb;        //   raw slots (2 buffers x CC slots of rb bytes),
    int32_t pat_off;            //   pattern rows (PB buffers of pat_bytes), then stage offsets and
    int32_t desc_bytes;         //   descriptors (PB buffers of desc_bytes),
    int32_t bar_off;            //   two mbarriers
    // part mode (the partial sums of the SB-factored dedispersion, one TAB per block z): the
    // 16-bit sums of each channel segment go to P[tab][seg][i - i0][Np] instead of a series
    uint16_t* P;
    int64_t tab_stride, seg_stride;  // elements
    int32_t Np, i0, n_slab;          // row length; first trial and trials of the slab
    const int2* sseg;                // [n_stages]: {bit gl set = group gl closes its segment, segment of group 0}
};

int num_fact_variants();
const FactVariant& fact_variant(int idx);
bool fact_cc_ok(const FactVariant& v, int Lw, int CC, int max_desc);
// Fills a.tmap for a.in (n_rows rows of a.pitch_bytes, a.n_valid valid bytes each; box = one
// of the fact_boxes(a.Lw) pieces of a row).
cudaError_t encode_fact_map(FactArgs& a, int64_t n_rows);
// True if pattern-factored variant `variant` is built for E bytes per sample (plain or part mode).
bool fact_has_width(int variant, int E, bool part);
cudaError_t launch_dedisp_fact(int variant, const FactArgs& a, size_t smem, cudaStream_t s);
// Part mode of pattern-factored variant `variant`: a.P, a.i0 (a multiple of the variant's DM
// block), a.n_slab and a.sseg set; grid = tiles x DM blocks of the slab x n_tab.
cudaError_t launch_sbf_part_fact(int variant, const FactArgs& a, size_t smem, int n_tab, cudaStream_t s);

// cuTensorMapEncodeTiled, reached through the runtime's driver entry-point
// query (the library links only the runtime); nullptr if unavailable.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled_fn();

// ---------------------------------------------------------------------------
// SB-factored dedispersion (k_sbf.cu; tables and slab loop in fdd_sbf.cu).
// Channels are cut into segments on which every SB takes one TAB.  Pass 1
// ("part") dedisperses every TAB over every segment into 16-bit partial
// sums P[tab][seg][trial][t]; pass 2 ("comb") adds, for every SB, the
// partials of the TABs it selects.  The sums are the same integers as brute
// force, regrouped; partials of one TAB and segment serve every SB that
// selects that TAB there.  Both passes run per slab of consecutive DM trials
// so that P fits a bounded scratch buffer.
struct SbfPartArgs {
    const uint8_t* in;          // rows (tab, c) at in + (tab * n_chan + c) * pitch_bytes
    int64_t pitch_bytes;
    int64_t n_valid;            // valid samples per row
    const int32_t* base;        // brute-force tables of the variant's BD: [n_blk][n_chan]
    const int32_t* off;         // [n_blk][n_chan][BD]
    const int4* stages;         // [n_stages]: first channel, channels, first segment, segments
    const int2* segs;           // [n_seg]: first channel, channels
    uint16_t* P;                // slab partials [tab][seg][slab_rows][Np]
    int64_t tab_stride, seg_stride;  // elements
    int32_t Np;                 // row pitch of P (elements, multiple of 512)
    int32_t n_chan, n_dm, n_out, Lw, CC, n_stages;
    int32_t i0, n_slab;         // slab trials [i0, i0 + n_slab); i0 a multiple of BD
};

struct SbfCombArgs {
    CUtensorMap tmap;           // P as a 4-D tensor (t, trial, segment, TAB); filled by launch_sbf_comb
    unsigned int* status;       // device status word: bit 0 set if a tile wait gave up (kSpinLimit)
    const uint16_t* P;
    int64_t tab_stride, seg_stride;
    int32_t Np;
    const uint8_t* seg_tab;     // [n_sb][seg_pitch]: TAB SB s takes on segment u (seg_pitch % 8 == 0)
    int32_t seg_pitch;
    int32_t* series;            // this range: [n_sb][n_dm][n_out]
    unsigned long long* stat;   // this range: [n_sb * n_dm][2]
    int32_t n_sb, n_seg, n_dm, n_out, n_tab;
    int32_t n_emit;             // outputs written and counted (<= n_out, the row stride)
    int32_t i0, n_slab;
    int32_t flush;              // segments summed in 16-bit lanes between folds
    int32_t uc;                 // segments per shared-memory chunk (sbf_comb_uc)
};

// SB-factored variants: part kernels of the brute-force tile, then part kernels of the pattern-
// factored tile (sbf_fact_variant(idx) >= 0: that pattern-factored variant in part mode; its
// DedispVariant gives E = 1, the DM block and the tile, MAXIT = 0).
int num_sbf_variants();
const DedispVariant& sbf_variant(int idx);
int sbf_fact_variant(int idx);
// Shared memory of a part block: CC channel rows (4/E copies) + offsets.
size_t sbf_smem_bytes(const DedispVariant& v, int Lw, int CC);
bool sbf_cc_ok(const DedispVariant& v, int Lw, int CC, size_t smem_budget);
cudaError_t launch_sbf_part(int idx, const SbfPartArgs& a, int n_tab, cudaStream_t s);
// SBs handled by one comb block (the grid's z covers ceil(n_sb / this)).
int sbf_comb_sbs_per_block();
int sbf_comb_uc(int n_tab);
size_t sbf_comb_smem_bytes(int n_tab);
// Fills a.tmap from a.P and its strides (once per slab layout).
cudaError_t encode_comb_map(SbfCombArgs& a);
cudaError_t launch_sbf_comb(const SbfCombArgs& a, cudaStream_t s);

// ---------------------------------------------------------------------------
struct BoxcarArgs {
    const int32_t* series;              // [n_sb][n_dm][n_out] of this range
    const unsigned long long* stat;     // [n_sb * n_dm][2]
    fdd_candidate* cands;
    unsigned long long* count;
    int64_t cap;
    int64_t t_offset;                   // native sample of series sample 0
    double dm0, ddm;
    int32_t n_sb, n_dm, n_out;          // n_out: row stride of the series
    int32_t n_emit;                     // samples of each series searched (<= n_out)
    int32_t dm_index0;
    int32_t D;
    int32_t n_width;
    int32_t wmax;
    float thr;
    int32_t widths[FDD_MAX_WIDTHS];
    float inv_sqrt_w[FDD_MAX_WIDTHS];
};

cudaError_t launch_boxcar(const BoxcarArgs& a, cudaStream_t s);

// ---------------------------------------------------------------------------
// out[row][j] = sum_{k<D} in[row][offset + j*D + k], j < floor((n_in - offset) / D); 0 <= offset < n_in
// (offset = the bin phase of a window whose bins are aligned to stream sample 0).
cudaError_t launch_downsample(const uint8_t* in, int64_t n_rows, int64_t n_in, int64_t in_pitch,
                              int D, uint16_t* out, int64_t out_pitch, cudaStream_t s, int64_t offset = 0);

// ---------------------------------------------------------------------------
// Batched search: many chunks ("jobs") of one plan, every range, in one
// prep launch, one downsample launch, ONE persistent dedispersion launch and
// one boxcar launch.  Jobs travel as kernel parameters (graph-capturable,
// nothing to stage); per-range geometry lives in a plan-owned device table.
constexpr int kMaxBatchJobs = FDD_MAX_BATCH_JOBS;
constexpr int kMaxRanges = FDD_MAX_RANGES;
constexpr int kMaxDs = 4;  // distinct downsampling factors per plan (batched)

struct BatchRange {
    const int32_t* base;          // batched-variant tables of this range
    const int32_t* off;
    int32_t E, D, ds_index;       // ds_index: -1 = raw input, else index into job.ds
    int32_t n_dm, n_blk, n_tiles, n_out;
    int32_t Lw, CC;
    int64_t item_off;             // first work item of this range among the job's ranges of the same E
    int64_t series_elem_off;      // first series element of this range inside a job's series buffer
    int64_t series_off;           // first series index (sb*n_dm + i) of this range inside a job
    // S/N stage
    double dm0, ddm;
    int32_t dm_index0, n_width, wmax, pad_;
    int32_t widths[FDD_MAX_WIDTHS];
    float inv_sqrt_w[FDD_MAX_WIDTHS];
};

// Persistent SB-factored batch (k_sbf_persist.cu): ONE launch runs the part
// and comb tasks of every job, range and DM slab.  A job's scratch holds
// kSbfSlots slab buffers; its groups (range, slab) are issued in the order
// P0 P1 .. P(S-1) C0 PS C1 P(S+1) C2 ... (S = kSbfSlots), so every task
// depends only on tasks issued before it: comb tasks of group g wait for
// g's part tasks, part tasks of group g for the comb tasks of group g - S
// (the previous user of their buffer).
constexpr int kSbfSlots = 3;
struct SbfPersistRange {
    const int32_t* base;          // part tables of the persistent variant (BD trials per block)
    const int32_t* off;
    const int4* stages;
    const int2* segs;
    const uint8_t* seg_tab;       // [n_sb][seg_pitch]
    int64_t slot_elems;           // uint16 elements between slab buffers (the same for every range;
                                  //   >= n_tab * n_seg * slab * Np)
    int64_t series_elem_off;      // this range inside a job's series buffer
    int64_t stat_off;             // first series index of this range inside a job
    int32_t E, D, ds_index;       // ds_index: -1 raw input, else index into job.ds
    int32_t Lw, CC, n_stages;
    int32_t seg_pitch, n_seg, flush;
    int32_t n_dm, n_out, Np, slab;  // n_out: series row stride; slab: DM rows per slab buffer
    int32_t part_tiles, comb_tiles, sb_groups;
};
struct SbfPersistGroup {
    int32_t range, i0, n_slab;    // DM rows [i0, i0 + n_slab) of the range
    int32_t n_part, n_comb;       // tasks
    int32_t slot;                 // slab buffer
};
struct SbfPersistSeg {
    int32_t start;                // first task of this segment within a job's task list
    int32_t group;                // group (within the job)
    int32_t kind;                 // 0 part, 1 comb
    int32_t count;
};

struct BatchJob {
    const uint8_t* tabs;          // [n_tab][n_chan][tab_pitch]
    int64_t tab_pitch;
    int64_t n_in;
    uint16_t* ds[kMaxDs];         // downsampled copies, one per distinct D
    int64_t ds_pitch[kMaxDs];     // elements
    int32_t* series;              // all ranges, packed as the per-range search does
    unsigned long long* stat;     // [series_per_job][2]
    fdd_candidate* cands;
    int64_t cap;
    unsigned long long* count;
    int64_t t_offset;
    int32_t emit[kMaxRanges];     // outputs searched per range (<= the range's n_out, the row stride)
    int32_t ds_phase[kMaxDs];     // first input sample of the downsampling bins, per distinct D
    uint16_t* sbf_scratch;        // persistent SB-factored mode: the job's kSbfSlots slab buffers
};

struct BatchParams {
    const BatchRange* ranges;     // device [n_range]
    const int16_t* sb_map;
    unsigned long long* counter;  // [2] work-item counters (raw, downsampled), zeroed by the prep launch
    int64_t items_per_job_e[2];   // work items per job of raw / downsampled ranges
    int64_t series_per_job;
    int32_t n_range, n_jobs, n_sb, n_chan, n_tab, n_ds;
    int32_t ds_factor[kMaxDs];
    // persistent SB-factored mode (sp_ranges == nullptr otherwise)
    const SbfPersistRange* sp_ranges;  // device [n_range]
    const SbfPersistGroup* sp_groups;  // device [sp_n_groups]: one job's groups
    const SbfPersistSeg* sp_segs;      // device [sp_n_segs]: one job's task segments, in issue order
    unsigned int* sp_done;             // [n_jobs][sp_n_groups][2]: part / comb tasks done; zeroed by prep
    unsigned int* status;              // plan status word (bit 0: a bounded wait gave up)
    int32_t sp_n_groups, sp_n_segs;
    int64_t sp_tasks_per_job;
    BatchJob jobs[kMaxBatchJobs];
};

// Persistent dedispersion variants (instantiated for raw and downsampled
// samples; one launch per sample width present in the plan).
struct PersistentVariant {
    int NW, DPW, WARPS, MAXIT;
    int bd() const { return WARPS * DPW; }
    int threads() const { return WARPS * 32; }
    DedispVariant as(int E) const { return DedispVariant{E, NW, DPW, WARPS, MAXIT}; }
};
int num_persistent_variants();
const PersistentVariant& persistent_variant(int idx);
// Resident blocks per SM of persistent variant idx with `smem` bytes of dynamic shared memory.
cudaError_t persistent_occupancy(int idx, int E, size_t smem, int* blocks_per_sm);
cudaError_t launch_batch_prep(const BatchParams& p, cudaStream_t s);
cudaError_t launch_batch_downsample(const BatchParams& p, cudaStream_t s);
cudaError_t launch_dedisp_persistent(int idx, int E, const BatchParams& p, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_boxcar_batch(const BatchParams& p, int wmax_all, int n_width_max, float thr, cudaStream_t s);
// Persistent SB-factored batch: the part variant (one per sample width, BD trials, T samples),
// shared memory of a block, resident blocks per SM, launch.
DedispVariant sbf_persist_part_variant(int E);
size_t sbf_persist_smem_bytes(size_t part_smem_max, int n_tab);
cudaError_t sbf_persist_occupancy(size_t smem, int* blocks_per_sm);
cudaError_t launch_sbf_persist(const BatchParams& p, int grid, size_t smem, cudaStream_t s);
int sbf_persist_comb_sbs();       // SBs per comb task
int sbf_persist_comb_tile();      // output samples per comb task

// ---------------------------------------------------------------------------
// Library-internal helpers shared between host files.
bool plan_timing_enabled(const fdd_plan* plan);
void set_last_error(const std::string& msg);

}  // namespace fdd
