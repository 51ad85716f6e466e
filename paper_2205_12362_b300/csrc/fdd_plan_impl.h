// fdd_plan_impl.h -- host-side plan state shared by the library's host files
// (fdd_plan.cu: plans, per-range search, tuner; fdd_batch.cu: batched search
// and graphs).  Not installed.
#pragma once

#include <string>
#include <vector>

#include "fdd_internal.cuh"

struct RangeState {
    double dm0 = 0, ddm = 0;
    int32_t n_dm = 0, D = 1, n_width = 0;
    int32_t widths[FDD_MAX_WIDTHS] = {};
    int32_t wmax = 1;
    int32_t dm_index0 = 0;
    int32_t dmax = 0;                 // largest delay, range samples
    std::vector<int32_t> delay;       // [n_dm][n_chan]
    // per-range launch: kernel configuration and its device tables
    int variant = -1;
    int32_t Lw = 0, CC = 0;
    float tuned_ms = 0.f;
    int32_t* d_off = nullptr;         // [n_blk][n_chan][BD]
    int32_t* d_base = nullptr;        // [n_blk][n_chan]
    // pattern-factored kernel (fact >= 0 selects it instead of `variant`)
    int fact = -1;
    int32_t f_CC = 0, f_Lw = 0, f_pat_bytes = 0, f_n_stages = 0, f_n_groups = 0;
    int32_t f_zero_off = 0, f_raw_off = 0, f_rb = 0, f_pat_off = 0, f_bar_off = 0, f_desc_bytes = 0, f_box_rows = 1;
    int32_t* d_fbbase = nullptr;      // [n_blk][ceil(n_chan / box_rows)] first staged sample of each box
    float f_work_ratio = 1.f;         // adds of the factored kernel per brute-force add
    size_t f_smem = 0;
    int32_t* d_fbase = nullptr;
    int32_t* d_goff = nullptr;
    int32_t* d_pdesc = nullptr;
    int32_t* d_pdidx = nullptr;
    // SB-factored kernel (sbf >= 0 selects it); segments are plan geometry
    std::vector<int2> segs;           // segments on which every SB keeps one TAB, cut at 16 channels (scratch sizing)
    int32_t seg_maxlen = 0;
    int32_t s_n_seg = 0;              // segments of the configured SB-factored kernel (cut at its CC)
    int2* d_segs = nullptr;           // configured segments
    uint8_t* d_segtab = nullptr;      // [n_sb][seg_pitch]
    int32_t seg_pitch = 0;
    int sbf = -1;
    int32_t s_CC = 0, s_Lw = 0, s_n_stages = 0, s_flush = 1;
    float s_work_ratio = 1.f;
    int32_t* d_sbase = nullptr;
    int32_t* d_soff = nullptr;
    int4* d_sstages = nullptr;
    // SB-factored with pattern-factored partial sums (s_fact >= 0: that pattern-factored variant in
    // part mode; its tables in d_fbase ... d_pdidx and the f_* layout, per stage d_fsseg)
    int s_fact = -1;
    int2* d_fsseg = nullptr;
    // two-step subband mode (approximate; sub_G > 0 selects it for fdd_search)
    int32_t sub_G = 0, sub_K = 0, sub_n = 0, sub_nq = 0;   // channels per subband, fine trials per coarse DM
    int32_t sub_d1max = 0, sub_d2max = 0, sub_dmax_exact = 0;
    int sub_pv = -1, sub_bv = -1;                          // step-1 (SB-factored part) / step-2 (brute E=2) variants
    int32_t sub_pCC = 0, sub_pLw = 0, sub_pstages = 0, sub_bCC = 0, sub_bLw = 0;
    int32_t* d_sub_pbase = nullptr;
    int32_t* d_sub_poff = nullptr;
    int4* d_sub_pstages = nullptr;
    int2* d_sub_psegs = nullptr;
    int32_t* d_sub_bbase = nullptr;
    int32_t* d_sub_boff = nullptr;
    int16_t* d_sub_sbmap = nullptr;                       // [n_sb][sub_n]
};

// Device tables of one range for the batched persistent kernel.
struct BatchRangeTables {
    int32_t Lw = 0, CC = 0;
    int32_t* d_off = nullptr;
    int32_t* d_base = nullptr;
};

// Two side streams and their fork / join events for one caller stream of batched searches (a
// caller stream gets its own pair, so batches enqueued on different streams stay independent).
struct LanePair {
    cudaStream_t caller = nullptr;
    cudaStream_t st[2] = {nullptr, nullptr};
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};  // fork (on the caller), join of lane 0, join of lane 1
};

struct BatchState {
    int variant = -1;                      // persistent kernel variant
    bool sbf = false;                      // every range through its SB-factored configuration instead
    bool sbp = false;                      // persistent SB-factored mode (one launch, k_sbf_persist.cu)
    fdd::SbfPersistRange* d_sp_ranges = nullptr;
    fdd::SbfPersistGroup* d_sp_groups = nullptr;
    fdd::SbfPersistSeg* d_sp_segs = nullptr;
    unsigned int* d_sp_done = nullptr;     // [FDD_MAX_BATCH_JOBS][groups][2]
    int32_t sp_n_groups = 0, sp_n_segs = 0;
    int64_t sp_tasks_per_job = 0;
    int sp_grid = 0;
    size_t sp_smem = 0;
    bool big_stages = false;               // channel stages sized to the full shared-memory budget
    int64_t n_out = -1;                    // chunk length the tables below were prepared for
    bool absolute = false;                 // prepared for windows whose bins are aligned to their stream
    std::vector<BatchRangeTables> tables;  // per range
    fdd::BatchRange* d_ranges = nullptr;   // device copy of the per-range descriptors
    std::vector<fdd::BatchRange> h_ranges;
    unsigned long long* d_counter = nullptr;  // work-item counters of the persistent launches
    int64_t items_per_job_e[2] = {0, 0};   // raw / downsampled work items per job
    int64_t series_per_job = 0;
    int grid_e[2] = {0, 0};                // resident blocks of each persistent launch
    size_t smem_e[2] = {0, 0};
    float tuned_ms = 0.f;
    std::vector<LanePair> lanes;           // per caller stream, created on first use, freed with the plan
};

struct fdd_plan {
    int32_t n_tab = 0, n_chan = 0, n_sb = 0;
    double t_samp = 0;
    float thr = 0;
    std::vector<double> freq;
    std::vector<int16_t> sb_map;
    int16_t* d_sb_map = nullptr;
    unsigned int* d_status = nullptr;  // device status word (fdd_plan_status)
    std::vector<RangeState> ranges;
    std::vector<int32_t> ds_factors;  // distinct D > 1
    int64_t max_delay_native = 0;
    int64_t n_dm_total = 0;
    size_t sbf_scratch_cap = size_t(4) << 30;  // SB-factored partial-sum scratch cap (fdd_plan_set_scratch_limit)
    int device = 0;
    // stage timing (fdd_plan_set_timing)
    bool timing = false;
    std::vector<cudaEvent_t> ev;          // 2 per stage, grown on demand
    std::vector<int32_t> st_kind, st_range;
    BatchState batch;
    int64_t last_launches = 0;            // kernels enqueued by the last search / batched search
};

namespace fdd {
namespace host {

// Cold-plasma dispersion constant, s MHz^2 / (pc cm^-3).  The paper gives no
// value; 4148.808 is the standard constant.
constexpr double kDispersionConstant = 4148.808;
constexpr size_t kSmemBudget = 200 * 1024;   // per block; the tuner weighs occupancy by timing
constexpr size_t kDefaultSmem = 100 * 1024;  // untuned default: leave room for two blocks per SM

int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
size_t align_up(size_t x, size_t a);

// Stage timing (fdd_plan_set_timing): an event pair per enqueued kernel.
// Kinds: 0 downsample, 1 dedispersion, 2 boxcar/threshold, 3 batch prep.
void stage_reset(fdd_plan* plan);
cudaError_t stage_begin(fdd_plan* plan, int kind, int range, cudaStream_t s);
cudaError_t stage_end(fdd_plan* plan, cudaStream_t s);

struct HostTables {
    std::vector<int32_t> base;  // [n_blk][n_chan]
    std::vector<int32_t> off;   // [n_blk][n_chan][BD]
    int32_t Lw = 0;
};
HostTables build_tables(const fdd_plan* p, const RangeState& r, const DedispVariant& v);
int upload_tables(int32_t** d_off, int32_t** d_base, const HostTables& h);
int pick_cc(const DedispVariant& v, int Lw);

struct FactTables {
    std::vector<int32_t> base, goff, pdesc, pd_idx;
    // Raw rows travel as TMA boxes of box_rows consecutive channels (8 or 4 where the block's channels
    // are consecutive tensor rows -- one TAB per block, or a one-TAB plan -- and the layout allows,
    // else 1) of rb / 4 words: box k of DM block b starts at sample bbase[b][k], the least staged start
    // of its channels, and each channel's row lands in its own slot, shifted by its start's distance.
    std::vector<int32_t> bbase;
    int32_t box_rows = 1;
    int32_t Lw = 0, pat_bytes = 0, n_groups = 0, n_stages = 0, desc_ints = 0;
    int32_t max_desc = 0;  // most pattern rows of one (block, stage)
    int32_t zero_off = 0, raw_off = 0, rb = 0, pat_off = 0, bar_off = 0;  // shared-memory layout (bytes)
    int32_t desc_bytes = 0, pat_bufs = 1;  // one descriptor buffer; pattern-row (and descriptor) buffers
    double work_ratio = 1.0;  // (pattern-build adds + per-trial adds) / brute-force adds, per time tile
    size_t smem_bytes = 0;
};
// Tables of the pattern-factored kernel for range r, variant v and CC
// channels per stage (Lw < 0: does not fit).
FactTables build_fact_tables(const fdd_plan* p, const RangeState& r, const FactVariant& v, int CC,
                             bool consecutive_rows);

struct Layout {
    size_t sbf = 0, sbf_bytes = 0;  // scratch of the SB-factored kernel's partial sums (every lane)
    size_t sbf_lane_bytes = 0;      // one lane of it (lane k starts at sbf + k * sbf_lane_bytes)
    int sbf_lanes = 1;
    size_t series = 0, series_bytes = 0;
    size_t stat = 0, stat_bytes = 0;
    std::vector<size_t> series_r;   // element offset of range r inside the series buffer
    std::vector<size_t> stat_r;     // series-index offset of range r inside the stat buffer
    std::vector<size_t> ds_off;     // per distinct D (plan order)
    std::vector<int64_t> ds_pitch;  // uint16 elements
    size_t total = 0;
};
// Series rows are floor(n_out / D_r) long (bins from input sample 0), or
// ceil(n_out / D_r) in a window whose bins are aligned to its stream
// (`absolute`), which holds one bin more when its phase allows.
// Lanes of the SB-factored scratch: a batched search runs its heaviest range in lane 0 and the other
// ranges in lane 1 on a second stream, at the same time (2 lanes for plans with two or more ranges and
// SBs); plain searches use lane 0 only.  lanes = 0: sbf_lanes(p).
int sbf_lanes(const fdd_plan* p);
Layout make_layout(const fdd_plan* p, int64_t n_in, int64_t n_out, bool with_series, bool absolute = false,
                   int lanes = 0);

// Downsampling bins of one search (Sec. "Downsampling").  Plain: bins from
// input sample 0, floor(n_out / D) outputs per range.  Absolute: input sample
// 0 is stream sample t0 and bins are aligned to stream sample 0; range r
// searches the bins starting in [t0, t0 + n_out), read from input sample
// phase = ceil(t0 / D) D - t0 on.
struct Bins {
    bool absolute = false;
    std::vector<int32_t> stride, emit, phase;  // per range: row stride, outputs searched, first input sample
    std::vector<int32_t> ds_phase;             // per distinct D (plan order)
};
Bins search_bins(const fdd_plan* p, int64_t n_out, int64_t t0, bool absolute);
// Input samples an absolute-bin window of n_out outputs needs at any start:
// n_out + max_r (D_r (max delay_r + 1) - 1).
int64_t window_input_len(const fdd_plan* p, int64_t n_out);
// SB-factored kernel (fdd_sbf.cu).
constexpr size_t kSbfScratchMax = size_t(4) << 30;
std::vector<int2> sbf_segments(const fdd_plan* p, int D, int cap);
size_t sbf_scratch_bytes(const fdd_plan* p, int64_t n_out);
int configure_sbf(fdd_plan* p, RangeState& r, int sv, int CC);
void free_sbf_tables(RangeState& r, bool geometry);
// Adds per brute-force add of the SB-factored kernel for range r.
double sbf_work_ratio(const fdd_plan* p, const RangeState& r);
// Enqueues 2 launches per DM slab; *launches (if given) receives their number.
cudaError_t launch_range_sbf(const fdd_plan* p, const RangeState& r, const fdd::DedispArgs& a, uint8_t* scratch,
                             size_t scratch_bytes, cudaStream_t s, int64_t* launches = nullptr);
// Two-step subband mode (fdd_subband.cu).
int configure_subband(fdd_plan* p, RangeState& r, int G, int K);
void free_subband_tables(RangeState& r);
size_t subband_scratch_bytes(const fdd_plan* p, int64_t n_out);
cudaError_t launch_range_subband(const fdd_plan* p, const RangeState& r, const fdd::DedispArgs& a, uint8_t* scratch,
                                 size_t scratch_bytes, cudaStream_t s, int64_t* launches);

// Global variant index / channels per stage of range r's current configuration,
// and re-applying such a pair (fdd_plan.cu).
int range_config_index(const RangeState& r);
int range_config_cc(const RangeState& r);
int restore_range_config(fdd_plan* p, RangeState& r, int variant, int CC);
// First SB-factored variant that fits range r (CC = 0), configured; error if none.
int configure_sbf_default(fdd_plan* p, RangeState& r);

int check_search_args(const fdd_plan* plan, const uint8_t* d_tabs, int64_t n_in, int64_t pitch, int64_t n_out,
                      const void* d_workspace, const void* d_series, const Bins* bins = nullptr);
// Prepare the plan's batched search for n_out and a bin mode, keeping its
// (possibly tuned) configuration; nothing if already prepared so.
int batch_prepare_mode(fdd_plan* plan, int64_t n_out, bool absolute);
// The search of fdd_search (absolute = false) and fdd_search_window.
int search_impl(fdd_plan* plan, const uint8_t* d_tabs, int64_t n_in, int64_t pitch, int64_t n_out, int64_t t_offset,
                bool absolute, void* d_workspace, size_t workspace_bytes, fdd_candidate* d_cands, int64_t cap,
                uint64_t* d_count, int32_t* d_series, cudaStream_t s);

}  // namespace host
}  // namespace fdd
