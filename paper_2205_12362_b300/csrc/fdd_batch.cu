// fdd_batch.cu -- host side of the batched search and its CUDA graphs.
//
// A batch is up to FDD_MAX_BATCH_JOBS chunks ("jobs") of one plan with the
// same output length.  fdd_search_batch enqueues four launches whatever the
// number of jobs, ranges and SBs: prep (zero moments and counters),
// downsample (every job x every distinct D), ONE persistent dedispersion
// launch over every (job, range, SB, DM block, time tile), and one boxcar
// launch over every series.  Nothing is allocated or synchronised in the
// call once fdd_batch_prepare has run for the chunk length, so the sequence
// can be captured (fdd_graph_*).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <new>
#include <vector>

#include "fdd_plan_impl.h"

using namespace fdd::host;

namespace {

// Side streams of a plan's batched searches (freed with the plan, not on a re-prepare).
void free_lanes(BatchState& b) {
    for (LanePair& lp : b.lanes) {
        for (cudaStream_t st : lp.st)
            if (st) cudaStreamDestroy(st);
        for (cudaEvent_t ev : lp.ev)
            if (ev) cudaEventDestroy(ev);
    }
    b.lanes.clear();
}

std::mutex g_lanes_mu;  // guards BatchState::lanes (caller streams may enqueue from several host threads)

// The side-stream pair of caller stream s (copied to *out), created on first use; false if it cannot be
// created (the launches then stay on s, which is correct: the lanes' scratch regions are disjoint).
bool lanes_for(fdd_plan* p, cudaStream_t s, LanePair* out) {
    std::lock_guard<std::mutex> lock(g_lanes_mu);
    for (const LanePair& lp : p->batch.lanes)
        if (lp.caller == s) {
            *out = lp;
            return true;
        }
    LanePair lp;
    lp.caller = s;
    bool ok = true;
    for (cudaStream_t& st : lp.st) ok = ok && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
    for (cudaEvent_t& ev : lp.ev) ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        for (cudaStream_t st : lp.st)
            if (st) cudaStreamDestroy(st);
        for (cudaEvent_t ev : lp.ev)
            if (ev) cudaEventDestroy(ev);
        cudaGetLastError();
        return false;
    }
    p->batch.lanes.push_back(lp);
    *out = lp;
    return true;
}

// Free the side-stream pair of caller stream s, if any (a graph's capture stream, when the graph goes).
void release_lanes(fdd_plan* p, cudaStream_t s) {
    std::lock_guard<std::mutex> lock(g_lanes_mu);
    std::vector<LanePair>& v = p->batch.lanes;
    for (size_t k = 0; k < v.size(); k++)
        if (v[k].caller == s) {
            for (cudaStream_t st : v[k].st)
                if (st) cudaStreamDestroy(st);
            for (cudaEvent_t ev : v[k].ev)
                if (ev) cudaEventDestroy(ev);
            v.erase(v.begin() + static_cast<std::ptrdiff_t>(k));
            return;
        }
}

void free_batch(BatchState& b) {
    for (BatchRangeTables& t : b.tables) {
        if (t.d_off) cudaFree(t.d_off);
        if (t.d_base) cudaFree(t.d_base);
    }
    b.tables.clear();
    if (b.d_ranges) cudaFree(b.d_ranges);
    b.d_ranges = nullptr;
    for (void** ptr : {reinterpret_cast<void**>(&b.d_sp_ranges), reinterpret_cast<void**>(&b.d_sp_groups),
                       reinterpret_cast<void**>(&b.d_sp_segs), reinterpret_cast<void**>(&b.d_sp_done)}) {
        if (*ptr) cudaFree(*ptr);
        *ptr = nullptr;
    }
    b.sp_n_groups = b.sp_n_segs = 0;
    b.sp_tasks_per_job = 0;
    b.sp_grid = 0;
    b.sp_smem = 0;
    b.n_out = -1;
}

// Index of the SB-factored variant the persistent kernel runs for sample width E.
int persistent_sbf_index(int E) {
    const fdd::DedispVariant want = fdd::sbf_persist_part_variant(E);
    for (int k = 0; k < fdd::num_sbf_variants(); k++) {
        const fdd::DedispVariant& v = fdd::sbf_variant(k);
        if (v.E == want.E && v.NW == want.NW && v.DPW == want.DPW && v.WARPS == want.WARPS && v.MAXIT == want.MAXIT)
            return k;
    }
    return -1;
}

template <typename T>
int upload_vec(T** dst, const std::vector<T>& v, const char* what) {
    cudaError_t e = cudaMalloc(dst, std::max<size_t>(v.size(), 1) * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (!v.empty() && (e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, what);
    return FDD_OK;
}

// Tables of the persistent SB-factored mode: per range the part tables of the
// persistent variant and the slab geometry (kSbfSlots slab buffers in a
// job's scratch), one job's groups (range, slab) and its task segments in
// issue order P(0) .. P(S-1) C(0) P(S) C(1) ... C(G-1).
int prepare_sb_persistent(fdd_plan* p, int64_t n_out, bool absolute, const Layout& L) {
    BatchState& b = p->batch;
    const Bins rows = search_bins(p, n_out, 0, absolute);
    std::vector<fdd::SbfPersistRange> hr(p->ranges.size());
    std::vector<fdd::SbfPersistGroup> groups;
    size_t part_smem = 0;
    // every range's slab buffers sit at the same kSbfSlots offsets of the scratch (slot k starts at
    // k * slot_elems elements, 1 KB aligned), so a range's layout never reaches into a slot another
    // range's group is still using
    const int64_t slot_elems = static_cast<int64_t>(L.sbf_lane_bytes) / 2 / fdd::kSbfSlots / 512 * 512;
    const int comb_sbs = fdd::sbf_persist_comb_sbs();
    const int comb_tile = fdd::sbf_persist_comb_tile();
    for (size_t ri = 0; ri < p->ranges.size(); ri++) {
        RangeState& r = p->ranges[ri];
        const int E = r.D == 1 ? 1 : 2;
        const int sv = persistent_sbf_index(E);
        if (sv < 0) return fail(FDD_ERR_UNSUPPORTED, "no SB-factored variant matches the persistent kernel");
        int rc;
        if (r.sbf != sv && (rc = configure_sbf(p, r, sv, r.sbf >= 0 ? r.s_CC : 0)) != FDD_OK &&
            (rc = configure_sbf(p, r, sv, 0)) != FDD_OK)
            return rc;
        const fdd::DedispVariant& v = fdd::sbf_variant(sv);
        part_smem = std::max(part_smem, fdd::sbf_smem_bytes(v, r.s_Lw, r.s_CC));
        const int64_t stride = rows.stride[ri];
        const int64_t Np = (std::max<int64_t>(stride, 1) + 511) / 512 * 512;
        const int64_t per_trial = static_cast<int64_t>(p->n_tab) * r.s_n_seg * Np * 2;
        int64_t slab = slot_elems / (per_trial / 2) / v.bd() * v.bd();
        slab = std::min<int64_t>(slab, (r.n_dm + v.bd() - 1) / v.bd() * v.bd());
        if (slab < v.bd())
            return fail(FDD_ERR_UNSUPPORTED, "scratch too small for three slabs of the persistent SB-factored mode");
        fdd::SbfPersistRange& R = hr[ri];
        R.base = r.d_sbase;
        R.off = r.d_soff;
        R.stages = r.d_sstages;
        R.segs = r.d_segs;
        R.seg_tab = r.d_segtab;
        R.slot_elems = slot_elems;
        R.series_elem_off = static_cast<int64_t>(L.series_r[ri]);
        R.stat_off = static_cast<int64_t>(L.stat_r[ri]);
        R.E = E;
        R.D = r.D;
        R.ds_index = (r.D == 1) ? -1
                                : static_cast<int32_t>(std::find(p->ds_factors.begin(), p->ds_factors.end(), r.D) -
                                                       p->ds_factors.begin());
        R.Lw = r.s_Lw;
        R.CC = r.s_CC;
        R.n_stages = r.s_n_stages;
        R.seg_pitch = r.seg_pitch;
        R.n_seg = r.s_n_seg;
        R.flush = r.s_flush;
        R.n_dm = r.n_dm;
        R.n_out = static_cast<int32_t>(stride);
        R.Np = static_cast<int32_t>(Np);
        R.slab = static_cast<int32_t>(slab);
        R.part_tiles = static_cast<int32_t>((stride + v.tile() - 1) / v.tile());
        R.comb_tiles = static_cast<int32_t>((stride + comb_tile - 1) / comb_tile);
        R.sb_groups = (p->n_sb + comb_sbs - 1) / comb_sbs;
        if (stride == 0) continue;
        for (int64_t i0 = 0; i0 < r.n_dm; i0 += slab) {
            fdd::SbfPersistGroup g{};
            g.range = static_cast<int32_t>(ri);
            g.i0 = static_cast<int32_t>(i0);
            g.n_slab = static_cast<int32_t>(std::min<int64_t>(slab, r.n_dm - i0));
            g.n_part = R.part_tiles * ((g.n_slab + v.bd() - 1) / v.bd()) * p->n_tab;
            g.n_comb = R.comb_tiles * g.n_slab * R.sb_groups;
            g.slot = static_cast<int32_t>(groups.size() % fdd::kSbfSlots);
            groups.push_back(g);
        }
    }
    const int G = static_cast<int>(groups.size());
    std::vector<fdd::SbfPersistSeg> segs;
    int64_t start = 0;
    auto add = [&](int g, int kind) {
        const int n = kind == 0 ? groups[g].n_part : groups[g].n_comb;
        segs.push_back(fdd::SbfPersistSeg{static_cast<int32_t>(start), g, kind, n});
        start += n;
    };
    for (int g = 0; g < G + fdd::kSbfSlots - 1; g++) {  // P(g) then C(g - (S-1))
        if (g < G) add(g, 0);
        if (g - (fdd::kSbfSlots - 1) >= 0) add(g - (fdd::kSbfSlots - 1), 1);
    }
    if (start >= (int64_t(1) << 31)) return fail(FDD_ERR_UNSUPPORTED, "too many persistent tasks per chunk");
    int rc;
    if ((rc = upload_vec(&b.d_sp_ranges, hr, "persistent ranges")) != FDD_OK) return rc;
    if ((rc = upload_vec(&b.d_sp_groups, groups, "persistent groups")) != FDD_OK) return rc;
    if ((rc = upload_vec(&b.d_sp_segs, segs, "persistent segments")) != FDD_OK) return rc;
    cudaError_t e = cudaMalloc(&b.d_sp_done, sizeof(unsigned int) * 2 * std::max(G, 1) * fdd::kMaxBatchJobs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(persistent counters)");
    b.sp_n_groups = G;
    b.sp_n_segs = static_cast<int32_t>(segs.size());
    b.sp_tasks_per_job = start;
    b.sp_smem = fdd::sbf_persist_smem_bytes(part_smem, p->n_tab);
    if (b.sp_smem > 227 * 1024) return fail(FDD_ERR_UNSUPPORTED, "persistent SB-factored kernel exceeds shared memory");
    int per_sm = 0, sms = 0;
    if ((e = fdd::sbf_persist_occupancy(b.sp_smem, &per_sm)) != cudaSuccess) return cuda_fail(e, "occupancy");
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device)) != cudaSuccess)
        return cuda_fail(e, "device attribute");
    if (per_sm < 1) return fail(FDD_ERR_UNSUPPORTED, "persistent SB-factored kernel does not fit on an SM");
    b.sp_grid = per_sm * sms;
    return FDD_OK;
}

int batch_eligible(const fdd_plan* p) {
    for (const RangeState& r : p->ranges)
        if (r.sub_G > 0)
            return fail(FDD_ERR_UNSUPPORTED, "batched search runs exact dedispersion only; a range is in subband mode");
    if (static_cast<int>(p->ranges.size()) > fdd::kMaxRanges)
        return fail(FDD_ERR_UNSUPPORTED, "batched search supports at most FDD_MAX_RANGES DM ranges");
    if (static_cast<int>(p->ds_factors.size()) > fdd::kMaxDs)
        return fail(FDD_ERR_UNSUPPORTED, "batched search supports at most 4 distinct downsampling factors");
    return FDD_OK;
}

// Build the batched-variant tables and the per-range descriptors for chunks
// of n_out native output samples.  Allocates and synchronises.
int prepare(fdd_plan* p, int64_t n_out, int variant, bool big_stages, bool absolute) {
    int rc = batch_eligible(p);
    if (rc != FDD_OK) return rc;
    if (variant < 0) {  // keep the current (possibly tuned) configuration
        variant = p->batch.sbp   ? FDD_BATCH_SB_PERSISTENT
                  : p->batch.sbf ? FDD_BATCH_SB_FACTORED
                                 : (p->batch.variant >= 0 ? p->batch.variant : 0);
        big_stages = p->batch.big_stages;
    }
    const bool sbp = variant == FDD_BATCH_SB_PERSISTENT;
    if (sbp && p->n_sb < 2) return fail(FDD_ERR_UNSUPPORTED, "the SB-factored kernels need at least two SBs");
    const bool sbf = variant == FDD_BATCH_SB_FACTORED || sbp;
    if (sbp) {
        variant = 0;  // the per-range descriptors below are still built (boxcar stage)
    } else if (sbf) {
        // every range through its SB-factored configuration (the first fitting one if it has none)
        for (RangeState& r : p->ranges)
            if (r.sbf < 0 && (rc = configure_sbf_default(p, r)) != FDD_OK) return rc;
        variant = 0;  // persistent tables are still built for the descriptors; no persistent launch runs
    } else if (variant >= fdd::num_persistent_variants()) {
        return fail(FDD_ERR_INVALID_ARG, "batch variant out of range");
    }
    BatchState& b = p->batch;
    free_batch(b);
    if (!b.d_counter) {
        cudaError_t e = cudaMalloc(&b.d_counter, 256);  // two counters used
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(batch counter)");
    }
    const fdd::PersistentVariant& pv = fdd::persistent_variant(variant);
    const Layout L = make_layout(p, 0, n_out, true, absolute);
    const Bins rows = search_bins(p, n_out, 0, absolute);  // row strides
    b.h_ranges.assign(p->ranges.size(), fdd::BatchRange{});
    b.tables.assign(p->ranges.size(), BatchRangeTables{});
    int64_t items[2] = {0, 0};
    size_t smem[2] = {0, 0};
    for (size_t ri = 0; ri < p->ranges.size(); ri++) {
        const RangeState& r = p->ranges[ri];
        const int E = (r.D == 1) ? 1 : 2;
        const fdd::DedispVariant v = pv.as(E);
        const HostTables h = build_tables(p, r, v);
        if (h.Lw < 0) return fail(FDD_ERR_UNSUPPORTED, "DM step too large for one block's staged rows");
        int CC = 0;
        if (big_stages)
            for (int cc : {64, 48, 32, 16, 8, 4, 2})
                if (fdd::dedisp_cc_ok(v, h.Lw, cc, kSmemBudget)) {
                    CC = cc;
                    break;
                }
        if (CC == 0) CC = pick_cc(v, h.Lw);
        if (CC == 0) return fail(FDD_ERR_UNSUPPORTED, "DM step too large for one block's staged rows");
        BatchRangeTables& t = b.tables[ri];
        if ((rc = upload_tables(&t.d_off, &t.d_base, h)) != FDD_OK) return rc;
        t.Lw = h.Lw;
        t.CC = CC;
        smem[E - 1] = std::max(smem[E - 1], fdd::dedisp_smem_bytes(v, h.Lw, CC));
        fdd::BatchRange& R = b.h_ranges[ri];
        R.base = t.d_base;
        R.off = t.d_off;
        R.E = E;
        R.D = r.D;
        R.ds_index = (r.D == 1) ? -1
                                : static_cast<int32_t>(std::find(p->ds_factors.begin(), p->ds_factors.end(), r.D) -
                                                       p->ds_factors.begin());
        R.n_dm = r.n_dm;
        R.n_blk = (r.n_dm + v.bd() - 1) / v.bd();
        R.n_out = rows.stride[ri];
        R.n_tiles = (R.n_out + v.tile() - 1) / v.tile();
        R.Lw = h.Lw;
        R.CC = CC;
        R.item_off = items[E - 1];
        if (!sbf) items[E - 1] += static_cast<int64_t>(p->n_sb) * R.n_blk * R.n_tiles;
        R.series_elem_off = static_cast<int64_t>(L.series_r[ri]);
        R.series_off = static_cast<int64_t>(L.stat_r[ri]);
        R.dm0 = r.dm0;
        R.ddm = r.ddm;
        R.dm_index0 = r.dm_index0;
        R.n_width = r.n_width;
        R.wmax = r.wmax;
        for (int k = 0; k < FDD_MAX_WIDTHS; k++) {
            R.widths[k] = r.widths[k];
            R.inv_sqrt_w[k] = k < r.n_width ? static_cast<float>(1.0 / std::sqrt(static_cast<double>(r.widths[k]))) : 0.f;
        }
    }
    cudaError_t e = cudaMalloc(&b.d_ranges, sizeof(fdd::BatchRange) * b.h_ranges.size());
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(batch ranges)");
    e = cudaMemcpy(b.d_ranges, b.h_ranges.data(), sizeof(fdd::BatchRange) * b.h_ranges.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(batch ranges)");
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device)) != cudaSuccess)
        return cuda_fail(e, "device attribute");
    for (int E = 1; E <= 2; E++) {
        b.grid_e[E - 1] = 0;
        b.smem_e[E - 1] = smem[E - 1];
        b.items_per_job_e[E - 1] = items[E - 1];
        if (items[E - 1] == 0) continue;
        int per_sm = 0;
        if ((e = fdd::persistent_occupancy(variant, E, smem[E - 1], &per_sm)) != cudaSuccess)
            return cuda_fail(e, "occupancy");
        if (per_sm < 1) return fail(FDD_ERR_UNSUPPORTED, "persistent kernel does not fit on an SM");
        b.grid_e[E - 1] = per_sm * sms;
    }
    if (sbp && (rc = prepare_sb_persistent(p, n_out, absolute, L)) != FDD_OK) {
        free_batch(b);
        return rc;
    }
    b.variant = variant;
    b.sbf = sbf && !sbp;
    b.sbp = sbp;
    b.big_stages = big_stages;
    b.series_per_job = static_cast<int64_t>(L.stat_bytes / (2 * sizeof(unsigned long long)));
    b.n_out = n_out;
    b.absolute = absolute;
    b.tuned_ms = 0.f;
    return FDD_OK;
}

// Bin mode of a batch: that of its first job (fill_params refuses a mix).
bool jobs_absolute(const fdd_job* jobs, int32_t n_jobs) { return jobs && n_jobs > 0 && jobs[0].bins_absolute != 0; }

// Per (job, range) arguments of the SB-factored launches of a batch.
struct SbfJobRange {
    fdd::DedispArgs a;
    uint8_t* scratch;
    size_t scratch_bytes;
    int range;
    int lane;  // 0: the caller's stream's first side stream (the heaviest range), 1: the second
};

struct BatchLaunch {
    fdd::BatchParams P;
    std::vector<SbfJobRange> sbf;
};

int fill_params(const fdd_plan* p, const fdd_job* jobs, int32_t n_jobs, int64_t n_out, BatchLaunch& BL) {
    fdd::BatchParams& P = BL.P;
    BL.sbf.clear();
    if (!jobs || n_jobs < 1 || n_jobs > fdd::kMaxBatchJobs) return fail(FDD_ERR_INVALID_ARG, "n_jobs outside [1, FDD_MAX_BATCH_JOBS]");
    const BatchState& b = p->batch;
    P = fdd::BatchParams{};
    P.ranges = b.d_ranges;
    P.sb_map = p->d_sb_map;
    P.counter = b.d_counter;
    P.items_per_job_e[0] = b.items_per_job_e[0];
    P.items_per_job_e[1] = b.items_per_job_e[1];
    P.series_per_job = b.series_per_job;
    P.n_range = static_cast<int32_t>(p->ranges.size());
    P.n_jobs = n_jobs;
    P.n_sb = p->n_sb;
    P.n_chan = p->n_chan;
    P.n_tab = p->n_tab;
    P.n_ds = static_cast<int32_t>(p->ds_factors.size());
    for (int k = 0; k < P.n_ds; k++) P.ds_factor[k] = p->ds_factors[k];
    P.status = p->d_status;
    if (b.sbp) {
        P.sp_ranges = b.d_sp_ranges;
        P.sp_groups = b.d_sp_groups;
        P.sp_segs = b.d_sp_segs;
        P.sp_done = b.d_sp_done;
        P.sp_n_groups = b.sp_n_groups;
        P.sp_n_segs = b.sp_n_segs;
        P.sp_tasks_per_job = b.sp_tasks_per_job;
    }
    for (int j = 0; j < n_jobs; j++) {
        const fdd_job& J = jobs[j];
        if (!J.d_count || (J.cap > 0 && !J.d_cands) || J.cap < 0) return fail(FDD_ERR_INVALID_ARG, "bad job output buffers");
        if ((J.bins_absolute != 0) != b.absolute)
            return fail(FDD_ERR_INVALID_ARG, "all jobs of a batch share one bin mode (bins_absolute)");
        if (b.absolute && J.t_offset_native < 0) return fail(FDD_ERR_INVALID_ARG, "window start must be >= 0");
        const Bins bins = search_bins(p, n_out, J.t_offset_native, b.absolute);
        // a window reads no more than fdd_window_sizes' n_in (its workspace is sized for that)
        const int64_t n_in = b.absolute ? std::min<int64_t>(J.n_in, window_input_len(p, n_out)) : J.n_in;
        int rc = check_search_args(p, J.d_tabs, n_in, J.pitch, n_out, J.d_workspace, J.d_series, &bins);
        if (rc != FDD_OK) return rc;
        const Layout L = make_layout(p, n_in, n_out, J.d_series == nullptr, b.absolute);
        if (J.workspace_bytes < L.total) return fail(FDD_ERR_WORKSPACE, "job workspace smaller than fdd_workspace_size()");
        uint8_t* ws = static_cast<uint8_t*>(J.d_workspace);
        fdd::BatchJob& B = P.jobs[j];
        B.tabs = J.d_tabs;
        B.tab_pitch = J.pitch;
        B.n_in = n_in;
        for (int k = 0; k < P.n_ds; k++) {
            B.ds[k] = reinterpret_cast<uint16_t*>(ws + L.ds_off[k]);
            B.ds_pitch[k] = L.ds_pitch[k];
        }
        B.series = J.d_series ? J.d_series : reinterpret_cast<int32_t*>(ws + L.series);
        B.stat = reinterpret_cast<unsigned long long*>(ws + L.stat);
        B.cands = J.d_cands;
        B.cap = J.cap;
        B.count = reinterpret_cast<unsigned long long*>(J.d_count);
        B.t_offset = J.t_offset_native;
        for (size_t ri = 0; ri < p->ranges.size(); ri++) B.emit[ri] = bins.emit[ri];
        for (size_t k = 0; k < bins.ds_phase.size(); k++) B.ds_phase[k] = bins.ds_phase[k];
        B.sbf_scratch = b.sbp ? reinterpret_cast<uint16_t*>(ws + L.sbf) : nullptr;
        if (!b.sbf) continue;
        // lanes: the range with the most trial-samples in lane 0, the others in lane 1
        size_t heavy = 0;
        for (size_t ri = 1; ri < p->ranges.size(); ri++)
            if (static_cast<int64_t>(p->ranges[ri].n_dm) * b.h_ranges[ri].n_out >
                static_cast<int64_t>(p->ranges[heavy].n_dm) * b.h_ranges[heavy].n_out)
                heavy = ri;
        for (size_t ri = 0; ri < p->ranges.size(); ri++) {
            const RangeState& r = p->ranges[ri];
            const fdd::BatchRange& R = b.h_ranges[ri];
            if (R.n_out == 0 || bins.emit[ri] <= 0) continue;
            SbfJobRange q{};
            q.range = static_cast<int>(ri);
            q.a.in = R.ds_index < 0 ? B.tabs : reinterpret_cast<const uint8_t*>(B.ds[R.ds_index]);
            q.a.pitch_bytes = R.ds_index < 0 ? B.tab_pitch : B.ds_pitch[R.ds_index] * 2;
            q.a.n_valid = (B.n_in - bins.phase[ri]) / r.D;
            q.a.series = B.series + R.series_elem_off;
            q.a.stat = B.stat + 2 * R.series_off;
            q.a.n_chan = p->n_chan;
            q.a.n_dm = r.n_dm;
            q.a.n_out = R.n_out;
            q.a.n_emit = bins.emit[ri];
            q.a.n_sb = p->n_sb;
            q.lane = L.sbf_lanes > 1 && ri != heavy ? 1 : 0;
            q.scratch = ws + L.sbf + static_cast<size_t>(q.lane) * L.sbf_lane_bytes;
            q.scratch_bytes = L.sbf_lane_bytes;
            BL.sbf.push_back(q);
        }
    }
    return FDD_OK;
}

// The launches of a batch, each kind inside a stage-timing event pair when
// the plan's timing is on (the events become graph nodes under capture).
int enqueue(fdd_plan* p, const BatchLaunch& BL, cudaStream_t s) {
    const fdd::BatchParams& P = BL.P;
    int64_t n_launch = 1 + (P.n_ds > 0 ? 1 : 0) + 1;  // prep, downsample, boxcar
    int wmax = 1, nwm = 1;
    for (const RangeState& r : p->ranges) {
        wmax = std::max(wmax, r.wmax);
        nwm = std::max(nwm, r.n_width);
    }
    stage_reset(p);
    cudaError_t e;
    if ((e = stage_begin(p, 3, -1, s)) != cudaSuccess) return cuda_fail(e, "timing event");
    if ((e = fdd::launch_batch_prep(P, s)) != cudaSuccess) return cuda_fail(e, "batch prep launch");
    if ((e = stage_end(p, s)) != cudaSuccess) return cuda_fail(e, "timing event");
    if (P.n_ds > 0) {
        if ((e = stage_begin(p, 0, -1, s)) != cudaSuccess) return cuda_fail(e, "timing event");
        if ((e = fdd::launch_batch_downsample(P, s)) != cudaSuccess) return cuda_fail(e, "batch downsample launch");
        if ((e = stage_end(p, s)) != cudaSuccess) return cuda_fail(e, "timing event");
    }
    if (p->batch.sbp && p->batch.sp_tasks_per_job > 0) {
        n_launch++;
        if ((e = stage_begin(p, 1, -1, s)) != cudaSuccess) return cuda_fail(e, "timing event");
        if ((e = fdd::launch_sbf_persist(P, p->batch.sp_grid, p->batch.sp_smem, s)) != cudaSuccess)
            return cuda_fail(e, "persistent SB-factored launch");
        if ((e = stage_end(p, s)) != cudaSuccess) return cuda_fail(e, "timing event");
    }
    if (!BL.sbf.empty()) {
        if ((e = stage_begin(p, 1, -1, s)) != cudaSuccess) return cuda_fail(e, "timing event");
        // two lanes: fork onto the caller stream's side streams, lane by lane in order, then join
        bool two = false;
        for (const SbfJobRange& q : BL.sbf) two = two || q.lane == 1;
        LanePair lanes;
        const LanePair* lp = two && lanes_for(p, s, &lanes) ? &lanes : nullptr;
        if (lp) {
            if ((e = cudaEventRecord(lp->ev[0], s)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(lp->st[0], lp->ev[0], 0)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(lp->st[1], lp->ev[0], 0)) != cudaSuccess)
                return cuda_fail(e, "lane fork");
        }
        for (const SbfJobRange& q : BL.sbf)
            if ((e = launch_range_sbf(p, p->ranges[q.range], q.a, q.scratch, q.scratch_bytes, lp ? lp->st[q.lane] : s,
                                      &n_launch)) != cudaSuccess)
                return cuda_fail(e, "SB-factored dedispersion launch");
        if (lp) {
            if ((e = cudaEventRecord(lp->ev[1], lp->st[0])) != cudaSuccess ||
                (e = cudaEventRecord(lp->ev[2], lp->st[1])) != cudaSuccess ||
                (e = cudaStreamWaitEvent(s, lp->ev[1], 0)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(s, lp->ev[2], 0)) != cudaSuccess)
                return cuda_fail(e, "lane join");
        }
        if ((e = stage_end(p, s)) != cudaSuccess) return cuda_fail(e, "timing event");
    }
    for (int E = 1; E <= 2; E++) {
        if (p->batch.items_per_job_e[E - 1] == 0) continue;
        n_launch++;
        if ((e = stage_begin(p, 1, -E, s)) != cudaSuccess) return cuda_fail(e, "timing event");
        if ((e = fdd::launch_dedisp_persistent(p->batch.variant, E, P, p->batch.grid_e[E - 1], p->batch.smem_e[E - 1],
                                               s)) != cudaSuccess)
            return cuda_fail(e, "persistent dedispersion launch");
        if ((e = stage_end(p, s)) != cudaSuccess) return cuda_fail(e, "timing event");
    }
    if ((e = stage_begin(p, 2, -1, s)) != cudaSuccess) return cuda_fail(e, "timing event");
    if ((e = fdd::launch_boxcar_batch(P, wmax, nwm, p->thr, s)) != cudaSuccess) return cuda_fail(e, "batch boxcar launch");
    if ((e = stage_end(p, s)) != cudaSuccess) return cuda_fail(e, "timing event");
    p->last_launches = n_launch;
    return FDD_OK;
}

}  // namespace

struct fdd_graph {
    fdd_plan* plan = nullptr;
    int32_t n_jobs = 0;
    int64_t n_out = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
};

namespace {

int capture(fdd_graph* g, const BatchLaunch& P, cudaGraph_t* out) {
    LanePair lanes;
    if (g->plan->batch.sbf) lanes_for(g->plan, g->cap_stream, &lanes);  // side streams exist before capture
    cudaError_t e = cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    // Events recorded under capture only order nodes; they carry no timestamps,
    // so stage timing is left out of graphs.
    const bool timing = g->plan->timing;
    g->plan->timing = false;
    const int rc = enqueue(g->plan, P, g->cap_stream);
    g->plan->timing = timing;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(g->cap_stream, &graph);
    if (rc != FDD_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    *out = graph;
    return FDD_OK;
}

}  // namespace

extern "C" {

int fdd_batch_prepare(fdd_plan* plan, int64_t n_out, int32_t variant) {
    if (!plan || n_out < 0) return fail(FDD_ERR_INVALID_ARG, "bad argument");
    return prepare(plan, n_out, variant, false, false);
}

int fdd_search_batch(fdd_plan* plan, const fdd_job* jobs, int32_t n_jobs, int64_t n_out, fdd_stream_t stream) {
    if (!plan || n_out < 0) return fail(FDD_ERR_INVALID_ARG, "bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool absolute = jobs_absolute(jobs, n_jobs);
    if (plan->batch.n_out != n_out || plan->batch.absolute != absolute) {
        cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(s, &st);
        if (st != cudaStreamCaptureStatusNone)
            return fail(FDD_ERR_INVALID_ARG, "prepare the batch for this n_out and bin mode before capturing");
        const int rc = prepare(plan, n_out, -1, false, absolute);
        if (rc != FDD_OK) return rc;
    }
    BatchLaunch P;
    const int rc = fill_params(plan, jobs, n_jobs, n_out, P);
    if (rc != FDD_OK) return rc;
    return enqueue(plan, P, s);
}

int fdd_batch_autotune(fdd_plan* plan, const fdd_job* jobs, int32_t n_jobs, int64_t n_out, int32_t reps,
                       fdd_stream_t stream) {
    if (!plan || n_out < 0) return fail(FDD_ERR_INVALID_ARG, "bad argument");
    if (reps < 1) reps = 1;
    const bool absolute = jobs_absolute(jobs, n_jobs);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t ev0, ev1;
    cudaError_t e;
    if ((e = cudaEventCreate(&ev0)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    if ((e = cudaEventCreate(&ev1)) != cudaSuccess) {
        cudaEventDestroy(ev0);
        return cuda_fail(e, "cudaEventCreate");
    }
    int best = -1;
    bool best_big = false;
    float best_ms = 1e30f;
    int rc = FDD_OK;
    for (int vb = 0; vb < 2 * fdd::num_persistent_variants(); vb++) {
        const int v = vb >> 1;
        const bool big = (vb & 1) != 0;
        if (prepare(plan, n_out, v, big, absolute) != FDD_OK) continue;  // variant does not fit this plan
        BatchLaunch P;
        if ((rc = fill_params(plan, jobs, n_jobs, n_out, P)) != FDD_OK) break;
        if ((rc = enqueue(plan, P, s)) != FDD_OK) break;  // warm-up
        cudaEventRecord(ev0, s);
        for (int k = 0; k < reps && rc == FDD_OK; k++) rc = enqueue(plan, P, s);
        cudaEventRecord(ev1, s);
        if (rc != FDD_OK) break;
        if ((e = cudaEventSynchronize(ev1)) != cudaSuccess) {
            rc = cuda_fail(e, "batch tuning");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        ms /= reps;
        if (std::getenv("FDD_TUNE_VERBOSE")) {
            const fdd::PersistentVariant& pv = fdd::persistent_variant(v);
            std::fprintf(stderr, "fdd batch tune: variant %d (bd %d threads %d) %s stages, grid %d/%d: %.4f ms\n", v,
                         pv.bd(), pv.threads(), big ? "large" : "default", plan->batch.grid_e[0],
                         plan->batch.grid_e[1], ms);
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = v;
            best_big = big;
        }
    }
    // SB-factored mode: per range, greedily, the fastest SB-factored variant (whole batch timed)
    if (rc == FDD_OK && plan->n_sb >= 2) {
        std::vector<std::pair<int, int>> saved;
        for (const RangeState& r : plan->ranges) saved.emplace_back(range_config_index(r), range_config_cc(r));
        bool ok = true;
        for (RangeState& r : plan->ranges)
            if (r.sbf < 0 && configure_sbf_default(plan, r) != FDD_OK) ok = false;
        float sbf_ms = 1e30f;
        for (size_t ri = 0; ok && ri < plan->ranges.size() && rc == FDD_OK; ri++) {
            RangeState& r = plan->ranges[ri];
            int keep = r.sbf, keep_cc = r.s_CC;
            float keep_ms = 1e30f;
            for (int sv = 0; sv < fdd::num_sbf_variants() && rc == FDD_OK; sv++) {
                if (fdd::sbf_variant(sv).E != (r.D == 1 ? 1 : 2)) continue;
                for (int cc : {16, 32, 64}) {
                    if (configure_sbf(plan, r, sv, cc) != FDD_OK) continue;
                    if (prepare(plan, n_out, FDD_BATCH_SB_FACTORED, false, absolute) != FDD_OK) continue;
                    BatchLaunch P;
                    if ((rc = fill_params(plan, jobs, n_jobs, n_out, P)) != FDD_OK) break;
                    if ((rc = enqueue(plan, P, s)) != FDD_OK) break;
                    cudaEventRecord(ev0, s);
                    for (int k = 0; k < reps && rc == FDD_OK; k++) rc = enqueue(plan, P, s);
                    cudaEventRecord(ev1, s);
                    if (rc != FDD_OK) break;
                    if ((e = cudaEventSynchronize(ev1)) != cudaSuccess) {
                        rc = cuda_fail(e, "batch tuning");
                        break;
                    }
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, ev0, ev1);
                    ms /= reps;
                    if (std::getenv("FDD_TUNE_VERBOSE"))
                        std::fprintf(stderr, "fdd batch tune: range %zu SB-factored variant %d cc %d: %.4f ms\n", ri,
                                     sv, cc, ms);
                    if (ms < keep_ms) {
                        keep_ms = ms;
                        keep = sv;
                        keep_cc = cc;
                    }
                }
            }
            if (rc == FDD_OK && configure_sbf(plan, r, keep, keep_cc) != FDD_OK) ok = false;
            sbf_ms = keep_ms;
        }
        if (rc == FDD_OK && ok && sbf_ms < best_ms) {
            best_ms = sbf_ms;
            best = FDD_BATCH_SB_FACTORED;
        }
        // persistent SB-factored mode: one launch for every job, range and slab (its own part variant)
        std::vector<std::pair<int, int>> tuned;
        for (const RangeState& r : plan->ranges) tuned.emplace_back(range_config_index(r), range_config_cc(r));
        float sbp_ms = 1e30f;
        if (rc == FDD_OK && prepare(plan, n_out, FDD_BATCH_SB_PERSISTENT, false, absolute) == FDD_OK) {
            BatchLaunch P;
            if ((rc = fill_params(plan, jobs, n_jobs, n_out, P)) == FDD_OK && (rc = enqueue(plan, P, s)) == FDD_OK) {
                cudaEventRecord(ev0, s);
                for (int k = 0; k < reps && rc == FDD_OK; k++) rc = enqueue(plan, P, s);
                cudaEventRecord(ev1, s);
                if (rc == FDD_OK) {
                    if ((e = cudaEventSynchronize(ev1)) != cudaSuccess) {
                        rc = cuda_fail(e, "batch tuning");
                    } else {
                        cudaEventElapsedTime(&sbp_ms, ev0, ev1);
                        sbp_ms /= reps;
                        if (std::getenv("FDD_TUNE_VERBOSE"))
                            std::fprintf(stderr, "fdd batch tune: persistent SB-factored: %.4f ms\n", sbp_ms);
                    }
                }
            }
        }
        if (rc == FDD_OK && sbp_ms < best_ms) {
            best_ms = sbp_ms;
            best = FDD_BATCH_SB_PERSISTENT;
        } else if (best == FDD_BATCH_SB_FACTORED) {
            for (size_t ri = 0; ri < plan->ranges.size(); ri++)  // the tuned SB-factored configuration
                if (tuned[ri].first >= 0) restore_range_config(plan, plan->ranges[ri], tuned[ri].first, tuned[ri].second);
        } else {
            for (size_t ri = 0; ri < plan->ranges.size(); ri++)  // put the per-range configuration back
                if (saved[ri].first >= 0) restore_range_config(plan, plan->ranges[ri], saved[ri].first, saved[ri].second);
        }
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (rc != FDD_OK) return rc;
    if (best < 0) return fail(FDD_ERR_UNSUPPORTED, "no persistent variant fits this plan");
    rc = prepare(plan, n_out, best, best_big, absolute);
    if (rc == FDD_OK) plan->batch.tuned_ms = best_ms;
    return rc;
}

int fdd_batch_config(const fdd_plan* plan, int32_t* variant, int32_t* grid, int32_t* threads, int32_t* dm_per_block,
                     float* tuned_ms) {
    if (!plan) return fail(FDD_ERR_INVALID_ARG, "null plan");
    const BatchState& b = plan->batch;
    if (b.variant < 0) return fail(FDD_ERR_INVALID_ARG, "batch not prepared");
    const fdd::PersistentVariant& pv = fdd::persistent_variant(b.variant);
    if (b.sbp) {
        if (variant) *variant = FDD_BATCH_SB_PERSISTENT;
        if (grid) *grid = b.sp_grid;
        if (threads) *threads = fdd::sbf_persist_part_variant(1).threads();
        if (dm_per_block) *dm_per_block = fdd::sbf_persist_part_variant(1).bd();
        if (tuned_ms) *tuned_ms = b.tuned_ms;
        return FDD_OK;
    }
    if (b.sbf) {
        if (variant) *variant = FDD_BATCH_SB_FACTORED;
        if (grid) *grid = 0;
        if (threads) *threads = 0;
        if (dm_per_block) *dm_per_block = 0;
        if (tuned_ms) *tuned_ms = b.tuned_ms;
        return FDD_OK;
    }
    if (variant) *variant = b.variant;
    if (grid) *grid = b.grid_e[0] ? b.grid_e[0] : b.grid_e[1];
    if (threads) *threads = pv.threads();
    if (dm_per_block) *dm_per_block = pv.bd();
    if (tuned_ms) *tuned_ms = b.tuned_ms;
    return FDD_OK;
}

int fdd_graph_create(fdd_plan* plan, const fdd_job* jobs, int32_t n_jobs, int64_t n_out, fdd_graph** out) {
    if (!plan || !out || n_out < 0) return fail(FDD_ERR_INVALID_ARG, "bad argument");
    *out = nullptr;
    const bool absolute = jobs_absolute(jobs, n_jobs);
    if (plan->batch.n_out != n_out || plan->batch.absolute != absolute) {
        const int rc = prepare(plan, n_out, -1, false, absolute);
        if (rc != FDD_OK) return rc;
    }
    BatchLaunch P;
    int rc = fill_params(plan, jobs, n_jobs, n_out, P);
    if (rc != FDD_OK) return rc;
    fdd_graph* g = new (std::nothrow) fdd_graph();
    if (!g) return fail(FDD_ERR_NO_MEMORY, "host allocation");
    g->plan = plan;
    g->n_jobs = n_jobs;
    g->n_out = n_out;
    cudaError_t e = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete g;
        return cuda_fail(e, "cudaStreamCreate");
    }
    if ((rc = capture(g, P, &g->graph)) != FDD_OK) {
        fdd_graph_destroy(g);
        return rc;
    }
    if ((e = cudaGraphInstantiate(&g->exec, g->graph, 0)) != cudaSuccess) {
        fdd_graph_destroy(g);
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    *out = g;
    return FDD_OK;
}

int fdd_graph_update(fdd_graph* g, const fdd_job* jobs, int32_t n_jobs) {
    if (!g || n_jobs != g->n_jobs) return fail(FDD_ERR_INVALID_ARG, "graph update needs the same number of jobs");
    if (g->plan->batch.n_out != g->n_out) return fail(FDD_ERR_INVALID_ARG, "plan re-prepared for another n_out");
    BatchLaunch P;
    int rc = fill_params(g->plan, jobs, n_jobs, g->n_out, P);
    if (rc != FDD_OK) return rc;
    cudaGraph_t fresh = nullptr;
    if ((rc = capture(g, P, &fresh)) != FDD_OK) return rc;
    cudaGraphExecUpdateResultInfo info;
    cudaError_t e = cudaGraphExecUpdate(g->exec, fresh, &info);
    if (e != cudaSuccess) {  // topology changed: instantiate afresh
        cudaGetLastError();
        cudaGraphExec_t exec = nullptr;
        if ((e = cudaGraphInstantiate(&exec, fresh, 0)) != cudaSuccess) {
            cudaGraphDestroy(fresh);
            return cuda_fail(e, "cudaGraphInstantiate");
        }
        cudaGraphExecDestroy(g->exec);
        g->exec = exec;
    }
    cudaGraphDestroy(g->graph);
    g->graph = fresh;
    return FDD_OK;
}

int fdd_graph_launch(fdd_graph* g, fdd_stream_t stream) {
    if (!g || !g->exec) return fail(FDD_ERR_INVALID_ARG, "null graph");
    const cudaError_t e = cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return FDD_OK;
}

int fdd_graph_destroy(fdd_graph* g) {
    if (!g) return FDD_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->cap_stream) {
        if (g->plan) release_lanes(g->plan, g->cap_stream);  // the plan outlives its graphs
        cudaStreamDestroy(g->cap_stream);
    }
    delete g;
    return FDD_OK;
}

}  // extern "C"

int fdd::host::batch_prepare_mode(fdd_plan* plan, int64_t n_out, bool absolute) {
    if (plan->batch.n_out == n_out && plan->batch.absolute == absolute) return FDD_OK;
    return prepare(plan, n_out, -1, false, absolute);
}

void fdd_free_batch_state(fdd_plan* plan) {
    free_lanes(plan->batch);
    free_batch(plan->batch);
    if (plan->batch.d_counter) cudaFree(plan->batch.d_counter);
    plan->batch.d_counter = nullptr;
}
