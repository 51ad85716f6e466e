// fdd_plan.cu -- host side of the C ABI: plan construction (delay tables,
// staged-offset tables, kernel variant per range), workspace layout and the
// per-chunk search orchestration.  Every stage of the search itself runs in
// the CUDA kernels of k_downsample.cu, k_dedisp.cu and k_boxcar.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fdd_plan_impl.h"

namespace {

thread_local std::string g_last_error;

}  // namespace

namespace fdd {
namespace host {

int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return FDD_ERR_CUDA;
}

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

void stage_reset(fdd_plan* plan) {
    plan->st_kind.clear();
    plan->st_range.clear();
}

// Record the opening event of a timed stage (no-op unless timing is on).
cudaError_t stage_begin(fdd_plan* plan, int kind, int range, cudaStream_t s) {
    if (!plan->timing) return cudaSuccess;
    const size_t k = plan->st_kind.size();
    while (plan->ev.size() < 2 * (k + 1)) {
        cudaEvent_t e;
        const cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return err;
        plan->ev.push_back(e);
    }
    plan->st_kind.push_back(kind);
    plan->st_range.push_back(range);
    return cudaEventRecord(plan->ev[2 * k], s);
}

cudaError_t stage_end(fdd_plan* plan, cudaStream_t s) {
    if (!plan->timing) return cudaSuccess;
    return cudaEventRecord(plan->ev[2 * (plan->st_kind.size() - 1) + 1], s);
}

}  // namespace host
}  // namespace fdd

using namespace fdd::host;

void fdd_free_batch_state(fdd_plan* plan);  // fdd_batch.cu

// Staged-row geometry of range r for kernel variant v: for every (DM block,
// channel) the aligned first staged sample, and for every trial its byte
// offset (copy q = misalignment, aligned word) inside the channel slot.
HostTables fdd::host::build_tables(const fdd_plan* p, const RangeState& r, const fdd::DedispVariant& v) {
    const int E = v.E, BD = v.bd(), NW = v.NW;
    const int A = 16 / E;  // alignment of the staged row start, in samples
    const int n_chan = p->n_chan;
    const int n_blk = (r.n_dm + BD - 1) / BD;
    HostTables h;
    h.base.resize(static_cast<size_t>(n_blk) * n_chan);
    int64_t max_span_words = 0;
    for (int b = 0; b < n_blk; b++) {
        const int ia = b * BD, ib = std::min(r.n_dm, (b + 1) * BD);
        for (int c = 0; c < n_chan; c++) {
            int32_t lo = r.delay[static_cast<size_t>(ia) * n_chan + c], hi = lo;
            for (int i = ia; i < ib; i++) {
                const int32_t d = r.delay[static_cast<size_t>(i) * n_chan + c];
                lo = std::min(lo, d);
                hi = std::max(hi, d);
            }
            const int32_t bs = lo / A * A;
            h.base[static_cast<size_t>(b) * n_chan + c] = bs;
            max_span_words = std::max<int64_t>(max_span_words, (static_cast<int64_t>(hi - bs) * E) >> 2);
        }
    }
    const int64_t Lw = static_cast<int64_t>(align_up(static_cast<size_t>(max_span_words + 32 * NW), 4));
    h.Lw = Lw > (1 << 20) ? -1 : static_cast<int32_t>(Lw);
    if (h.Lw < 0) return h;
    h.off.resize(static_cast<size_t>(n_blk) * n_chan * BD);
    for (int b = 0; b < n_blk; b++)
        for (int c = 0; c < n_chan; c++)
            for (int jj = 0; jj < BD; jj++) {
                const int i = std::min(b * BD + jj, r.n_dm - 1);  // padding trials repeat the last one
                const int32_t o = (r.delay[static_cast<size_t>(i) * n_chan + c] -
                                   h.base[static_cast<size_t>(b) * n_chan + c]) * E;
                const int32_t q = (o & 3) / E;
                h.off[(static_cast<size_t>(b) * n_chan + c) * BD + jj] = q * h.Lw * 4 + (o & ~3);
            }
    return h;
}

int fdd::host::pick_cc(const fdd::DedispVariant& v, int Lw) {
    for (int cc : {32, 16, 8, 4, 2})
        if (fdd::dedisp_cc_ok(v, Lw, cc, kDefaultSmem)) return cc;
    for (int cc : {32, 16, 8, 4, 2})
        if (fdd::dedisp_cc_ok(v, Lw, cc, kSmemBudget)) return cc;
    return 0;
}

int fdd::host::upload_tables(int32_t** d_off, int32_t** d_base, const HostTables& h) {
    cudaError_t e = cudaMalloc(d_off, h.off.size() * sizeof(int32_t));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(offset table)");
    e = cudaMalloc(d_base, h.base.size() * sizeof(int32_t));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(base table)");
    e = cudaMemcpy(*d_off, h.off.data(), h.off.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(offset table)");
    e = cudaMemcpy(*d_base, h.base.data(), h.base.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(base table)");
    return FDD_OK;
}

fdd::host::Bins fdd::host::search_bins(const fdd_plan* p, int64_t n_out, int64_t t0, bool absolute) {
    Bins b;
    b.absolute = absolute;
    for (const RangeState& r : p->ranges) {
        if (!absolute) {
            b.stride.push_back(static_cast<int32_t>(n_out / r.D));
            b.emit.push_back(static_cast<int32_t>(n_out / r.D));
            b.phase.push_back(0);
            continue;
        }
        const int64_t j_first = (t0 + r.D - 1) / r.D;           // ceil(t0 / D): first bin starting in the window
        const int64_t j_end = (t0 + n_out + r.D - 1) / r.D;     // ceil((t0 + n_out) / D)
        b.stride.push_back(static_cast<int32_t>((n_out + r.D - 1) / r.D));
        b.emit.push_back(static_cast<int32_t>(j_end - j_first));
        b.phase.push_back(static_cast<int32_t>(j_first * r.D - t0));
    }
    for (int32_t D : p->ds_factors) b.ds_phase.push_back(absolute ? static_cast<int32_t>((D - t0 % D) % D) : 0);
    return b;
}

int64_t fdd::host::window_input_len(const fdd_plan* p, int64_t n_out) {
    int64_t extra = 0;
    for (const RangeState& r : p->ranges)
        extra = std::max<int64_t>(extra, static_cast<int64_t>(r.D) * (r.dmax + 1) - 1);
    return n_out + extra;
}

int fdd::host::sbf_lanes(const fdd_plan* p) { return p->n_sb >= 2 && p->ranges.size() >= 2 ? 2 : 1; }

size_t fdd::plain_workspace_bytes(const fdd_plan* plan, int64_t n_in, int64_t n_out, bool with_series) {
    return fdd::host::make_layout(plan, n_in, n_out, with_series, false, 1).total;
}

fdd::host::Layout fdd::host::make_layout(const fdd_plan* p, int64_t n_in, int64_t n_out, bool with_series,
                                         bool absolute, int lanes) {
    Layout L;
    size_t series_elems = 0, n_series = 0;
    for (const RangeState& r : p->ranges) {
        L.series_r.push_back(series_elems);
        L.stat_r.push_back(n_series);
        const size_t nr = static_cast<size_t>(absolute ? (n_out + r.D - 1) / r.D : n_out / r.D);
        series_elems += static_cast<size_t>(p->n_sb) * r.n_dm * nr;
        n_series += static_cast<size_t>(p->n_sb) * r.n_dm;
    }
    L.series_bytes = series_elems * sizeof(int32_t);
    L.stat_bytes = n_series * 2 * sizeof(unsigned long long);
    size_t cur = 0;
    // absolute windows: ceil(n_out / D) <= floor((n_out + D_max - 1) / D) outputs per row
    const int64_t n_rows = absolute ? n_out + (p->ds_factors.empty() ? 0 : *std::max_element(p->ds_factors.begin(),
                                                                                               p->ds_factors.end()) - 1)
                                    : n_out;
    L.sbf_lane_bytes = align_up(std::max(sbf_scratch_bytes(p, n_rows), subband_scratch_bytes(p, n_rows)), 256);
    L.sbf_lanes = lanes > 0 ? lanes : sbf_lanes(p);
    L.sbf_bytes = L.sbf_lane_bytes * static_cast<size_t>(L.sbf_lanes);
    if (L.sbf_bytes) {
        L.sbf = cur;
        cur = align_up(cur + L.sbf_bytes, 256);
    }
    if (with_series) {
        L.series = cur;
        cur = align_up(cur + L.series_bytes, 256);
    }
    L.stat = cur;
    cur = align_up(cur + L.stat_bytes, 256);
    for (int32_t D : p->ds_factors) {
        const int64_t pitch = static_cast<int64_t>(align_up(static_cast<size_t>(n_in / D), 8));
        L.ds_pitch.push_back(pitch);
        L.ds_off.push_back(cur);
        cur = align_up(cur + static_cast<size_t>(p->n_tab) * p->n_chan * pitch * sizeof(uint16_t), 256);
    }
    L.total = std::max<size_t>(cur, 256);
    return L;
}

int fdd::host::check_search_args(const fdd_plan* plan, const uint8_t* d_tabs, int64_t n_in, int64_t pitch, int64_t n_out,
                      const void* d_workspace, const void* d_series, const Bins* bins) {
    if (!plan || !d_tabs || !d_workspace || n_in < 0 || n_out < 0 || pitch < n_in)
        return fail(FDD_ERR_INVALID_ARG, "bad search argument");
    if (n_out > (1LL << 30) || n_in > (1LL << 31) - 64)
        return fail(FDD_ERR_UNSUPPORTED, "chunk longer than the kernels' 32-bit sample indexing");
    if ((reinterpret_cast<uintptr_t>(d_tabs) & 15) || (pitch & 15) ||
        (reinterpret_cast<uintptr_t>(d_workspace) & 255) || (reinterpret_cast<uintptr_t>(d_series) & 15))
        return fail(FDD_ERR_MISALIGNED, "d_tabs/pitch must be 16-byte aligned, workspace 256-byte aligned");
    if (bins && bins->absolute) {
        for (size_t ri = 0; ri < plan->ranges.size(); ri++) {
            const RangeState& r = plan->ranges[ri];
            if (bins->emit[ri] > 0 &&
                bins->phase[ri] + static_cast<int64_t>(r.D) * (bins->emit[ri] + static_cast<int64_t>(r.dmax)) > n_in)
                return fail(FDD_ERR_SHORT_INPUT, "n_in < phase + D * (bins + max delay) for some DM range "
                                                 "(fdd_window_input_len)");
        }
        return FDD_OK;
    }
    for (const RangeState& r : plan->ranges)
        if (n_out / r.D + r.dmax > n_in / r.D)
            return fail(FDD_ERR_SHORT_INPUT, "n_in < n_out + max delay for some DM range");
    return FDD_OK;
}

namespace {

void free_fact_tables(RangeState& r) {
    for (int32_t** ptr : {&r.d_fbase, &r.d_goff, &r.d_pdesc, &r.d_pdidx, &r.d_fbbase}) {
        if (*ptr) cudaFree(*ptr);
        *ptr = nullptr;
    }
    r.fact = -1;
}

void free_brute_tables(RangeState& r) {
    if (r.d_off) cudaFree(r.d_off);
    if (r.d_base) cudaFree(r.d_base);
    r.d_off = nullptr;
    r.d_base = nullptr;
}

void free_range_tables(RangeState& r) {
    free_brute_tables(r);
    free_fact_tables(r);
    free_sbf_tables(r, true);
}

int upload_vec(int32_t** dst, const std::vector<int32_t>& v, const char* what) {
    cudaError_t e = cudaMalloc(dst, std::max<size_t>(v.size(), 4) * sizeof(int32_t));
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (!v.empty() && (e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, what);
    return FDD_OK;
}

// Configure range r for pattern-factored variant fv with CC channels per
// stage (0 = the largest that fits).
int configure_fact(fdd_plan* p, RangeState& r, int fv, int CC) {
    if (fv < 0 || fv >= fdd::num_fact_variants()) return fail(FDD_ERR_INVALID_ARG, "kernel variant out of range");
    if (!fdd::fact_has_width(fv, r.D == 1 ? 1 : 2, false))
        return fail(FDD_ERR_INVALID_ARG, "this factored variant is not built for the range's sample width");
    const fdd::FactVariant& v = fdd::fact_variant(fv);
    FactTables best;
    int best_cc = 0;
    for (int cc : {64, 48, 32, 16, 8, 4}) {
        if (CC != 0 && cc != CC) continue;
        if (cc % v.G) continue;
        FactTables ft = build_fact_tables(p, r, v, cc, p->n_tab == 1);
        if (ft.Lw < 0 || !fdd::fact_cc_ok(v, ft.Lw, cc, ft.max_desc) || ft.smem_bytes > kSmemBudget) continue;
        best = std::move(ft);
        best_cc = cc;
        break;
    }
    if (best_cc == 0) return fail(FDD_ERR_UNSUPPORTED, "factored kernel does not fit this range and stage size");
    free_fact_tables(r);
    free_sbf_tables(r, true);
    int rc;
    if ((rc = upload_vec(&r.d_fbase, best.base, "factored base table")) != FDD_OK) return rc;
    if ((rc = upload_vec(&r.d_goff, best.goff, "factored offset table")) != FDD_OK) return rc;
    if ((rc = upload_vec(&r.d_pdesc, best.pdesc, "factored descriptors")) != FDD_OK) return rc;
    if ((rc = upload_vec(&r.d_pdidx, best.pd_idx, "factored descriptor index")) != FDD_OK) return rc;
    if ((rc = upload_vec(&r.d_fbbase, best.bbase, "factored box starts")) != FDD_OK) return rc;
    r.f_box_rows = best.box_rows;
    r.fact = fv;
    r.f_CC = best_cc;
    r.f_Lw = best.Lw;
    r.f_pat_bytes = best.pat_bytes;
    r.f_n_stages = best.n_stages;
    r.f_n_groups = best.n_groups;
    r.f_smem = best.smem_bytes;
    r.f_zero_off = best.zero_off;
    r.f_raw_off = best.raw_off;
    r.f_rb = best.rb;
    r.f_pat_off = best.pat_off;
    r.f_bar_off = best.bar_off;
    r.f_desc_bytes = best.desc_bytes;
    r.f_work_ratio = static_cast<float>(best.work_ratio);
    return FDD_OK;
}

// Configure range r for kernel variant `variant` with channel stage CC
// (0 = the largest that fits).
int configure_range(fdd_plan* p, RangeState& r, int variant, int CC) {
    const int nbf = fdd::num_dedisp_variants() + fdd::num_fact_variants();
    if (variant >= nbf) {  // SB-factored variants follow the pattern-factored ones
        const int rc = configure_sbf(p, r, variant - nbf, CC);
        if (rc == FDD_OK) {
            free_brute_tables(r);
            if (r.s_fact < 0) free_fact_tables(r);  // a pattern-factored part keeps its tables
        }
        return rc;
    }
    if (variant >= fdd::num_dedisp_variants())  // factored variants follow the brute-force ones
        return configure_fact(p, r, variant - fdd::num_dedisp_variants(), CC);
    if (variant < 0) return fail(FDD_ERR_INVALID_ARG, "kernel variant out of range");
    const fdd::DedispVariant& v = fdd::dedisp_variant(variant);
    if (v.E != (r.D == 1 ? 1 : 2)) return fail(FDD_ERR_INVALID_ARG, "kernel variant for the wrong sample width");
    const HostTables h = build_tables(p, r, v);
    if (h.Lw < 0) return fail(FDD_ERR_UNSUPPORTED, "DM step too large for one block's staged rows");
    if (CC == 0) CC = pick_cc(v, h.Lw);
    if (CC == 0 || !fdd::dedisp_cc_ok(v, h.Lw, CC, kSmemBudget))
        return fail(FDD_ERR_UNSUPPORTED, "DM step too large for one block's staged rows; lower ddm or raise downsamp");
    free_range_tables(r);
    const int rc = upload_tables(&r.d_off, &r.d_base, h);
    if (rc != FDD_OK) return rc;
    r.variant = variant;
    r.Lw = h.Lw;
    r.CC = CC;
    return FDD_OK;
}

// Launch range r's dedispersion kernel (brute force or pattern-factored).
cudaError_t launch_range_dedisp(const fdd_plan* p, const RangeState& r, const fdd::DedispArgs& a, cudaStream_t s) {
    if (r.fact < 0) return fdd::launch_dedisp(r.variant, a, s);
    fdd::FactArgs fa{};
    fa.status = p->d_status;
    fa.in = a.in;
    fa.pitch_bytes = a.pitch_bytes;
    fa.n_valid = a.n_valid;
    fa.E = r.D == 1 ? 1 : 2;
    fa.fold_ch = 256 / r.D;  // 16-bit lanes hold at most 256 / D channels of 255 D
    fa.sb_map = a.sb_map;
    fa.base = r.d_fbase;
    fa.goff = r.d_goff;
    fa.pdesc = r.d_pdesc;
    fa.pd_idx = r.d_pdidx;
    fa.bbase = r.d_fbbase;
    fa.box_rows = r.f_box_rows;
    fa.series = a.series;
    fa.stat = a.stat;
    fa.n_chan = a.n_chan;
    fa.n_dm = a.n_dm;
    fa.n_out = a.n_out;
    fa.n_emit = a.n_emit;
    fa.n_sb = a.n_sb;
    fa.Lw = r.f_Lw;
    fa.CC = r.f_CC;
    fa.n_stages = r.f_n_stages;
    fa.n_groups = r.f_n_groups;
    fa.pat_bytes = r.f_pat_bytes;
    fa.zero_off = r.f_zero_off;
    fa.raw_off = r.f_raw_off;
    fa.rb = r.f_rb;
    fa.pat_off = r.f_pat_off;
    fa.bar_off = r.f_bar_off;
    fa.desc_bytes = r.f_desc_bytes;
    if (cudaError_t e = fdd::encode_fact_map(fa, static_cast<int64_t>(p->n_tab) * p->n_chan); e != cudaSuccess) return e;
    return fdd::launch_dedisp_fact(r.fact, fa, r.f_smem, s);
}

int range_variant_index(const RangeState& r) {
    if (r.sbf >= 0) return fdd::num_dedisp_variants() + fdd::num_fact_variants() + r.sbf;
    return r.fact >= 0 ? fdd::num_dedisp_variants() + r.fact : r.variant;
}

// Dedispersion of one range with whichever kernel it is configured for.
cudaError_t launch_range(const fdd_plan* p, const RangeState& r, const fdd::DedispArgs& a, const Layout& L,
                         uint8_t* ws, cudaStream_t s, int64_t* launches = nullptr) {
    if (r.sub_G > 0) return launch_range_subband(p, r, a, ws + L.sbf, L.sbf_lane_bytes, s, launches);
    if (r.sbf >= 0) return launch_range_sbf(p, r, a, ws + L.sbf, L.sbf_lane_bytes, s, launches);
    if (launches) *launches += 1;
    return launch_range_dedisp(p, r, a, s);
}

int default_variant(int E) {
    for (int k = 0; k < fdd::num_dedisp_variants(); k++)
        if (fdd::dedisp_variant(k).E == E) return k;
    return -1;
}


fdd::DedispArgs dedisp_args(const fdd_plan* plan, const RangeState& r, size_t ri, const Layout& L,
                            const uint8_t* d_tabs, int64_t pitch, uint8_t* ws, int32_t* series,
                            unsigned long long* stat, int64_t n_in, const Bins& bins) {
    fdd::DedispArgs a{};
    if (r.D == 1) {
        a.in = d_tabs;
        a.pitch_bytes = pitch;
    } else {
        const size_t k = std::find(plan->ds_factors.begin(), plan->ds_factors.end(), r.D) - plan->ds_factors.begin();
        a.in = ws + L.ds_off[k];
        a.pitch_bytes = L.ds_pitch[k] * 2;
    }
    a.n_valid = (n_in - bins.phase[ri]) / r.D;
    a.sb_map = plan->d_sb_map;
    a.base = r.d_base;
    a.off = r.d_off;
    a.series = series + L.series_r[ri];
    a.stat = stat + 2 * L.stat_r[ri];
    a.n_chan = plan->n_chan;
    a.n_dm = r.n_dm;
    a.n_out = bins.stride[ri];
    a.n_emit = bins.emit[ri];
    a.n_sb = plan->n_sb;
    a.Lw = r.Lw;
    a.CC = r.CC;
    return a;
}


}  // namespace

int fdd::host::range_config_index(const RangeState& r) { return range_variant_index(r); }

int fdd::host::range_config_cc(const RangeState& r) { return r.sbf >= 0 ? r.s_CC : (r.fact >= 0 ? r.f_CC : r.CC); }

int fdd::host::restore_range_config(fdd_plan* p, RangeState& r, int variant, int CC) {
    return configure_range(p, r, variant, CC);
}

namespace fdd {
bool plan_timing_enabled(const fdd_plan* plan) { return plan && plan->timing; }
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace fdd

// Host part of plan construction: validation and every range's delay table.
static int build_host_plan(const fdd_plan_desc* desc, const int16_t* sb_map_host, fdd_plan* p) {
    if (!desc || !sb_map_host) return fail(FDD_ERR_INVALID_ARG, "null argument");
    if (desc->n_tab < 1 || desc->n_tab > FDD_MAX_TABS || desc->n_chan < 1 || desc->n_chan > FDD_MAX_CHANNELS ||
        desc->n_sb < 1 || desc->n_sb > 65535 || desc->n_range < 1 || !desc->ranges || !desc->chan_freq_mhz ||
        !(desc->t_samp_s > 0))
        return fail(FDD_ERR_INVALID_ARG, "bad plan dimensions");
    for (int c = 0; c < desc->n_chan; c++)
        if (!(desc->chan_freq_mhz[c] > 0) || !std::isfinite(desc->chan_freq_mhz[c]))
            return fail(FDD_ERR_INVALID_ARG, "channel frequencies must be positive and finite");
    for (int64_t k = 0; k < static_cast<int64_t>(desc->n_sb) * desc->n_chan; k++)
        if (sb_map_host[k] < 0 || sb_map_host[k] >= desc->n_tab)
            return fail(FDD_ERR_INVALID_ARG, "sb_map entry outside [0, n_tab)");
    p->n_tab = desc->n_tab;
    p->n_chan = desc->n_chan;
    p->n_sb = desc->n_sb;
    p->t_samp = desc->t_samp_s;
    p->thr = desc->snr_thresh;
    p->freq.assign(desc->chan_freq_mhz, desc->chan_freq_mhz + desc->n_chan);
    p->sb_map.assign(sb_map_host, sb_map_host + static_cast<size_t>(desc->n_sb) * desc->n_chan);
    const double f_top = *std::max_element(p->freq.begin(), p->freq.end());
    int32_t dm_index = 0;
    for (int ri = 0; ri < desc->n_range; ri++) {
        const fdd_range& in = desc->ranges[ri];
        if (!(in.dm0 >= 0) || !(in.ddm > 0) || in.n_dm < 1 || in.downsamp < 1 || in.downsamp > 257 ||
            in.n_width < 1 || in.n_width > FDD_MAX_WIDTHS || !in.widths) {
            return fail(FDD_ERR_INVALID_ARG, "bad DM range");
        }
        RangeState r;
        r.dm0 = in.dm0;
        r.ddm = in.ddm;
        r.n_dm = in.n_dm;
        r.D = in.downsamp;
        r.n_width = in.n_width;
        r.wmax = 1;
        for (int k = 0; k < in.n_width; k++) {
            if (in.widths[k] < 1 || in.widths[k] > FDD_MAX_WIDTH) {
                return fail(FDD_ERR_INVALID_ARG, "boxcar width outside [1, FDD_MAX_WIDTH]");
            }
            r.widths[k] = in.widths[k];
            r.wmax = std::max(r.wmax, in.widths[k]);
        }
        // Box sums are formed as differences of wrapping 32-bit prefix sums of
        // the series centred on round(mean): exact while |B_w - w round(mean)|
        // < 2^31, which holds for every input when n_chan * 255 * D * w_max does.
        if (static_cast<int64_t>(desc->n_chan) * 255 * in.downsamp * r.wmax > (1LL << 31) - 1)
            return fail(FDD_ERR_UNSUPPORTED,
                        "n_chan * 255 * downsamp * widest boxcar >= 2^31: box sums could leave int32");
        r.dm_index0 = dm_index;
        dm_index += in.n_dm;
        // Delay table: cold-plasma law, FP64, same operation order for every
        // entry, rounded half away from zero.
        r.delay.resize(static_cast<size_t>(r.n_dm) * p->n_chan);
        int64_t dmax = 0;
        for (int i = 0; i < r.n_dm; i++) {
            const double dm = r.dm0 + static_cast<double>(i) * r.ddm;
            for (int c = 0; c < p->n_chan; c++) {
                const double f = p->freq[c];
                const double x = ((kDispersionConstant * dm) * (1.0 / (f * f) - 1.0 / (f_top * f_top))) /
                                 (static_cast<double>(r.D) * p->t_samp);
                const long long d = std::llround(x);
                if (d < 0 || d > (1LL << 28)) {
                    return fail(FDD_ERR_UNSUPPORTED, "delay out of range");
                }
                r.delay[static_cast<size_t>(i) * p->n_chan + c] = static_cast<int32_t>(d);
                dmax = std::max<int64_t>(dmax, d);
            }
        }
        r.dmax = static_cast<int32_t>(dmax);
        p->max_delay_native = std::max<int64_t>(p->max_delay_native, dmax * r.D);
        p->ranges.push_back(std::move(r));
        if (in.downsamp > 1 &&
            std::find(p->ds_factors.begin(), p->ds_factors.end(), in.downsamp) == p->ds_factors.end())
            p->ds_factors.push_back(in.downsamp);
    }
    p->n_dm_total = dm_index;
    for (RangeState& r : p->ranges) {
        r.segs = sbf_segments(p, r.D, 16);
        r.seg_maxlen = 0;
        for (const int2& sg : r.segs) r.seg_maxlen = std::max(r.seg_maxlen, sg.y);
    }

    return FDD_OK;
}

int fdd::host::search_impl(fdd_plan* plan, const uint8_t* d_tabs, int64_t n_in, int64_t pitch, int64_t n_out,
                           int64_t t_offset_native, bool absolute, void* d_workspace, size_t workspace_bytes,
                           fdd_candidate* d_cands, int64_t cap, uint64_t* d_count, int32_t* d_series, cudaStream_t s) {
    if (!d_count || (cap > 0 && !d_cands) || cap < 0) return fail(FDD_ERR_INVALID_ARG, "bad search argument");
    if (!plan) return fail(FDD_ERR_INVALID_ARG, "bad search argument");
    if (absolute && t_offset_native < 0) return fail(FDD_ERR_INVALID_ARG, "window start must be >= 0");
    // a window reads no more than fdd_window_sizes' n_in (its workspace is sized for that)
    if (absolute && n_in > window_input_len(plan, n_out)) n_in = window_input_len(plan, n_out);
    const Bins bins = search_bins(plan, n_out, t_offset_native, absolute);
    {
        const int rc = check_search_args(plan, d_tabs, n_in, pitch, n_out, d_workspace, d_series, &bins);
        if (rc != FDD_OK) return rc;
    }
    const bool own_series = (d_series == nullptr);
    const Layout L = make_layout(plan, n_in, n_out, own_series, absolute, 1);  // one scratch lane
    if (workspace_bytes < L.total) return fail(FDD_ERR_WORKSPACE, "workspace smaller than fdd_workspace_size()");

    uint8_t* ws = static_cast<uint8_t*>(d_workspace);
    fdd::host::stage_reset(plan);
    auto stage_begin = [&](int kind, int range) { return fdd::host::stage_begin(plan, kind, range, s); };
    auto stage_end = [&]() { return fdd::host::stage_end(plan, s); };
    int32_t* series = own_series ? reinterpret_cast<int32_t*>(ws + L.series) : d_series;
    unsigned long long* stat = reinterpret_cast<unsigned long long*>(ws + L.stat);

    cudaError_t e = cudaMemsetAsync(stat, 0, L.stat_bytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(stat)");
    e = cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(count)");

    int64_t n_launch = 0;
    plan->last_launches = 0;
    for (size_t k = 0; k < plan->ds_factors.size(); k++) {
        n_launch++;
        if ((e = stage_begin(0, plan->ds_factors[k])) != cudaSuccess) return cuda_fail(e, "timing event");
        e = fdd::launch_downsample(d_tabs, static_cast<int64_t>(plan->n_tab) * plan->n_chan, n_in, pitch,
                                   plan->ds_factors[k], reinterpret_cast<uint16_t*>(ws + L.ds_off[k]),
                                   L.ds_pitch[k], s, bins.ds_phase[k]);
        if (e != cudaSuccess) return cuda_fail(e, "downsample launch");
        if ((e = stage_end()) != cudaSuccess) return cuda_fail(e, "timing event");
    }

    for (size_t ri = 0; ri < plan->ranges.size(); ri++) {
        const RangeState& r = plan->ranges[ri];
        const int64_t nr = bins.emit[ri];
        if (nr <= 0) continue;
        const fdd::DedispArgs a = dedisp_args(plan, r, ri, L, d_tabs, pitch, ws, series, stat, n_in, bins);
        if ((e = stage_begin(1, static_cast<int>(ri))) != cudaSuccess) return cuda_fail(e, "timing event");
        e = launch_range(plan, r, a, L, ws, s, &n_launch);
        if (e != cudaSuccess) return cuda_fail(e, "dedispersion launch");
        if ((e = stage_end()) != cudaSuccess) return cuda_fail(e, "timing event");

        fdd::BoxcarArgs b{};
        b.series = a.series;
        b.stat = a.stat;
        b.cands = d_cands;
        b.count = reinterpret_cast<unsigned long long*>(d_count);
        b.cap = cap;
        b.t_offset = t_offset_native + bins.phase[ri];
        b.dm0 = r.dm0;
        b.ddm = r.ddm;
        b.n_sb = plan->n_sb;
        b.n_dm = r.n_dm;
        b.n_out = bins.stride[ri];
        b.n_emit = static_cast<int32_t>(nr);
        b.dm_index0 = r.dm_index0;
        b.D = r.D;
        b.n_width = r.n_width;
        b.wmax = r.wmax;
        b.thr = plan->thr;
        for (int k = 0; k < r.n_width; k++) {
            b.widths[k] = r.widths[k];
            b.inv_sqrt_w[k] = static_cast<float>(1.0 / std::sqrt(static_cast<double>(r.widths[k])));
        }
        if ((e = stage_begin(2, static_cast<int>(ri))) != cudaSuccess) return cuda_fail(e, "timing event");
        e = fdd::launch_boxcar(b, s);
        if (e != cudaSuccess) return cuda_fail(e, "boxcar launch");
        n_launch++;
        if ((e = stage_end()) != cudaSuccess) return cuda_fail(e, "timing event");
    }
    plan->last_launches = n_launch;
    return FDD_OK;
}


extern "C" {

const char* fdd_version(void) { return "fdd 0.1 (sm_103a)"; }

const char* fdd_error_string(int code) {
    switch (code) {
        case FDD_OK: return "ok";
        case FDD_ERR_INVALID_ARG: return "invalid argument";
        case FDD_ERR_SHORT_INPUT: return "input shorter than n_out + maximum delay";
        case FDD_ERR_NO_MEMORY: return "out of memory";
        case FDD_ERR_MISALIGNED: return "pointer or pitch not 16-byte aligned";
        case FDD_ERR_UNSUPPORTED: return "plan outside the kernels' limits";
        case FDD_ERR_CUDA: return "CUDA runtime error";
        case FDD_ERR_WORKSPACE: return "workspace too small";
        case FDD_ERR_SEQUENCE: return "chunk out of sequence";
        case FDD_ERR_BUSY: return "beam backlogged";
        case FDD_ERR_TIMEOUT: return "device wait for a tile copy gave up";
        default: return "unknown error";
    }
}

const char* fdd_last_error_message(void) { return g_last_error.c_str(); }

int fdd_plan_create(const fdd_plan_desc* desc, const int16_t* sb_map_host, fdd_plan** out) {
    if (!desc || !sb_map_host || !out) return fail(FDD_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    fdd_plan* p = new (std::nothrow) fdd_plan();
    if (!p) return fail(FDD_ERR_NO_MEMORY, "host allocation");
    const int hrc = build_host_plan(desc, sb_map_host, p);
    if (hrc != FDD_OK) {
        delete p;
        return hrc;
    }
    cudaGetDevice(&p->device);

    cudaError_t e = cudaMalloc(&p->d_sb_map, p->sb_map.size() * sizeof(int16_t));
    if (e != cudaSuccess) {
        fdd_plan_destroy(p);
        return cuda_fail(e, "cudaMalloc(sb_map)");
    }
    e = cudaMemcpy(p->d_sb_map, p->sb_map.data(), p->sb_map.size() * sizeof(int16_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        fdd_plan_destroy(p);
        return cuda_fail(e, "cudaMemcpy(sb_map)");
    }
    if ((e = cudaMalloc(&p->d_status, sizeof(unsigned int))) != cudaSuccess ||
        (e = cudaMemset(p->d_status, 0, sizeof(unsigned int))) != cudaSuccess) {
        fdd_plan_destroy(p);
        return cuda_fail(e, "cudaMalloc(status word)");
    }
    for (RangeState& r : p->ranges) {
        int rc = FDD_ERR_UNSUPPORTED;
        const int E = (r.D == 1) ? 1 : 2;
        for (int k = default_variant(E); k >= 0 && k < fdd::num_dedisp_variants() && rc != FDD_OK; k++)
            if (fdd::dedisp_variant(k).E == E) rc = configure_range(p, r, k, 0);
        if (rc != FDD_OK) {
            fdd_plan_destroy(p);
            return rc;
        }
    }
    *out = p;
    return FDD_OK;
}

int fdd_plan_destroy(fdd_plan* plan) {
    if (!plan) return FDD_OK;
    fdd_free_batch_state(plan);
    for (cudaEvent_t e : plan->ev) cudaEventDestroy(e);
    for (RangeState& r : plan->ranges) {
        free_range_tables(r);
        free_sbf_tables(r, true);
        free_subband_tables(r);
    }
    if (plan->d_sb_map) cudaFree(plan->d_sb_map);
    if (plan->d_status) cudaFree(plan->d_status);
    delete plan;
    return FDD_OK;
}

int fdd_plan_status(fdd_plan* plan, int32_t* status, int32_t clear) {
    if (!plan || !status) return fail(FDD_ERR_INVALID_ARG, "null argument");
    unsigned int w = 0;
    cudaError_t e = cudaMemcpy(&w, plan->d_status, sizeof(w), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(status word)");
    if (clear && w && (e = cudaMemset(plan->d_status, 0, sizeof(w))) != cudaSuccess)
        return cuda_fail(e, "cudaMemset(status word)");
    *status = static_cast<int32_t>(w);
    return w ? fail(FDD_ERR_TIMEOUT, "a kernel's bounded wait for a tile copy gave up (status word set)") : FDD_OK;
}

int fdd_plan_max_delay(const fdd_plan* plan, int64_t* max_delay_native) {
    if (!plan || !max_delay_native) return fail(FDD_ERR_INVALID_ARG, "null argument");
    *max_delay_native = plan->max_delay_native;
    return FDD_OK;
}

int fdd_plan_info(const fdd_plan* plan, int64_t n_out, int64_t* max_delay_native, int64_t* workspace_bytes) {
    if (!plan || n_out < 0 || !max_delay_native || !workspace_bytes) return fail(FDD_ERR_INVALID_ARG, "bad argument");
    *max_delay_native = plan->max_delay_native;
    *workspace_bytes =
        static_cast<int64_t>(make_layout(plan, n_out + plan->max_delay_native, n_out, true).total);
    return FDD_OK;
}

int fdd_plan_total_dms(const fdd_plan* plan, int64_t* n_dm_total) {
    if (!plan || !n_dm_total) return fail(FDD_ERR_INVALID_ARG, "null argument");
    *n_dm_total = plan->n_dm_total;
    return FDD_OK;
}

int fdd_plan_delays(const fdd_plan* plan, int32_t r, int32_t* dst) {
    if (!plan || !dst || r < 0 || r >= static_cast<int32_t>(plan->ranges.size()))
        return fail(FDD_ERR_INVALID_ARG, "bad range index");
    const RangeState& rs = plan->ranges[r];
    std::memcpy(dst, rs.delay.data(), rs.delay.size() * sizeof(int32_t));
    return FDD_OK;
}

int fdd_workspace_size(const fdd_plan* plan, int64_t n_in, int64_t n_out, int32_t with_series, size_t* bytes) {
    if (!plan || !bytes || n_in < 0 || n_out < 0) return fail(FDD_ERR_INVALID_ARG, "bad argument");
    *bytes = make_layout(plan, n_in, n_out, with_series != 0).total;
    return FDD_OK;
}

int fdd_series_size(const fdd_plan* plan, int64_t n_out, size_t* bytes) {
    if (!plan || !bytes || n_out < 0) return fail(FDD_ERR_INVALID_ARG, "bad argument");
    *bytes = make_layout(plan, 0, n_out, true).series_bytes;
    return FDD_OK;
}

int fdd_search(fdd_plan* plan, const uint8_t* d_tabs, int64_t n_in, int64_t pitch, int64_t n_out,
               int64_t t_offset_native, void* d_workspace, size_t workspace_bytes, fdd_candidate* d_cands,
               int64_t cap, uint64_t* d_count, int32_t* d_series, fdd_stream_t stream) {
    return search_impl(plan, d_tabs, n_in, pitch, n_out, t_offset_native, false, d_workspace, workspace_bytes,
                       d_cands, cap, d_count, d_series, reinterpret_cast<cudaStream_t>(stream));
}

int fdd_search_window(fdd_plan* plan, const uint8_t* d_tabs, int64_t n_in, int64_t pitch, int64_t n_out,
                      int64_t t0_native, void* d_workspace, size_t workspace_bytes, fdd_candidate* d_cands,
                      int64_t cap, uint64_t* d_count, int32_t* d_series, fdd_stream_t stream) {
    return search_impl(plan, d_tabs, n_in, pitch, n_out, t0_native, true, d_workspace, workspace_bytes, d_cands,
                       cap, d_count, d_series, reinterpret_cast<cudaStream_t>(stream));
}

int fdd_window_sizes(const fdd_plan* plan, int64_t n_out, int64_t* n_in, size_t* workspace_bytes,
                     size_t* series_bytes) {
    if (!plan || n_out < 0) return fail(FDD_ERR_INVALID_ARG, "bad argument");
    const int64_t need = window_input_len(plan, n_out);
    if (n_in) *n_in = need;
    if (workspace_bytes) *workspace_bytes = make_layout(plan, need, n_out, true, true).total;
    if (series_bytes) *series_bytes = make_layout(plan, need, n_out, true, true).series_bytes;
    return FDD_OK;
}

int fdd_plan_last_launches(const fdd_plan* plan, int64_t* n) {
    if (!plan || !n) return fail(FDD_ERR_INVALID_ARG, "null argument");
    *n = plan->last_launches;
    return FDD_OK;
}

int fdd_num_variants(int32_t* n) {
    if (!n) return fail(FDD_ERR_INVALID_ARG, "null argument");
    *n = fdd::num_dedisp_variants() + fdd::num_fact_variants() + fdd::num_sbf_variants();
    return FDD_OK;
}

int fdd_variant_kind(int32_t variant, int32_t* kind) {
    const int nb = fdd::num_dedisp_variants(), nf = fdd::num_fact_variants(), ns = fdd::num_sbf_variants();
    if (!kind || variant < 0 || variant >= nb + nf + ns) return fail(FDD_ERR_INVALID_ARG, "bad variant");
    *kind = variant < nb ? 0 : (variant < nb + nf ? 1 : (fdd::sbf_fact_variant(variant - nb - nf) >= 0 ? 3 : 2));
    return FDD_OK;
}

int fdd_variant_info(int32_t variant, int32_t* bytes_per_sample, int32_t* dm_per_block, int32_t* tile,
                     int32_t* threads, int32_t* group) {
    const int nb = fdd::num_dedisp_variants(), nf = fdd::num_fact_variants();
    if (variant < 0 || variant >= nb + nf + fdd::num_sbf_variants()) return fail(FDD_ERR_INVALID_ARG, "bad variant");
    if (variant >= nb + nf) {
        const fdd::DedispVariant& v = fdd::sbf_variant(variant - nb - nf);
        const int fvi = fdd::sbf_fact_variant(variant - nb - nf);
        if (bytes_per_sample) *bytes_per_sample = v.E;
        if (dm_per_block) *dm_per_block = v.bd();
        if (tile) *tile = v.tile();
        if (threads) *threads = v.threads();
        if (group) *group = fvi >= 0 ? fdd::fact_variant(fvi).G : 0;
        return FDD_OK;
    }
    if (variant >= nb) {
        const fdd::FactVariant& v = fdd::fact_variant(variant - nb);
        if (bytes_per_sample) *bytes_per_sample = 1;
        if (dm_per_block) *dm_per_block = v.bd();
        if (tile) *tile = v.tile();
        if (threads) *threads = v.threads();
        if (group) *group = v.G;
        return FDD_OK;
    }
    const fdd::DedispVariant& v = fdd::dedisp_variant(variant);
    if (bytes_per_sample) *bytes_per_sample = v.E;
    if (dm_per_block) *dm_per_block = v.bd();
    if (tile) *tile = v.tile();
    if (threads) *threads = v.threads();
    if (group) *group = 0;
    return FDD_OK;
}

int fdd_plan_get_config(const fdd_plan* plan, int32_t r, fdd_kernel_config* out) {
    if (!plan || !out || r < 0 || r >= static_cast<int32_t>(plan->ranges.size()))
        return fail(FDD_ERR_INVALID_ARG, "bad range index");
    const RangeState& rs = plan->ranges[r];
    out->variant = range_variant_index(rs);
    if (rs.sbf >= 0) {
        const fdd::DedispVariant& v = fdd::sbf_variant(rs.sbf);
        out->dm_per_block = v.bd();
        out->tile = v.tile();
        out->chan_per_stage = rs.s_CC;
        out->threads = v.threads();
        out->row_words = rs.s_Lw;
        out->work_ratio = rs.s_work_ratio;
    } else if (rs.fact >= 0) {
        const fdd::FactVariant& v = fdd::fact_variant(rs.fact);
        out->dm_per_block = v.bd();
        out->tile = v.tile();
        out->chan_per_stage = rs.f_CC;
        out->threads = v.threads();
        out->row_words = rs.f_Lw;
        out->work_ratio = rs.f_work_ratio;
    } else {
        const fdd::DedispVariant& v = fdd::dedisp_variant(rs.variant);
        out->dm_per_block = v.bd();
        out->tile = v.tile();
        out->chan_per_stage = rs.CC;
        out->threads = v.threads();
        out->row_words = rs.Lw;
        out->work_ratio = 1.f;
    }
    out->tuned_ms = rs.tuned_ms;
    return FDD_OK;
}

int fdd_plan_set_config(fdd_plan* plan, int32_t r, int32_t variant, int32_t chan_per_stage) {
    if (!plan || r < 0 || r >= static_cast<int32_t>(plan->ranges.size()) || chan_per_stage < 0)
        return fail(FDD_ERR_INVALID_ARG, "bad range index");
    RangeState& rs = plan->ranges[r];
    const int old_variant = range_variant_index(rs);
    const int old_cc = rs.sbf >= 0 ? rs.s_CC : (rs.fact >= 0 ? rs.f_CC : rs.CC);
    const int rc = configure_range(plan, rs, variant, chan_per_stage);
    if (rc != FDD_OK && old_variant >= 0) configure_range(plan, rs, old_variant, old_cc);
    if (rc == FDD_OK) rs.tuned_ms = 0.f;
    return rc;
}

int fdd_plan_autotune(fdd_plan* plan, const uint8_t* d_tabs, int64_t n_in, int64_t pitch, int64_t n_out,
                      void* d_workspace, size_t workspace_bytes, int32_t reps, fdd_stream_t stream) {
    {
        const int rc = check_search_args(plan, d_tabs, n_in, pitch, n_out, d_workspace, nullptr);
        if (rc != FDD_OK) return rc;
    }
    if (reps < 1) reps = 1;
    const Layout L = make_layout(plan, n_in, n_out, true, false, 1);  // plain searches: one scratch lane
    const Bins bins = search_bins(plan, n_out, 0, false);
    if (workspace_bytes < L.total) return fail(FDD_ERR_WORKSPACE, "workspace smaller than fdd_workspace_size()");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint8_t* ws = static_cast<uint8_t*>(d_workspace);
    int32_t* series = reinterpret_cast<int32_t*>(ws + L.series);
    unsigned long long* stat = reinterpret_cast<unsigned long long*>(ws + L.stat);
    cudaError_t e;
    for (size_t k = 0; k < plan->ds_factors.size(); k++) {
        e = fdd::launch_downsample(d_tabs, static_cast<int64_t>(plan->n_tab) * plan->n_chan, n_in, pitch,
                                   plan->ds_factors[k], reinterpret_cast<uint16_t*>(ws + L.ds_off[k]),
                                   L.ds_pitch[k], s);
        if (e != cudaSuccess) return cuda_fail(e, "downsample launch");
    }
    cudaEvent_t ev0, ev1;
    if ((e = cudaEventCreate(&ev0)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    if ((e = cudaEventCreate(&ev1)) != cudaSuccess) {
        cudaEventDestroy(ev0);
        return cuda_fail(e, "cudaEventCreate");
    }
    int rc = FDD_OK;
    for (size_t ri = 0; ri < plan->ranges.size() && rc == FDD_OK; ri++) {
        RangeState& r = plan->ranges[ri];
        if (n_out / r.D == 0) continue;
        const int E = (r.D == 1) ? 1 : 2;
        int best_v = r.variant, best_cc = r.CC;
        float best = 1e30f;
        for (int v = 0; v < fdd::num_dedisp_variants() && rc == FDD_OK; v++) {
            const fdd::DedispVariant& dv = fdd::dedisp_variant(v);
            if (dv.E != E) continue;
            const HostTables h = build_tables(plan, r, dv);
            if (h.Lw < 0) continue;
            bool uploaded = false;
            for (int cc : {8, 16, 32, 48, 64}) {
                if (!fdd::dedisp_cc_ok(dv, h.Lw, cc, kSmemBudget)) continue;
                if (!uploaded) {
                    free_range_tables(r);
                    if ((rc = upload_tables(&r.d_off, &r.d_base, h)) != FDD_OK) break;
                    uploaded = true;
                }
                r.variant = v;
                r.Lw = h.Lw;
                r.CC = cc;
                const fdd::DedispArgs a = dedisp_args(plan, r, ri, L, d_tabs, pitch, ws, series, stat, n_in, bins);
                if ((e = fdd::launch_dedisp(v, a, s)) != cudaSuccess) { rc = cuda_fail(e, "tuning launch"); break; }
                cudaEventRecord(ev0, s);
                for (int k = 0; k < reps && e == cudaSuccess; k++) e = fdd::launch_dedisp(v, a, s);
                cudaEventRecord(ev1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
                if (e != cudaSuccess) { rc = cuda_fail(e, "tuning launch"); break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev0, ev1);
                ms /= reps;
                if (std::getenv("FDD_TUNE_VERBOSE"))
                    std::fprintf(stderr, "fdd tune: range %zu variant %d (bd %d tile %d threads %d) cc %d: %.4f ms\n",
                                 ri, v, dv.bd(), dv.tile(), dv.threads(), cc, ms);
                if (ms < best) {
                    best = ms;
                    best_v = v;
                    best_cc = cc;
                }
            }
        }
        for (int fv = 0; fv < fdd::num_fact_variants() && rc == FDD_OK; fv++) {
            if (!fdd::fact_has_width(fv, E, false)) continue;
            for (int cc : {16, 32, 48, 64}) {
                if (configure_fact(plan, r, fv, cc) != FDD_OK) continue;  // does not fit
                const fdd::DedispArgs a = dedisp_args(plan, r, ri, L, d_tabs, pitch, ws, series, stat, n_in, bins);
                if ((e = launch_range_dedisp(plan, r, a, s)) != cudaSuccess) { rc = cuda_fail(e, "tuning launch"); break; }
                cudaEventRecord(ev0, s);
                for (int k = 0; k < reps && e == cudaSuccess; k++) e = launch_range_dedisp(plan, r, a, s);
                cudaEventRecord(ev1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
                if (e != cudaSuccess) { rc = cuda_fail(e, "tuning launch"); break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev0, ev1);
                ms /= reps;
                if (std::getenv("FDD_TUNE_VERBOSE")) {
                    const fdd::FactVariant& fvv = fdd::fact_variant(fv);
                    std::fprintf(stderr, "fdd tune: range %zu factored variant %d (G %d bd %d tile %d) cc %d: %.4f ms\n",
                                 ri, fdd::num_dedisp_variants() + fv, fvv.G, fvv.bd(), fvv.tile(), cc, ms);
                }
                if (ms < best) {
                    best = ms;
                    best_v = fdd::num_dedisp_variants() + fv;
                    best_cc = cc;
                }
            }
        }
        const int nbf = fdd::num_dedisp_variants() + fdd::num_fact_variants();
        for (int sv = 0; plan->n_sb >= 2 && sv < fdd::num_sbf_variants() && rc == FDD_OK; sv++) {
            if (fdd::sbf_variant(sv).E != E) continue;
            for (int cc : {16, 32, 48, 64}) {
                if (configure_range(plan, r, nbf + sv, cc) != FDD_OK) continue;  // does not fit
                const fdd::DedispArgs a = dedisp_args(plan, r, ri, L, d_tabs, pitch, ws, series, stat, n_in, bins);
                if ((e = launch_range(plan, r, a, L, ws, s)) != cudaSuccess) { rc = cuda_fail(e, "tuning launch"); break; }
                cudaEventRecord(ev0, s);
                for (int k = 0; k < reps && e == cudaSuccess; k++) e = launch_range(plan, r, a, L, ws, s);
                cudaEventRecord(ev1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
                if (e != cudaSuccess) { rc = cuda_fail(e, "tuning launch"); break; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev0, ev1);
                ms /= reps;
                if (std::getenv("FDD_TUNE_VERBOSE")) {
                    const fdd::DedispVariant& dv = fdd::sbf_variant(sv);
                    std::fprintf(stderr, "fdd tune: range %zu SB-factored variant %d (bd %d tile %d) cc %d: %.4f ms\n",
                                 ri, nbf + sv, dv.bd(), dv.tile(), cc, ms);
                }
                if (ms < best) {
                    best = ms;
                    best_v = nbf + sv;
                    best_cc = cc;
                }
            }
        }
        if (rc == FDD_OK) {
            rc = configure_range(plan, r, best_v, best_cc);
            if (rc == FDD_OK) r.tuned_ms = best;
        }
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    return rc;
}

int fdd_fact_tables_host(const fdd_plan_desc* desc, const int16_t* sb_map_host, int32_t range, int32_t variant,
                         int32_t chan_per_stage, int64_t* info, int32_t* base, int32_t* goff, int32_t* pdesc,
                         int32_t* pd_idx, int32_t* delays, int32_t* bbase) {
    if (!info) return fail(FDD_ERR_INVALID_ARG, "null info");
    fdd_plan p;
    int rc = build_host_plan(desc, sb_map_host, &p);
    if (rc != FDD_OK) return rc;
    const int fv = variant - fdd::num_dedisp_variants();
    if (range < 0 || range >= static_cast<int32_t>(p.ranges.size()) || fv < 0 || fv >= fdd::num_fact_variants() ||
        chan_per_stage < 1)
        return fail(FDD_ERR_INVALID_ARG, "bad range, variant or stage size");
    const fdd::FactVariant& v = fdd::fact_variant(fv);
    if (chan_per_stage % v.G) return fail(FDD_ERR_INVALID_ARG, "stage size must be a multiple of G");
    const RangeState& r = p.ranges[range];
    const FactTables ft = build_fact_tables(&p, r, v, chan_per_stage, p.n_tab == 1);
    const int64_t n_blk = (r.n_dm + v.bd() - 1) / v.bd();
    info[0] = ft.Lw;
    info[1] = ft.pat_bytes;
    info[2] = ft.n_groups;
    info[3] = ft.n_stages;
    info[4] = ft.desc_ints;
    info[5] = static_cast<int64_t>(ft.smem_bytes);
    info[6] = ft.desc_ints ? static_cast<int64_t>(ft.pdesc.size()) / ft.desc_ints : 0;
    info[7] = n_blk;
    info[8] = ft.zero_off;
    info[9] = ft.raw_off;
    info[10] = ft.rb;
    info[11] = ft.pat_off;
    info[12] = ft.bar_off;
    info[13] = ft.pat_bufs;
    info[14] = ft.box_rows;
    if (ft.Lw < 0) return FDD_OK;
    if (base) std::memcpy(base, ft.base.data(), ft.base.size() * sizeof(int32_t));
    if (goff) std::memcpy(goff, ft.goff.data(), ft.goff.size() * sizeof(int32_t));
    if (pdesc) std::memcpy(pdesc, ft.pdesc.data(), ft.pdesc.size() * sizeof(int32_t));
    if (pd_idx) std::memcpy(pd_idx, ft.pd_idx.data(), ft.pd_idx.size() * sizeof(int32_t));
    if (delays) std::memcpy(delays, r.delay.data(), r.delay.size() * sizeof(int32_t));
    if (bbase && !ft.bbase.empty()) std::memcpy(bbase, ft.bbase.data(), ft.bbase.size() * sizeof(int32_t));
    return FDD_OK;
}

int fdd_plan_set_subband(fdd_plan* plan, int32_t r, int32_t chan_per_subband, int32_t dm_per_coarse) {
    if (!plan || r < 0 || r >= static_cast<int32_t>(plan->ranges.size()) || chan_per_subband < 0 || dm_per_coarse < 0)
        return fail(FDD_ERR_INVALID_ARG, "bad argument");
    RangeState& rs = plan->ranges[r];
    if (rs.sub_G == 0) rs.sub_dmax_exact = rs.dmax;
    if (chan_per_subband == 0) {
        free_subband_tables(rs);
        rs.dmax = rs.sub_dmax_exact;
    } else {
        const int rc = configure_subband(plan, rs, chan_per_subband, dm_per_coarse);
        if (rc != FDD_OK) return rc;
        rs.dmax = std::max(rs.sub_dmax_exact, rs.sub_d1max + rs.sub_d2max);
    }
    plan->max_delay_native = 0;
    for (const RangeState& q : plan->ranges)
        plan->max_delay_native = std::max<int64_t>(plan->max_delay_native, static_cast<int64_t>(q.dmax) * q.D);
    return FDD_OK;
}

int fdd_plan_get_subband(const fdd_plan* plan, int32_t r, int32_t* chan_per_subband, int32_t* dm_per_coarse) {
    if (!plan || r < 0 || r >= static_cast<int32_t>(plan->ranges.size()) || !chan_per_subband || !dm_per_coarse)
        return fail(FDD_ERR_INVALID_ARG, "bad argument");
    *chan_per_subband = plan->ranges[r].sub_G;
    *dm_per_coarse = plan->ranges[r].sub_K;
    return FDD_OK;
}

int fdd_plan_set_scratch_limit(fdd_plan* plan, int64_t bytes) {
    if (!plan || bytes < 0) return fail(FDD_ERR_INVALID_ARG, "bad argument");
    plan->sbf_scratch_cap = bytes > 0 ? static_cast<size_t>(bytes) : kSbfScratchMax;
    return FDD_OK;
}

int fdd_plan_set_timing(fdd_plan* plan, int32_t enable) {
    if (!plan) return fail(FDD_ERR_INVALID_ARG, "null plan");
    plan->timing = enable != 0;
    return FDD_OK;
}

int fdd_plan_stage_times(fdd_plan* plan, int32_t max_n, int32_t* kind, int32_t* range, float* ms,
                         int32_t* n_stages) {
    if (!plan || !n_stages || max_n < 0 || (max_n > 0 && (!kind || !range || !ms)))
        return fail(FDD_ERR_INVALID_ARG, "bad argument");
    const int32_t n = static_cast<int32_t>(plan->st_kind.size());
    *n_stages = n;
    for (int32_t k = 0; k < n && k < max_n; k++) {
        kind[k] = plan->st_kind[k];
        range[k] = plan->st_range[k];
        const cudaError_t e = cudaEventElapsedTime(&ms[k], plan->ev[2 * k], plan->ev[2 * k + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "stage timing not ready");
    }
    return FDD_OK;
}

int fdd_downsample_u8(const uint8_t* d_in, int64_t n_rows, int64_t n_in, int64_t in_pitch, int32_t downsamp,
                      uint16_t* d_out, int64_t out_pitch, fdd_stream_t stream) {
    if (!d_in || !d_out || n_rows < 0 || n_in < 0 || in_pitch < n_in || downsamp < 1 || downsamp > 257 ||
        out_pitch < n_in / downsamp)
        return fail(FDD_ERR_INVALID_ARG, "bad downsample argument");
    if ((reinterpret_cast<uintptr_t>(d_in) & 15) || (reinterpret_cast<uintptr_t>(d_out) & 15) || (in_pitch & 15) ||
        (out_pitch & 7))
        return fail(FDD_ERR_MISALIGNED, "downsample buffers must be 16-byte aligned, out_pitch a multiple of 8");
    cudaError_t e = fdd::launch_downsample(d_in, n_rows, n_in, in_pitch, downsamp, d_out, out_pitch,
                                           reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "downsample launch");
    return FDD_OK;
}

}  // extern "C"
