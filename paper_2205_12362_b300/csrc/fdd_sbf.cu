// fdd_sbf.cu -- host side of the SB-factored dedispersion: channel segments,
// channel stages, per-range configuration and the slab loop (kernels in
// k_sbf.cu).
//
// Segments: maximal runs of consecutive channels on which every SB takes
// the same TAB throughout, cut to at most min(CC, 65535 / (255 D)) channels
// so a segment's sum of D-sample sums fits a 16-bit lane and a segment fits
// one channel stage.  Stages: whole segments packed into at most CC
// channels.  The scratch is sized for segments cut at 16 channels, which
// no configuration with CC >= 16 exceeds in number.  The partial sums of a slab of
// DM trials, [n_tab][n_seg][slab][Np] uint16, live in a scratch region of
// the search workspace bounded by kSbfScratchMax; the slab is the largest
// multiple of the variant's DM block that fits.
#include <algorithm>

#include "fdd_plan_impl.h"

using namespace fdd::host;

namespace {

int64_t round_up64(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

int64_t sbf_np(int64_t nr) { return round_up64(std::max<int64_t>(nr, 1), 512); }

template <typename T>
int upload(T** dst, const std::vector<T>& v, const char* what) {
    cudaError_t e = cudaMalloc(dst, std::max<size_t>(v.size(), 1) * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (!v.empty() && (e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, what);
    return FDD_OK;
}

// Slab of DM trials whose partial sums fit the scratch (a multiple of BD).
int64_t slab_trials(const fdd_plan* p, const RangeState& r, int64_t nr, int BD, size_t scratch_bytes) {
    const int64_t per_trial = static_cast<int64_t>(p->n_tab) * static_cast<int64_t>(r.s_n_seg) * sbf_np(nr) * 2;
    int64_t slab = static_cast<int64_t>(scratch_bytes) / per_trial / BD * BD;
    return std::min<int64_t>(slab, round_up64(r.n_dm, BD));
}

}  // namespace

namespace fdd {
namespace host {

std::vector<int2> sbf_segments(const fdd_plan* p, int D, int cap) {
    const int max_len = std::max(1, std::min(cap, 65535 / (255 * D)));
    std::vector<int2> segs;
    int c0 = 0;
    for (int c = 1; c <= p->n_chan; c++) {
        bool cut = c == p->n_chan || c - c0 == max_len;
        for (int s = 0; !cut && s < p->n_sb; s++)
            cut = p->sb_map[static_cast<size_t>(s) * p->n_chan + c] != p->sb_map[static_cast<size_t>(s) * p->n_chan + c - 1];
        if (cut) {
            segs.push_back(make_int2(c0, c - c0));
            c0 = c;
        }
    }
    return segs;
}

size_t sbf_scratch_bytes(const fdd_plan* p, int64_t n_out) {
    if (p->n_sb < 2) return 0;
    size_t bytes = 0;
    for (const RangeState& r : p->ranges) {
        const int64_t nr = n_out / r.D;
        if (nr == 0) continue;
        const size_t per_trial = static_cast<size_t>(p->n_tab) * r.segs.size() * static_cast<size_t>(sbf_np(nr)) * 2;
        const size_t full = per_trial * static_cast<size_t>(round_up64(r.n_dm, 64));
        const size_t one_block = per_trial * 64;
        bytes = std::max(bytes, std::min(full, std::max(p->sbf_scratch_cap, one_block)));
        // the persistent batched mode keeps kSbfSlots slabs of 32 trials (+ 1 KB alignment per slab)
        bytes = std::max(bytes, (per_trial * 32 + 2048) * static_cast<size_t>(fdd::kSbfSlots));
    }
    return align_up(bytes, 256);
}

double sbf_work_ratio(const fdd_plan* p, const RangeState& r) {
    // per (trial, sample): n_tab * n_chan partial adds + n_sb * n_seg combine adds
    const double brute = static_cast<double>(p->n_sb) * p->n_chan;
    const double fact = static_cast<double>(p->n_tab) * p->n_chan + static_cast<double>(p->n_sb) * r.s_n_seg;
    return fact / brute;
}

void free_sbf_tables(RangeState& r, bool geometry) {
    for (int32_t** ptr : {&r.d_sbase, &r.d_soff}) {
        if (*ptr) cudaFree(*ptr);
        *ptr = nullptr;
    }
    if (r.d_sstages) cudaFree(r.d_sstages);
    r.d_sstages = nullptr;
    if (r.s_fact >= 0) {  // the pattern-factored part's tables
        for (int32_t** ptr : {&r.d_fbase, &r.d_goff, &r.d_pdesc, &r.d_pdidx, &r.d_fbbase}) {
            if (*ptr) cudaFree(*ptr);
            *ptr = nullptr;
        }
    }
    if (r.d_fsseg) cudaFree(r.d_fsseg);
    r.d_fsseg = nullptr;
    r.s_fact = -1;
    r.sbf = -1;
    if (geometry) {
        if (r.d_segs) cudaFree(r.d_segs);
        if (r.d_segtab) cudaFree(r.d_segtab);
        r.d_segs = nullptr;
        r.d_segtab = nullptr;
    }
}

namespace {

// Segment table and per-SB TAB table of the combine step for segments `segs`.
int upload_segments(fdd_plan* p, RangeState& r, const std::vector<int2>& segs) {
    int rc;
    if ((rc = upload(&r.d_segs, segs, "segment table")) != FDD_OK) return rc;
    r.seg_pitch = static_cast<int32_t>(round_up64(static_cast<int64_t>(segs.size()), 8));  // whole 8-segment chunks
    std::vector<uint8_t> tab(static_cast<size_t>(p->n_sb) * r.seg_pitch, 0);
    for (int s = 0; s < p->n_sb; s++)
        for (size_t g = 0; g < segs.size(); g++)
            tab[static_cast<size_t>(s) * r.seg_pitch + g] =
                static_cast<uint8_t>(p->sb_map[static_cast<size_t>(s) * p->n_chan + segs[g].x]);
    if ((rc = upload(&r.d_segtab, tab, "segment TAB table")) != FDD_OK) return rc;
    int seg_max = 1;
    for (const int2& sg : segs) seg_max = std::max(seg_max, sg.y);
    r.s_n_seg = static_cast<int32_t>(segs.size());
    r.s_flush = std::max(1, 65535 / (seg_max * 255 * r.D));
    return FDD_OK;
}

// SB-factored variant sv whose partial sums come from pattern-factored variant fdd::sbf_fact_variant(sv)
// in part mode (every segment a run of whole channel groups; raw or downsampled rows by the variant's E).
int configure_sbf_fact(fdd_plan* p, RangeState& r, int sv, int CC) {
    const int fvi = fdd::sbf_fact_variant(sv);
    if (fdd::sbf_variant(sv).E != (r.D == 1 ? 1 : 2) || !fdd::fact_has_width(fvi, r.D == 1 ? 1 : 2, true))
        return fail(FDD_ERR_INVALID_ARG, "kernel variant for the wrong sample width");
    const fdd::FactVariant& v = fdd::fact_variant(fvi);
    const std::vector<int2> segs = sbf_segments(p, r.D, 16);
    if (segs.size() > r.segs.size()) return fail(FDD_ERR_UNSUPPORTED, "more segments than the scratch was sized for");
    for (const int2& sg : segs)
        if (sg.x % v.G != 0 || ((sg.x + sg.y) % v.G != 0 && sg.x + sg.y != p->n_chan))
            return fail(FDD_ERR_UNSUPPORTED, "channel segments are not whole channel groups of the pattern-factored part");
    FactTables best;
    int cc_pick = 0;
    for (int cc : {64, 48, 32, 16, 8, 4}) {
        if (CC != 0 && cc != CC) continue;
        if (cc % v.G) continue;
        FactTables ft = build_fact_tables(p, r, v, cc, true);  // one TAB per block: consecutive rows
        if (ft.Lw < 0 || !fdd::fact_cc_ok(v, ft.Lw, cc, ft.max_desc) || ft.smem_bytes > kSmemBudget) continue;
        best = std::move(ft);
        cc_pick = cc;
        break;
    }
    if (cc_pick == 0) return fail(FDD_ERR_UNSUPPORTED, "pattern-factored part does not fit this range and stage size");
    // per stage: bit gl set if group gl closes its segment; the segment of the stage's first group
    const int gps = cc_pick / v.G;
    const int n_groups = (p->n_chan + v.G - 1) / v.G;
    std::vector<int32_t> seg_of(p->n_chan);
    for (size_t u = 0; u < segs.size(); u++)
        for (int c = segs[u].x; c < segs[u].x + segs[u].y; c++) seg_of[c] = static_cast<int32_t>(u);
    std::vector<int2> sseg(best.n_stages);
    for (int st = 0; st < best.n_stages; st++) {
        int mask = 0;
        for (int gl = 0; gl < gps; gl++) {
            const int g = st * gps + gl;
            if (g >= n_groups) break;
            const int c_end = std::min(p->n_chan, (g + 1) * v.G);  // one past the group's last channel
            const int2 sg = segs[seg_of[c_end - 1]];
            if (c_end == sg.x + sg.y) mask |= 1 << gl;
        }
        sseg[st] = make_int2(mask, seg_of[st * cc_pick]);
    }
    free_sbf_tables(r, true);
    // the tables of a pattern-factored configuration of this range
    for (int32_t** ptr : {&r.d_fbase, &r.d_goff, &r.d_pdesc, &r.d_pdidx, &r.d_fbbase}) {
        if (*ptr) cudaFree(*ptr);
        *ptr = nullptr;
    }
    r.fact = -1;
    int rc;
    if ((rc = upload_segments(p, r, segs)) != FDD_OK) return rc;
    r.s_fact = fvi;  // from here free_sbf_tables also frees the tables below
    if ((rc = upload(&r.d_fbase, best.base, "factored base table")) != FDD_OK) return rc;
    if ((rc = upload(&r.d_goff, best.goff, "factored offset table")) != FDD_OK) return rc;
    if ((rc = upload(&r.d_pdesc, best.pdesc, "factored descriptors")) != FDD_OK) return rc;
    if ((rc = upload(&r.d_pdidx, best.pd_idx, "factored descriptor index")) != FDD_OK) return rc;
    if ((rc = upload(&r.d_fsseg, sseg, "segment closings per stage")) != FDD_OK) return rc;
    if ((rc = upload(&r.d_fbbase, best.bbase, "factored box starts")) != FDD_OK) return rc;
    r.f_box_rows = best.box_rows;
    r.f_CC = cc_pick;
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
    r.sbf = sv;
    r.s_CC = cc_pick;
    r.s_Lw = best.Lw;
    r.s_n_stages = best.n_stages;
    // per (trial, sample): the pattern-factored adds of n_tab TABs' partials + n_sb * n_seg combine adds
    r.s_work_ratio = static_cast<float>((static_cast<double>(p->n_tab) * p->n_chan * best.work_ratio +
                                         static_cast<double>(p->n_sb) * r.s_n_seg) /
                                        (static_cast<double>(p->n_sb) * p->n_chan));
    return FDD_OK;
}

}  // namespace

// Configure range r for SB-factored variant sv with CC channels per stage
// (0 = the largest that fits).  Tables of other kernels are left to the caller.
int configure_sbf(fdd_plan* p, RangeState& r, int sv, int CC) {
    if (sv < 0 || sv >= fdd::num_sbf_variants()) return fail(FDD_ERR_INVALID_ARG, "kernel variant out of range");
    if (p->n_sb < 2) return fail(FDD_ERR_UNSUPPORTED, "the SB-factored kernel needs at least two SBs");
    if (fdd::sbf_comb_smem_bytes(p->n_tab) > kSmemBudget)
        return fail(FDD_ERR_UNSUPPORTED, "too many TABs for the SB-factored kernel's shared-memory rows");
    if (fdd::sbf_fact_variant(sv) >= 0) return configure_sbf_fact(p, r, sv, CC);
    const fdd::DedispVariant& v = fdd::sbf_variant(sv);
    if (v.E != (r.D == 1 ? 1 : 2)) return fail(FDD_ERR_INVALID_ARG, "kernel variant for the wrong sample width");
    const HostTables h = build_tables(p, r, v);
    if (h.Lw < 0) return fail(FDD_ERR_UNSUPPORTED, "DM step too large for one block's staged rows");
    int cc_pick = 0;
    std::vector<int2> segs;
    for (int cc : {64, 48, 32, 16, 8, 4, 2, 1}) {
        if (CC != 0 && cc != CC) continue;
        if (!fdd::sbf_cc_ok(v, h.Lw, cc, kSmemBudget)) continue;
        std::vector<int2> sg = sbf_segments(p, r.D, cc);
        if (sg.size() > r.segs.size()) continue;  // more segments than the scratch was sized for
        cc_pick = cc;
        segs.swap(sg);
        break;
    }
    if (cc_pick == 0) return fail(FDD_ERR_UNSUPPORTED, "SB-factored kernel does not fit this range and stage size");
    std::vector<int4> stages;
    for (size_t g = 0; g < segs.size(); g++) {
        const int2 sg = segs[g];
        if (!stages.empty() && stages.back().y + sg.y <= cc_pick) {
            stages.back().y += sg.y;
            stages.back().w += 1;
        } else {
            stages.push_back(make_int4(sg.x, sg.y, static_cast<int>(g), 1));
        }
    }
    free_sbf_tables(r, true);
    int rc;
    if ((rc = upload_segments(p, r, segs)) != FDD_OK) return rc;
    if ((rc = upload(&r.d_sbase, h.base, "base table")) != FDD_OK) return rc;
    if ((rc = upload(&r.d_soff, h.off, "offset table")) != FDD_OK) return rc;
    if ((rc = upload(&r.d_sstages, stages, "stage table")) != FDD_OK) return rc;
    r.sbf = sv;
    r.s_CC = cc_pick;
    r.s_Lw = h.Lw;
    r.s_n_stages = static_cast<int32_t>(stages.size());
    r.s_work_ratio = static_cast<float>(sbf_work_ratio(p, r));
    return FDD_OK;
}

int configure_sbf_default(fdd_plan* p, RangeState& r) {
    int rc = fail(FDD_ERR_UNSUPPORTED, "no SB-factored variant fits this range");
    for (int sv = 0; sv < fdd::num_sbf_variants(); sv++) {
        if (fdd::sbf_variant(sv).E != (r.D == 1 ? 1 : 2)) continue;
        if ((rc = configure_sbf(p, r, sv, 0)) == FDD_OK) return FDD_OK;
    }
    return rc;
}

cudaError_t launch_range_sbf(const fdd_plan* p, const RangeState& r, const fdd::DedispArgs& a, uint8_t* scratch,
                             size_t scratch_bytes, cudaStream_t s, int64_t* launches) {
    const fdd::DedispVariant& v = fdd::sbf_variant(r.sbf);
    const int BD = r.s_fact >= 0 ? fdd::fact_variant(r.s_fact).bd() : v.bd();
    const int64_t nr = a.n_out;
    const int64_t Np = sbf_np(nr);
    const int64_t slab = slab_trials(p, r, nr, BD, scratch_bytes);
    if (slab < BD) return cudaErrorInvalidValue;  // scratch sized by sbf_scratch_bytes always holds one block
    const int64_t n_seg = r.s_n_seg;
    fdd::SbfPartArgs pa{};
    pa.in = a.in;
    pa.pitch_bytes = a.pitch_bytes;
    pa.n_valid = a.n_valid;
    pa.base = r.d_sbase;
    pa.off = r.d_soff;
    pa.stages = r.d_sstages;
    pa.segs = r.d_segs;
    pa.P = reinterpret_cast<uint16_t*>(scratch);
    pa.seg_stride = slab * Np;
    pa.tab_stride = n_seg * slab * Np;
    pa.Np = static_cast<int32_t>(Np);
    pa.n_chan = p->n_chan;
    pa.n_dm = r.n_dm;
    pa.n_out = a.n_out;
    pa.Lw = r.s_Lw;
    pa.CC = r.s_CC;
    pa.n_stages = r.s_n_stages;
    fdd::SbfCombArgs ca{};
    ca.P = pa.P;
    ca.tab_stride = pa.tab_stride;
    ca.seg_stride = pa.seg_stride;
    ca.Np = pa.Np;
    ca.seg_tab = r.d_segtab;
    ca.seg_pitch = r.seg_pitch;
    ca.series = a.series;
    ca.stat = a.stat;
    ca.n_sb = p->n_sb;
    ca.n_seg = static_cast<int32_t>(n_seg);
    ca.n_dm = r.n_dm;
    ca.n_out = a.n_out;
    ca.n_emit = a.n_emit;
    ca.flush = r.s_flush;
    ca.n_tab = p->n_tab;
    ca.uc = fdd::sbf_comb_uc(p->n_tab);
    ca.status = p->d_status;
    if (cudaError_t e = fdd::encode_comb_map(ca); e != cudaSuccess) return e;
    fdd::FactArgs fa{};  // pattern-factored part (r.s_fact >= 0)
    if (r.s_fact >= 0) {
        fa.status = p->d_status;
        fa.in = a.in;
        fa.pitch_bytes = a.pitch_bytes;
        fa.n_valid = a.n_valid;
        fa.E = r.D == 1 ? 1 : 2;
        fa.fold_ch = 256 / r.D;  // unused in part mode (segments fit the 16-bit lanes)
        fa.base = r.d_fbase;
        fa.goff = r.d_goff;
        fa.pdesc = r.d_pdesc;
        fa.pd_idx = r.d_pdidx;
        fa.bbase = r.d_fbbase;
        fa.box_rows = r.f_box_rows;
        fa.n_chan = p->n_chan;
        fa.n_dm = r.n_dm;
        fa.n_out = a.n_out;
        fa.n_emit = a.n_emit;
        fa.n_sb = p->n_sb;
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
        fa.P = pa.P;
        fa.tab_stride = pa.tab_stride;
        fa.seg_stride = pa.seg_stride;
        fa.Np = pa.Np;
        fa.sseg = r.d_fsseg;
        if (cudaError_t e = fdd::encode_fact_map(fa, static_cast<int64_t>(p->n_tab) * p->n_chan); e != cudaSuccess)
            return e;
    }
    for (int64_t i0 = 0; i0 < r.n_dm; i0 += slab) {
        pa.i0 = static_cast<int32_t>(i0);
        pa.n_slab = static_cast<int32_t>(std::min<int64_t>(slab, r.n_dm - i0));
        cudaError_t e;
        if (r.s_fact >= 0) {
            fa.i0 = pa.i0;
            fa.n_slab = pa.n_slab;
            e = fdd::launch_sbf_part_fact(r.s_fact, fa, r.f_smem, p->n_tab, s);
        } else {
            e = fdd::launch_sbf_part(r.sbf, pa, p->n_tab, s);
        }
        if (e != cudaSuccess) return e;
        ca.i0 = pa.i0;
        ca.n_slab = pa.n_slab;
        if ((e = fdd::launch_sbf_comb(ca, s)) != cudaSuccess) return e;
        if (launches) *launches += 2;
    }
    return cudaSuccess;
}

}  // namespace host
}  // namespace fdd
