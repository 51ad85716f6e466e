// fdd_subband.cu -- two-step subband dedispersion (approximate), built from
// the library's own kernels.
//
// The paper's AMBER dedisperses "in a single step, or using a more efficient
// two step process including subbanding" (Sec. "AMBER", "Dedispersion";
// Table "dedispersion setup": 32 subbands, subbanding DM step 32x the fine
// step).  With subbands of G channels and coarse blocks of K fine trials:
//   step 1: P[tab][b][q][u] = sum_{c in b} y[tab][c][u + d1[q][c]], the
//           subband's channels aligned to its top channel at the block's
//           midpoint DM -- the SB-factored "part" kernel run on a delay table
//           of coarse DMs with subbands as segments;
//   step 2: S[s][i][t] = sum_b P[tab(s,b)][b][q(i)][t + d2[i][b]], the
//           subbands aligned at the fine DM -- the brute-force kernel on
//           uint16 rows (tab, b) of P, each DM block reading the rows of its
//           coarse block (K a multiple of the block's BD).
// Delays use the plan's law and rounding with the subband's top channel as
// reference (d1) and as channel (d2).  The SB map must be constant within
// each subband.  The result is exact for this definition (integer sums),
// approximate against brute force; fdd_search uses it for a range once
// fdd_plan_set_subband selects it.
#include <algorithm>
#include <cmath>

#include "fdd_plan_impl.h"

using namespace fdd::host;

namespace {

int64_t round_up64(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
int64_t sub_np(int64_t n1) { return round_up64(std::max<int64_t>(n1, 1), 512); }

template <typename T>
int upload(T** dst, const std::vector<T>& v, const char* what) {
    cudaError_t e = cudaMalloc(dst, std::max<size_t>(v.size(), 1) * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (!v.empty() && (e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, what);
    return FDD_OK;
}

template <typename T>
void release(T** ptr) {
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
}

}  // namespace

namespace fdd {
namespace host {

void free_subband_tables(RangeState& r) {
    release(&r.d_sub_pbase);
    release(&r.d_sub_poff);
    release(&r.d_sub_pstages);
    release(&r.d_sub_psegs);
    release(&r.d_sub_bbase);
    release(&r.d_sub_boff);
    release(&r.d_sub_sbmap);
    r.sub_G = r.sub_K = 0;
    r.sub_pv = r.sub_bv = -1;
}

size_t subband_scratch_bytes(const fdd_plan* p, int64_t n_out) {
    size_t bytes = 0;
    for (const RangeState& r : p->ranges) {
        if (r.sub_G <= 0) continue;
        const int64_t n1 = n_out / r.D + r.sub_d2max;
        bytes = std::max(bytes, static_cast<size_t>(p->n_tab) * r.sub_n * r.sub_nq * sub_np(n1) * 2);
    }
    return bytes ? align_up(bytes, 256) : 0;
}

int configure_subband(fdd_plan* p, RangeState& r, int G, int K) {
    const int E = r.D == 1 ? 1 : 2;
    if (G < 1 || K < 1 || G > 64 || G > 65535 / (255 * r.D))
        return fail(FDD_ERR_INVALID_ARG, "subband size must be 1..64 channels and keep a subband sum within 16 bits");
    const int n_sub = (p->n_chan + G - 1) / G;
    for (int s = 0; s < p->n_sb; s++)
        for (int c = 0; c < p->n_chan; c++)
            if (p->sb_map[static_cast<size_t>(s) * p->n_chan + c] != p->sb_map[static_cast<size_t>(s) * p->n_chan + c / G * G])
                return fail(FDD_ERR_UNSUPPORTED, "the SB map changes TAB inside a subband");
    const int n_q = (r.n_dm + K - 1) / K;
    // reference (top) frequency per subband, delays of both steps (plan's law and rounding)
    std::vector<double> f_ref(n_sub);
    for (int b = 0; b < n_sub; b++) {
        f_ref[b] = p->freq[b * G];
        for (int c = b * G; c < std::min(p->n_chan, (b + 1) * G); c++) f_ref[b] = std::max(f_ref[b], p->freq[c]);
    }
    const double f_top = *std::max_element(p->freq.begin(), p->freq.end());
    const double tD = static_cast<double>(r.D) * p->t_samp;
    RangeState s1;  // step 1: coarse DMs x channels
    s1.n_dm = n_q;
    s1.D = r.D;
    s1.delay.resize(static_cast<size_t>(n_q) * p->n_chan);
    int32_t d1max = 0, d2max = 0;
    for (int q = 0; q < n_q; q++) {
        const double dmc = r.dm0 + (static_cast<double>(q) * K + 0.5 * static_cast<double>(K - 1)) * r.ddm;
        for (int c = 0; c < p->n_chan; c++) {
            const double f = p->freq[c], fb = f_ref[c / G];
            const long long d = std::llround(((kDispersionConstant * dmc) * (1.0 / (f * f) - 1.0 / (fb * fb))) / tD);
            if (d < 0 || d > (1LL << 28)) return fail(FDD_ERR_UNSUPPORTED, "subband delay out of range");
            s1.delay[static_cast<size_t>(q) * p->n_chan + c] = static_cast<int32_t>(d);
            d1max = std::max<int32_t>(d1max, static_cast<int32_t>(d));
        }
    }
    RangeState s2;  // step 2: fine DMs x subbands
    s2.n_dm = r.n_dm;
    s2.D = r.D;
    s2.delay.resize(static_cast<size_t>(r.n_dm) * n_sub);
    for (int i = 0; i < r.n_dm; i++) {
        const double dm = r.dm0 + static_cast<double>(i) * r.ddm;
        for (int b = 0; b < n_sub; b++) {
            const double fb = f_ref[b];
            const long long d = std::llround(((kDispersionConstant * dm) * (1.0 / (fb * fb) - 1.0 / (f_top * f_top))) / tD);
            if (d < 0 || d > (1LL << 28)) return fail(FDD_ERR_UNSUPPORTED, "subband delay out of range");
            s2.delay[static_cast<size_t>(i) * n_sub + b] = static_cast<int32_t>(d);
            d2max = std::max<int32_t>(d2max, static_cast<int32_t>(d));
        }
    }
    // step 1 kernel: an SB-factored part variant of this sample width whose stages hold a subband
    int pv = -1, pCC = 0;
    HostTables h1;
    for (int v = 0; v < fdd::num_sbf_variants() && pv < 0; v++) {
        const fdd::DedispVariant& dv = fdd::sbf_variant(v);
        if (dv.E != E) continue;
        HostTables h = build_tables(p, s1, dv);
        if (h.Lw < 0) continue;
        for (int cc : {64, 48, 32, 16, 8, 4, 2, 1}) {
            if (cc < G || !fdd::sbf_cc_ok(dv, h.Lw, cc, kSmemBudget)) continue;
            pv = v;
            pCC = cc;
            h1 = std::move(h);
            break;
        }
    }
    if (pv < 0) return fail(FDD_ERR_UNSUPPORTED, "no kernel stage holds a subband of this size");
    // step 2 kernel: a brute-force uint16 variant whose DM block divides K
    fdd_plan p2;
    p2.n_chan = n_sub;
    int bv = -1, bCC = 0;
    HostTables h2;
    for (int v = 0; v < fdd::num_dedisp_variants() && bv < 0; v++) {
        const fdd::DedispVariant& dv = fdd::dedisp_variant(v);
        if (dv.E != 2 || K % dv.bd() != 0) continue;
        HostTables h = build_tables(&p2, s2, dv);
        if (h.Lw < 0) continue;
        const int cc = pick_cc(dv, h.Lw);
        if (cc == 0) continue;
        bv = v;
        bCC = cc;
        h2 = std::move(h);
    }
    if (bv < 0) return fail(FDD_ERR_UNSUPPORTED, "no subband-combining kernel's DM block divides the coarse block");
    std::vector<int4> stages;
    std::vector<int2> segs;
    for (int b = 0; b < n_sub; b++) {
        const int c0 = b * G, nc = std::min(p->n_chan, c0 + G) - c0;
        segs.push_back(make_int2(c0, nc));
        if (!stages.empty() && stages.back().y + nc <= pCC) {
            stages.back().y += nc;
            stages.back().w += 1;
        } else {
            stages.push_back(make_int4(c0, nc, b, 1));
        }
    }
    std::vector<int16_t> sbmap(static_cast<size_t>(p->n_sb) * n_sub);
    for (int s = 0; s < p->n_sb; s++)
        for (int b = 0; b < n_sub; b++)
            sbmap[static_cast<size_t>(s) * n_sub + b] = p->sb_map[static_cast<size_t>(s) * p->n_chan + b * G];
    free_subband_tables(r);
    int rc;
    if ((rc = upload(&r.d_sub_pbase, h1.base, "subband tables")) != FDD_OK ||
        (rc = upload(&r.d_sub_poff, h1.off, "subband tables")) != FDD_OK ||
        (rc = upload(&r.d_sub_pstages, stages, "subband tables")) != FDD_OK ||
        (rc = upload(&r.d_sub_psegs, segs, "subband tables")) != FDD_OK ||
        (rc = upload(&r.d_sub_bbase, h2.base, "subband tables")) != FDD_OK ||
        (rc = upload(&r.d_sub_boff, h2.off, "subband tables")) != FDD_OK ||
        (rc = upload(&r.d_sub_sbmap, sbmap, "subband tables")) != FDD_OK) {
        free_subband_tables(r);
        return rc;
    }
    r.sub_G = G;
    r.sub_K = K;
    r.sub_n = n_sub;
    r.sub_nq = n_q;
    r.sub_d1max = d1max;
    r.sub_d2max = d2max;
    r.sub_pv = pv;
    r.sub_pCC = pCC;
    r.sub_pLw = h1.Lw;
    r.sub_pstages = static_cast<int32_t>(stages.size());
    r.sub_bv = bv;
    r.sub_bCC = bCC;
    r.sub_bLw = h2.Lw;
    return FDD_OK;
}

cudaError_t launch_range_subband(const fdd_plan* p, const RangeState& r, const fdd::DedispArgs& a, uint8_t* scratch,
                                 size_t scratch_bytes, cudaStream_t s, int64_t* launches) {
    const int64_t n1 = static_cast<int64_t>(a.n_out) + r.sub_d2max;
    const int64_t Np = sub_np(n1);
    if (static_cast<size_t>(p->n_tab) * r.sub_n * r.sub_nq * Np * 2 > scratch_bytes) return cudaErrorInvalidValue;
    fdd::SbfPartArgs pa{};
    pa.in = a.in;
    pa.pitch_bytes = a.pitch_bytes;
    pa.n_valid = a.n_valid;
    pa.base = r.d_sub_pbase;
    pa.off = r.d_sub_poff;
    pa.stages = r.d_sub_pstages;
    pa.segs = r.d_sub_psegs;
    pa.P = reinterpret_cast<uint16_t*>(scratch);
    pa.seg_stride = static_cast<int64_t>(r.sub_nq) * Np;
    pa.tab_stride = static_cast<int64_t>(r.sub_n) * r.sub_nq * Np;
    pa.Np = static_cast<int32_t>(Np);
    pa.n_chan = p->n_chan;
    pa.n_dm = r.sub_nq;
    pa.n_out = static_cast<int32_t>(n1);
    pa.Lw = r.sub_pLw;
    pa.CC = r.sub_pCC;
    pa.n_stages = r.sub_pstages;
    pa.i0 = 0;
    pa.n_slab = r.sub_nq;
    cudaError_t e = fdd::launch_sbf_part(r.sub_pv, pa, p->n_tab, s);
    if (e != cudaSuccess) return e;
    const fdd::DedispVariant& bv = fdd::dedisp_variant(r.sub_bv);
    fdd::DedispArgs b = a;
    b.in = scratch;
    b.pitch_bytes = static_cast<int64_t>(r.sub_nq) * Np * 2;
    b.n_valid = n1;
    b.sb_map = r.d_sub_sbmap;
    b.base = r.d_sub_bbase;
    b.off = r.d_sub_boff;
    b.n_chan = r.sub_n;
    b.Lw = r.sub_bLw;
    b.CC = r.sub_bCC;
    b.blk_per_coarse = r.sub_K / bv.bd();
    b.coarse_stride = Np * 2;
    if ((e = fdd::launch_dedisp(r.sub_bv, b, s)) != cudaSuccess) return e;
    if (launches) *launches += 2;
    return cudaSuccess;
}

}  // namespace host
}  // namespace fdd
