// fdd_fact.cu -- host tables of the pattern-factored dedispersion kernel.
//
// Brute-force dedispersion adds, for trial i, channel c's sample at
// t + d[i][c].  Split the channels into groups of G consecutive channels and
// write d[i][c] = ref_i,g + rel_i,g,c with ref_i,g the smallest delay of the
// group.  Every trial whose relative delays rel_i,g,* are equal ("pattern")
// adds the same group partial sum R_p(tau) = sum_{c in g} X_c(tau + rel_c),
// only shifted by ref_i,g.  Within a block of consecutive trials a group has
// few distinct patterns (about 4 for G = 4 and 10 for G = 8 over 64 trials on
// the ARTS band), so the kernel builds each pattern's partial sums once per
// block in shared memory and every trial reads one 16-bit partial per group
// instead of G bytes.  The sums are the same integers in another order: the
// result is bit-identical to brute force.
//
// For a range, kernel variant and channel-stage size this file computes:
//   base  [n_blk][n_chan]        first staged sample of each channel's raw row
//   goff  [n_blk][n_groups][BD]  shared-memory byte offset of trial jj's pattern
//                                row word for group g (copy = offset parity)
//   pdesc per (block, stage) the list of pattern rows to build:
//         {dst copy 0, dst copy 1, units of 4 samples, src byte address per
//         channel (any alignment)}
//   pd_idx [n_blk][n_stages][2]  (first descriptor, count)
// and the raw row length Lw and the pattern region size of the layout.
// Shared memory, from a 128-byte-aligned base: [zero row | 2 raw buffers x
// CC slots (one unshifted row each, TMA destinations, 128-byte aligned) |
// PB x pattern rows | (PB + 1) x stage offsets | PB x stage descriptors |
// 2 mbarriers]; stage s builds from raw buffer s & 1.  With PB = 2 stage s's
// pattern rows live in pattern buffer s & 1 (its descriptors' destinations
// and its trials' offsets carry that buffer's address), so the kernel can
// build stage s + 1 while it accumulates stage s.
#include <algorithm>
#include <map>
#include <vector>

#include "fdd_plan_impl.h"

using namespace fdd::host;

namespace fdd {
namespace host {

FactTables build_fact_tables(const fdd_plan* p, const RangeState& r, const FactVariant& v, int CC,
                             bool consecutive_rows) {
    FactTables ft;
    const int G = v.G, BD = v.bd(), T = v.tile();
    const int E = r.D == 1 ? 1 : 2;  // bytes per staged sample
    const int n_chan = p->n_chan;
    const int n_blk = (r.n_dm + BD - 1) / BD;
    const int n_groups = (n_chan + G - 1) / G;
    const int n_stages = (n_chan + CC - 1) / CC;
    const int gps = CC / G;
    ft.n_groups = n_groups;
    ft.n_stages = n_stages;
    ft.desc_ints = v.desc_ints();
    ft.base.assign(static_cast<size_t>(n_blk) * n_chan, 0);
    ft.goff.assign(static_cast<size_t>(n_blk) * n_groups * BD, 0);
    ft.pd_idx.assign(static_cast<size_t>(n_blk) * n_stages * 2, 0);
    auto D = [&](int i, int c) { return r.delay[static_cast<size_t>(i) * n_chan + c]; };

    // raw row starts (aligned to 16 samples) and the largest staged span
    int64_t max_need = 0;  // bytes of a staged row that some read touches
    for (int b = 0; b < n_blk; b++) {
        const int ia = b * BD, ib = std::min(r.n_dm, (b + 1) * BD);
        for (int c = 0; c < n_chan; c++) {
            int32_t lo = D(ia, c);
            for (int i = ia; i < ib; i++) lo = std::min(lo, D(i, c));
            ft.base[static_cast<size_t>(b) * n_chan + c] = lo / 16 * 16;
        }
    }
    // patterns per (block, group), pattern rows per (block, stage)
    struct Pat {
        std::vector<int32_t> rel;
        int32_t rmin = 0, rmax = 0;
    };
    int64_t pat_region = 0;
    double adds_fact = 0, adds_brute = 0;  // per time tile
    std::vector<int32_t> trial_pat(BD), trial_ref(BD);
    for (int b = 0; b < n_blk; b++) {
        const int ia = b * BD, ib = std::min(r.n_dm, (b + 1) * BD);
        for (int s = 0; s < n_stages; s++) {
            int64_t cursor = 0;  // bytes of pattern rows of this (block, stage)
            const int first_desc = static_cast<int>(ft.pdesc.size() / ft.desc_ints);
            for (int gl = 0; gl < gps; gl++) {
                const int g = s * gps + gl;
                if (g >= n_groups) break;
                const int c0 = g * G;
                const int gn = std::min(G, n_chan - c0);
                std::map<std::vector<int32_t>, int> index;
                std::vector<Pat> pats;
                for (int jj = 0; jj < BD; jj++) {
                    const int i = std::min(ia + jj, r.n_dm - 1);  // padding trials repeat the last one
                    int32_t ref = D(i, c0);
                    for (int k = 1; k < gn; k++) ref = std::min(ref, D(i, c0 + k));
                    std::vector<int32_t> rel(gn);
                    for (int k = 0; k < gn; k++) rel[k] = D(i, c0 + k) - ref;
                    auto it = index.find(rel);
                    int pi;
                    if (it == index.end()) {
                        pi = static_cast<int>(pats.size());
                        index.emplace(rel, pi);
                        Pat pt;
                        pt.rel = rel;
                        pt.rmin = pt.rmax = ref;
                        pats.push_back(pt);
                    } else {
                        pi = it->second;
                        pats[pi].rmin = std::min(pats[pi].rmin, ref);
                        pats[pi].rmax = std::max(pats[pi].rmax, ref);
                    }
                    trial_pat[jj] = pi;
                    trial_ref[jj] = ref;
                }
                (void)ib;
                std::vector<int32_t> dst0(pats.size()), dst1(pats.size());
                for (size_t pi = 0; pi < pats.size(); pi++) {
                    const Pat& pt = pats[pi];
                    const int32_t span = pt.rmax - pt.rmin;
                    const int32_t nw4 = (span + T) / 4 + 2;  // units of 4 samples built
                    const int32_t lpw = 2 * nw4;             // 32-bit words per copy
                    dst0[pi] = static_cast<int32_t>(cursor);
                    dst1[pi] = static_cast<int32_t>(cursor + 4LL * lpw);
                    cursor += 8LL * lpw;
                    std::vector<int32_t> d(ft.desc_ints, 0);
                    d[0] = dst0[pi];  // relative to the pattern region; made absolute below
                    d[1] = dst1[pi];
                    d[2] = nw4;
                    for (int k = 0; k < G; k++) {
                        if (k < gn) {
                            const int c = c0 + k;
                            // byte of the pattern's first sample in the channel's staged row
                            const int32_t o = E * (pt.rmin + pt.rel[k] - ft.base[static_cast<size_t>(b) * n_chan + c]);
                            // raw buffer (s & 1), channel slot cc, byte o of the row; slot bases added below
                            d[3 + k] = ((s & 1) << 30) | ((c - s * CC) << 20) | o;
                            max_need = std::max<int64_t>(max_need, static_cast<int64_t>(o) + 4LL * E * nw4 + 4);
                        } else {
                            d[3 + k] = -1;  // missing channel: the zero row
                        }
                    }
                    ft.pdesc.insert(ft.pdesc.end(), d.begin(), d.end());
                }
                const int valid = std::min(BD, r.n_dm - ia);
                adds_brute += static_cast<double>(valid) * gn * T;
                adds_fact += static_cast<double>(valid) * T;  // one pattern partial per trial and sample
                for (const Pat& pt : pats) adds_fact += static_cast<double>((pt.rmax - pt.rmin) + T) * (gn - 1);
                for (int jj = 0; jj < BD; jj++) {
                    const int pi = trial_pat[jj];
                    const int32_t o = trial_ref[jj] - pats[pi].rmin;
                    const int32_t dst = (o & 1) ? dst1[pi] : dst0[pi];
                    ft.goff[(static_cast<size_t>(b) * n_groups + g) * BD + jj] = dst + 4 * (o >> 1);
                }
            }
            const int n_desc = static_cast<int>(ft.pdesc.size() / ft.desc_ints) - first_desc;
            ft.max_desc = std::max(ft.max_desc, n_desc);
            ft.pd_idx[(static_cast<size_t>(b) * n_stages + s) * 2] = first_desc;
            ft.pd_idx[(static_cast<size_t>(b) * n_stages + s) * 2 + 1] = n_desc;
            pat_region = std::max(pat_region, cursor);
        }
    }
    ft.work_ratio = adds_brute > 0 ? adds_fact / adds_brute : 1.0;
    // raw row words: every staged read (brute-force span and pattern builds)
    const int64_t need_words = (max_need + 3) / 4;
    int64_t Lw = static_cast<int64_t>(align_up(static_cast<size_t>(need_words + 1), 4));
    if (Lw <= kFactMaxLw)
        Lw = static_cast<int64_t>(align_up(static_cast<size_t>(Lw), fdd::fact_lw_align(static_cast<int>(Lw))));
    if (Lw > kFactMaxLw || pat_region > (1 << 20)) {
        ft.Lw = -1;
        return ft;
    }
    ft.Lw = static_cast<int32_t>(Lw);
    ft.pat_bytes = static_cast<int32_t>(align_up(static_cast<size_t>(pat_region), 16));
    ft.pat_bufs = v.PB;
    // channel boxes: R = 8 (else 4) consecutive channels per TMA copy, when their rows are consecutive
    // in the tensor and a box row (the row plus the spread of the R starts) stays within one TMA box of
    // 256 words; the wider R that fits wins (fewer copies per stage)
    int kBoxRows = 1;
    int n_boxes = n_chan;
    std::vector<int32_t> bb;
    int64_t rb_box = 0;
    for (int R : {8, 4}) {
        if (!consecutive_rows || fdd::fact_boxes(static_cast<int>(Lw)) != 1 || CC % R != 0) continue;
        const int nbx = (n_chan + R - 1) / R;
        std::vector<int32_t> bbr(static_cast<size_t>(n_blk) * nbx);
        int64_t spread = 0;  // words
        for (int b = 0; b < n_blk; b++)
            for (int k = 0; k < nbx; k++) {
                int32_t lo = ft.base[static_cast<size_t>(b) * n_chan + k * R];
                for (int c = k * R; c < std::min(n_chan, (k + 1) * R); c++)
                    lo = std::min(lo, ft.base[static_cast<size_t>(b) * n_chan + c]);
                bbr[static_cast<size_t>(b) * nbx + k] = lo;
                for (int c = k * R; c < std::min(n_chan, (k + 1) * R); c++)
                    spread = std::max<int64_t>(
                        spread, (static_cast<int64_t>(ft.base[static_cast<size_t>(b) * n_chan + c]) - lo) * E / 4);
            }
        const int64_t rbr = static_cast<int64_t>(align_up(static_cast<size_t>(4 * (Lw + spread)), 128));
        if (rbr / 4 > 256) continue;
        kBoxRows = R;
        n_boxes = nbx;
        bb.swap(bbr);
        rb_box = rbr;
        break;
    }
    const bool boxes = kBoxRows > 1;
    ft.box_rows = kBoxRows;
    if (boxes) ft.bbase.swap(bb);
    // resolve shared-memory addresses
    ft.zero_off = 0;
    ft.rb = boxes ? static_cast<int32_t>(rb_box) : static_cast<int32_t>(align_up(static_cast<size_t>(4 * Lw), 128));
    ft.raw_off = static_cast<int32_t>(align_up(static_cast<size_t>(4 * Lw + 16), 128));
    ft.pat_off = ft.raw_off + 2 * CC * ft.rb;
    if (v.PB == 2) {
        // stage s's rows in pattern buffer s & 1
        for (int b = 0; b < n_blk; b++)
            for (int s = 0; s < n_stages; s++) {
                const int32_t shift = (s & 1) * ft.pat_bytes;
                const size_t k = (static_cast<size_t>(b) * n_stages + s) * 2;
                for (int d = ft.pd_idx[k]; d < ft.pd_idx[k] + ft.pd_idx[k + 1]; d++) {
                    ft.pdesc[static_cast<size_t>(d) * ft.desc_ints] += shift;
                    ft.pdesc[static_cast<size_t>(d) * ft.desc_ints + 1] += shift;
                }
                for (int gl = 0; gl < gps && s * gps + gl < n_groups; gl++)
                    for (int jj = 0; jj < BD; jj++)
                        ft.goff[(static_cast<size_t>(b) * n_groups + s * gps + gl) * BD + jj] += shift;
            }
    }
    // DM block and stage of every descriptor (for the channel-box shifts)
    std::vector<int32_t> desc_blk, desc_stage;
    if (boxes) {
        desc_blk.assign(ft.pdesc.size() / ft.desc_ints, 0);
        desc_stage.assign(ft.pdesc.size() / ft.desc_ints, 0);
        for (int b = 0; b < n_blk; b++)
            for (int s = 0; s < n_stages; s++) {
                const size_t k = (static_cast<size_t>(b) * n_stages + s) * 2;
                for (int d = ft.pd_idx[k]; d < ft.pd_idx[k] + ft.pd_idx[k + 1]; d++) {
                    desc_blk[d] = b;
                    desc_stage[d] = s;
                }
            }
    }
    for (size_t di = 0; di < ft.pdesc.size(); di += ft.desc_ints) {
        ft.pdesc[di] += ft.pat_off;
        ft.pdesc[di + 1] += ft.pat_off;
        for (int k = 0; k < G; k++) {
            int32_t& e = ft.pdesc[di + 3 + k];
            if (e < 0) {
                e = ft.zero_off;  // zero row
            } else {
                const int32_t par = e >> 30, cc = (e >> 20) & 1023, o = e & ((1 << 20) - 1);
                e = ft.raw_off + (par * CC + cc) * ft.rb + o;
                if (boxes) {  // the channel's row sits after the gap between its box's start and its own
                    const int b = desc_blk[di / ft.desc_ints];
                    const int c = desc_stage[di / ft.desc_ints] * CC + cc;
                    e += (ft.base[static_cast<size_t>(b) * n_chan + c] -
                          ft.bbase[static_cast<size_t>(b) * n_boxes + c / kBoxRows]) * E;
                }
            }
        }
    }
    for (int32_t& g : ft.goff) g += ft.pat_off;
    ft.desc_bytes = ft.max_desc * ft.desc_ints * 4;
    ft.bar_off = ft.pat_off + v.PB * ft.pat_bytes + (v.PB + 1) * gps * BD * 4 + v.PB * ft.desc_bytes;
    // + 16 bytes of mbarriers, + 128 for aligning the dynamic shared-memory base
    ft.smem_bytes = static_cast<size_t>(ft.bar_off) + 16 + 128;
    return ft;
}

}  // namespace host
}  // namespace fdd
