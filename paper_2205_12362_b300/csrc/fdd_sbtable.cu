// fdd_sbtable.cu -- synthesized-beam (SB) table from the array geometry
// (appendix "Tied-array beam simulations", "Synthesized Beams").
//
// The grating responses of the tied-array beams (TABs) move with 1/f, so an
// SB at a fixed position in the compound beam takes, band by band, the TAB
// whose grating response covers that position.  SB index n_SB (0 = centre) at
// the highest frequency f_max takes TAB n_TAB of grating response n_gr:
//     n_TAB = n_SB mod N, less N when above N/2 - 1;   n_gr = (n_SB - n_TAB) / N.
// Going down in frequency, TAB k_j = n_TAB - j sgn(n_SB) of the same grating
// response reaches the SB's position at
//     f_j = f_max (n_gr B_max + k_j alpha B_cq) / (n_gr B_max + n_TAB alpha B_cq),
// and the SB switches from k_j to k_{j+1} at 0.75 f_j + 0.25 f_{j+1} for even SB
// indices and 0.25 f_j + 0.75 f_{j+1} for odd ones (the appendix's weights for
// SBs half a beam width apart, applied between consecutive optimal
// frequencies).  A TAB index past N/2 - 1 or below -N/2 is the TAB N away on
// the next grating response.  Table rows are n_TAB + N/2.
#include <cmath>
#include <vector>

#include "fdd_plan_impl.h"

using namespace fdd::host;

namespace {

int tab_row(long long k, int N) {
    while (k > N / 2 - 1) k -= N;
    while (k < -(N / 2)) k += N;
    return static_cast<int>(k + N / 2);
}

}  // namespace

extern "C" int fdd_sb_table(int32_t n_tab, int32_t n_sb, int32_t n_chan, const double* chan_freq_mhz,
                            double f_max_mhz, double alpha, double b_max_m, double b_cq_m,
                            int32_t chan_per_subband, int16_t* sb_map_out) {
    if (n_tab < 2 || n_tab % 2 || n_tab > FDD_MAX_TABS || n_sb < 1 || n_chan < 1 || n_chan > FDD_MAX_CHANNELS ||
        !chan_freq_mhz || !sb_map_out || !(f_max_mhz > 0) || !(alpha > 0) || !(b_max_m > 0) || !(b_cq_m > 0) ||
        chan_per_subband < 1)
        return fail(FDD_ERR_INVALID_ARG, "bad SB table argument (the index convention needs an even TAB count)");
    const int N = n_tab;
    for (int s = 0; s < n_sb; s++) {
        const long long nsb = static_cast<long long>(s) - n_sb / 2;
        long long nt = ((nsb % N) + N) % N;
        if (nt > N / 2 - 1) nt -= N;
        const long long ngr = (nsb - nt) / N;
        const int sgn = (nsb > 0) - (nsb < 0);
        const bool even = (std::llabs(nsb) % 2) == 0;
        const double w_hi = even ? 0.75 : 0.25, w_lo = 1.0 - w_hi;
        const double den = static_cast<double>(ngr) * b_max_m + static_cast<double>(nt) * alpha * b_cq_m;
        auto f_opt = [&](long long j) {
            return f_max_mhz * (static_cast<double>(ngr) * b_max_m + static_cast<double>(nt - j * sgn) * alpha * b_cq_m) /
                   den;
        };
        for (int b0 = 0; b0 < n_chan; b0 += chan_per_subband) {
            const int b1 = std::min(n_chan, b0 + chan_per_subband);
            double f = 0;
            for (int c = b0; c < b1; c++) f += chan_freq_mhz[c];
            f /= (b1 - b0);
            long long j = 0;
            if (sgn != 0)
                while (j <= 4LL * N + 64 && f < w_hi * f_opt(j) + w_lo * f_opt(j + 1)) j++;
            const int16_t row = static_cast<int16_t>(tab_row(nt - j * sgn, N));
            for (int c = b0; c < b1; c++) sb_map_out[static_cast<int64_t>(s) * n_chan + c] = row;
        }
    }
    return FDD_OK;
}
