/*
 * oracle.c -- plain CPU reference of the ARTS single-pulse search hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle: tests, the
 * package smoke check and the benchmark's CPU-baseline leg may call it; the
 * product path never does.  It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * Everything is written as the definitions of the paper's AMBER stages
 * (Sec. "AMBER": downsampling, dedispersion, integration, S/N evaluation,
 * candidate selection), in the simplest loops that compute them:
 *   - delays in FP64 from the cold-plasma dispersion law, rounded half away
 *     from zero (llround), in units of D * t_samp;
 *   - downsampling = exact integer sum of D consecutive samples;
 *   - brute-force dedispersion with synthesized-beam gather, exact int64 sums;
 *   - per-series mean / population standard deviation, two-pass FP64;
 *   - sliding boxcar of width w (exact int64 sum), S/N = (B - w mu)/(sigma sqrt w);
 *   - candidate when S/N strictly exceeds the threshold ("exceeds", Sec.
 *     "Candidate selection"); one candidate per (SB, DM, width, time), no
 *     clustering.
 * Where the paper is silent (constant, rounding, statistics, boxcar form)
 * the reading taken is stated at the function that applies it.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (see build.py).
 * -ffp-contract=off keeps every FP64 expression in the written order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Dispersion constant in s MHz^2 / (pc cm^-3).  The paper quotes no value;
 * this is the standard cold-plasma constant 1/(2.41e-4). */
#define ORACLE_KDM 4148.808

void oracle_set_threads(int32_t n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int32_t oracle_get_threads(void) {
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/* Sec. "Dedispersion" (brute-force incoherent dedispersion): channel c of
 * trial DM_i is delayed, relative to the highest channel, by
 *     K_DM * DM_i * (f_c^-2 - f_top^-2) / (D * t_samp)   samples,
 * rounded half away from zero.  DM_i = dm0 + i * ddm is formed afresh for
 * each i.  Returns the largest delay; *n_near_tie counts real-valued delays
 * whose fractional part lies within 1e-9 of one half (rounding there is
 * sensitive to the last bit of the FP64 evaluation). */
int64_t oracle_delays(int32_t n_chan, const double* freq_mhz, double t_samp_s,
                      double dm0, double ddm, int32_t n_dm, int32_t downsamp,
                      int64_t* out, int64_t* n_near_tie) {
    double f_top = freq_mhz[0];
    for (int32_t c = 1; c < n_chan; c++)
        if (freq_mhz[c] > f_top) f_top = freq_mhz[c];
    int64_t dmax = 0, ties = 0;
    for (int32_t i = 0; i < n_dm; i++) {
        double dm = dm0 + (double)i * ddm;
        for (int32_t c = 0; c < n_chan; c++) {
            double f = freq_mhz[c];
            double x = ((ORACLE_KDM * dm) * (1.0 / (f * f) - 1.0 / (f_top * f_top)))
                       / ((double)downsamp * t_samp_s);
            double frac = x - floor(x);
            if (fabs(frac - 0.5) < 1e-9) ties++;
            int64_t d = (int64_t)llround(x);
            out[(int64_t)i * n_chan + c] = d;
            if (d > dmax) dmax = d;
        }
    }
    if (n_near_tie) *n_near_tie = ties;
    return dmax;
}

/* Sec. "Downsampling": y[r][j] = sum_{k<D} x[r][j*D + k], j < floor(n_in/D). */
void oracle_downsample(const uint8_t* x, int64_t rows, int64_t n_in, int64_t pitch,
                       int32_t downsamp, uint32_t* y) {
    int64_t n_y = n_in / downsamp;
    for (int64_t r = 0; r < rows; r++)
        for (int64_t j = 0; j < n_y; j++) {
            uint32_t s = 0;
            for (int32_t k = 0; k < downsamp; k++) s += x[r * pitch + j * downsamp + k];
            y[r * n_y + j] = s;
        }
}

/* Sec. "Dedispersion" with the synthesized-beam formation of Sec.
 * "Hierarchical beam forming": SB s takes channel c from TAB sb_map[s][c];
 *     S[s][i][t] = sum_c y[sb_map[s][c]][c][t + d[i][c]],  t < n_out.
 * One series, plain loops, exact int64. */
static void dedisperse_one(const uint32_t* y, int32_t n_chan, int64_t n_y,
                           const int32_t* sb_row, const int64_t* d_row, int64_t n_out,
                           int64_t* acc) {
    for (int64_t t = 0; t < n_out; t++) acc[t] = 0;
    for (int32_t c = 0; c < n_chan; c++) {
        const uint32_t* row = y + ((int64_t)sb_row[c] * n_chan + c) * n_y;
        int64_t off = d_row[c];
        for (int64_t t = 0; t < n_out; t++) acc[t] += (int64_t)row[t + off];
    }
}

/* Full dedispersion for all (SB, DM) pairs; the caller guarantees
 * n_out + max delay <= n_y. */
void oracle_dedisperse(const uint32_t* y, int32_t n_tab, int32_t n_chan, int64_t n_y,
                       const int32_t* sb_map, int32_t n_sb, const int64_t* delays,
                       int32_t n_dm, int64_t n_out, int64_t* series) {
    (void)n_tab;
    int64_t n_series = (int64_t)n_sb * n_dm;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < n_series; q++) {
        int32_t s = (int32_t)(q / n_dm), i = (int32_t)(q % n_dm);
        dedisperse_one(y, n_chan, n_y, sb_map + (int64_t)s * n_chan,
                       delays + (int64_t)i * n_chan, n_out, series + q * n_out);
    }
}

/* Sec. "S/N evaluation" (method left open by the paper): mean and population
 * standard deviation of the series over its own n samples, two-pass FP64. */
void oracle_stats(const int64_t* s, int64_t n, double* mean, double* std) {
    int64_t sum = 0;
    for (int64_t t = 0; t < n; t++) sum += s[t];
    double mu = (double)sum / (double)n;
    double ss = 0.0;
    for (int64_t t = 0; t < n; t++) {
        double d = (double)s[t] - mu;
        ss += d * d;
    }
    *mean = mu;
    *std = sqrt(ss / (double)n);
}

/* Sec. "Integration" + "S/N evaluation": sliding boxcar of width w,
 * B(t) = sum_{k<w} s[t+k] for t in [0, n-w], and
 * snr(t) = (B(t) - w*mean) / (std * sqrt(w)).  Writes n-w+1 values. */
void oracle_boxcar_snr(const int64_t* s, int64_t n, int32_t w, double mean, double std,
                       double* snr) {
    double norm = std * sqrt((double)w);
    for (int64_t t = 0; t + w <= n; t++) {
        int64_t b = 0;
        for (int32_t k = 0; k < w; k++) b += s[t + k];
        snr[t] = ((double)b - (double)w * mean) / norm;
    }
}

/* Two-step subband dedispersion (Sec. "AMBER", "Dedispersion": besides a
 * single step, the module dedisperses "using a more efficient two step
 * process including subbanding"; Table "dedispersion setup": 32 subbands and
 * a subbanding DM step 32x the fine step).  An approximation of brute force,
 * written in the paper's order:
 *   step 1, per subband b and coarse DM block q, the subband's channels are
 *     aligned to the subband's own reference frequency at the block's coarse
 *     DM:  P[tab][b][q][u] = sum_{c in b} y[tab][c][u + d1[q][c]];
 *   step 2, per fine trial i of block q, the subbands are aligned at the fine
 *     DM:  S[s][i][t] = sum_b P[tab(s,b)][b][q][t + d2[i][b]].
 * Readings (the paper gives only the sizes): subband b = channels
 * [b*G, (b+1)*G) (the last may be shorter); its reference f_b is its highest
 * channel frequency; fine trial i belongs to block q = i / K whose DM is the
 * block's midpoint DMc_q = dm0 + (q*K + (K-1)/2) * ddm;
 *   d1[q][c] = llround(kDM*DMc_q*(1/f_c^2 - 1/f_b^2) / (D t)),
 *   d2[i][b] = llround(kDM*DM_i*(1/f_b^2 - 1/f_top^2) / (D t)),
 * in the same FP64 expression order as oracle_delays; the SB takes, for the
 * whole subband, the TAB of the subband's first channel (tab(s,b)).
 * n1 = n_out + max d2 samples of P are formed per (tab, b, q).  series gets
 * n_sb*n_dm rows of n_out; returns -1 if n_y is too short, -2 on allocation
 * failure, else the largest d1 + d2. */
int64_t oracle_dedisperse_two_step(const uint32_t* y, int32_t n_tab, int32_t n_chan, int64_t n_y,
                                   const double* freq_mhz, double t_samp_s, int32_t downsamp,
                                   double dm0, double ddm, int32_t n_dm, int32_t G, int32_t K,
                                   const int32_t* sb_map, int32_t n_sb, int64_t n_out, int64_t* series) {
    const int32_t n_sub = (n_chan + G - 1) / G;
    const int32_t n_q = (n_dm + K - 1) / K;
    double f_top = freq_mhz[0];
    for (int32_t c = 1; c < n_chan; c++)
        if (freq_mhz[c] > f_top) f_top = freq_mhz[c];
    double* f_ref = (double*)malloc(sizeof(double) * (size_t)n_sub);
    int64_t* d1 = (int64_t*)malloc(sizeof(int64_t) * (size_t)n_q * (size_t)n_chan);
    int64_t* d2 = (int64_t*)malloc(sizeof(int64_t) * (size_t)n_dm * (size_t)n_sub);
    if (!f_ref || !d1 || !d2) { free(f_ref); free(d1); free(d2); return -2; }
    for (int32_t b = 0; b < n_sub; b++) {
        f_ref[b] = freq_mhz[b * G];
        for (int32_t c = b * G; c < n_chan && c < (b + 1) * G; c++)
            if (freq_mhz[c] > f_ref[b]) f_ref[b] = freq_mhz[c];
    }
    const double tD = (double)downsamp * t_samp_s;
    int64_t d1max = 0, d2max = 0, dsum = 0;
    for (int32_t q = 0; q < n_q; q++) {
        const double dmc = dm0 + ((double)q * K + 0.5 * (double)(K - 1)) * ddm;
        for (int32_t c = 0; c < n_chan; c++) {
            const double f = freq_mhz[c], fb = f_ref[c / G];
            const int64_t d = (int64_t)llround(((ORACLE_KDM * dmc) * (1.0 / (f * f) - 1.0 / (fb * fb))) / tD);
            d1[(int64_t)q * n_chan + c] = d;
            if (d > d1max) d1max = d;
        }
    }
    for (int32_t i = 0; i < n_dm; i++) {
        const double dm = dm0 + (double)i * ddm;
        for (int32_t b = 0; b < n_sub; b++) {
            const double fb = f_ref[b];
            const int64_t d = (int64_t)llround(((ORACLE_KDM * dm) * (1.0 / (fb * fb) - 1.0 / (f_top * f_top))) / tD);
            d2[(int64_t)i * n_sub + b] = d;
            if (d > d2max) d2max = d;
        }
    }
    for (int32_t i = 0; i < n_dm; i++)
        for (int32_t c = 0; c < n_chan; c++) {
            const int64_t v = d1[(int64_t)(i / K) * n_chan + c] + d2[(int64_t)i * n_sub + c / G];
            if (v > dsum) dsum = v;
        }
    const int64_t n1 = n_out + d2max;
    if (n1 + d1max > n_y || n_out + dsum > n_y) { free(f_ref); free(d1); free(d2); return -1; }
    int64_t* P = (int64_t*)malloc(sizeof(int64_t) * (size_t)n_tab * (size_t)n_sub * (size_t)(n1 > 0 ? n1 : 1));
    if (!P) { free(f_ref); free(d1); free(d2); return -2; }
    for (int32_t q = 0; q < n_q; q++) {
        /* step 1 for block q */
#pragma omp parallel for schedule(static)
        for (int64_t tb = 0; tb < (int64_t)n_tab * n_sub; tb++) {
            const int32_t tab = (int32_t)(tb / n_sub), b = (int32_t)(tb % n_sub);
            int64_t* prow = P + tb * n1;
            for (int64_t u = 0; u < n1; u++) prow[u] = 0;
            for (int32_t c = b * G; c < n_chan && c < (b + 1) * G; c++) {
                const uint32_t* row = y + ((int64_t)tab * n_chan + c) * n_y;
                const int64_t off = d1[(int64_t)q * n_chan + c];
                for (int64_t u = 0; u < n1; u++) prow[u] += (int64_t)row[u + off];
            }
        }
        /* step 2 for the fine trials of block q */
        const int32_t i_end = (q + 1) * K < n_dm ? (q + 1) * K : n_dm;
#pragma omp parallel for schedule(static)
        for (int64_t si = 0; si < (int64_t)n_sb * (i_end - q * K); si++) {
            const int32_t s = (int32_t)(si / (i_end - q * K)), i = q * K + (int32_t)(si % (i_end - q * K));
            int64_t* acc = series + ((int64_t)s * n_dm + i) * n_out;
            for (int64_t t = 0; t < n_out; t++) acc[t] = 0;
            for (int32_t b = 0; b < n_sub; b++) {
                const int32_t tab = sb_map[(int64_t)s * n_chan + b * G];
                const int64_t* prow = P + ((int64_t)tab * n_sub + b) * n1;
                const int64_t off = d2[(int64_t)i * n_sub + b];
                for (int64_t t = 0; t < n_out; t++) acc[t] += prow[t + off];
            }
        }
    }
    free(P);
    free(f_ref);
    free(d1);
    free(d2);
    return dsum;
}

typedef struct {
    int32_t sb, dm_index, downsamp, width_native;
    int64_t t_native;
    double dm, snr;
} oracle_cand; /* 40 bytes */

/* The whole hot path for one chunk: for every range r of the DM plan,
 * downsample by D_r, dedisperse every (SB, DM) pair, compute the series
 * statistics, run every boxcar width and keep (Sec. "Candidate selection")
 * each (sb, dm, width, t) whose S/N strictly exceeds thr.  Widths are in
 * range samples; a candidate reports width * D_r and t * D_r + t_offset in
 * native samples.  dm_index is global over the concatenated ranges.
 * Series with zero standard deviation emit nothing.
 * series_or_null, if given, receives int64 series per range, packed
 * [range][sb][dm][n_r] (n_r below).  Returns the total candidate count;
 * only the first cap are stored (order unspecified).  Returns -1 on a short
 * input and -2 on allocation failure.
 * Downsampling bins (Sec. "Downsampling"):
 *   bins_absolute == 0: bins start at input sample 0; n_r = floor(n_out/D_r);
 *     the input must hold D_r * (n_r + max delay_r) samples;
 *   bins_absolute != 0: input sample 0 is sample t_offset_native (>= 0) of
 *     the beam's stream and bins are aligned to stream sample 0 (bin J covers
 *     stream samples [J D, J D + D)), so consecutive windows of one stream
 *     tile the one-shot search of the whole stream.  The window searches the
 *     bins that start in [t_offset, t_offset + n_out): J from ceil(t_offset/D)
 *     to ceil((t_offset + n_out)/D) - 1, i.e. n_r of them, read from input
 *     sample phase_r = ceil(t_offset/D) D - t_offset on; a candidate's
 *     t_native is its bin's first stream sample.  The input must hold
 *     phase_r + D_r (n_r + max delay_r) samples. */
int64_t oracle_search(const uint8_t* x, int32_t n_tab, int32_t n_chan, int64_t n_in,
                      int64_t pitch, const int32_t* sb_map, int32_t n_sb,
                      const double* freq_mhz, double t_samp_s, int32_t n_range,
                      const double* dm0, const double* ddm, const int32_t* n_dm,
                      const int32_t* downsamp, const int32_t* n_width,
                      const int32_t* widths, double thr, int64_t n_out,
                      int64_t t_offset_native, oracle_cand* cands, int64_t cap,
                      int64_t* series_or_null, const int32_t* sub_chan, const int32_t* sub_k,
                      int32_t bins_absolute) {
    int64_t count = 0;
    if (bins_absolute && t_offset_native < 0) return -1;
    int32_t dm_base = 0, w_base = 0;
    int64_t series_base = 0;
    for (int32_t r = 0; r < n_range; r++) {
        int32_t D = downsamp[r];
        int64_t phase = 0, n_r = n_out / D;
        if (bins_absolute) {
            const int64_t j_first = (t_offset_native + D - 1) / D;           /* ceil(t_offset / D) */
            const int64_t j_end = (t_offset_native + n_out + D - 1) / D;     /* ceil((t_offset + n_out) / D) */
            phase = j_first * D - t_offset_native;
            n_r = j_end - j_first;
        }
        const int64_t n_y = (n_in - phase) / D;
        int64_t* d = (int64_t*)malloc(sizeof(int64_t) * (size_t)n_dm[r] * (size_t)n_chan);
        uint32_t* y = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n_tab * (size_t)n_chan * (size_t)n_y);
        if (!d || !y) { free(d); free(y); return -2; }
        int64_t dmax = oracle_delays(n_chan, freq_mhz, t_samp_s, dm0[r], ddm[r], n_dm[r], D, d, NULL);
        const int two_step = sub_chan && sub_k && sub_chan[r] > 0;
        if (!two_step && n_r + dmax > n_y) { free(d); free(y); return -1; }
        oracle_downsample(x + phase, (int64_t)n_tab * n_chan, n_in - phase, pitch, D, y);
        int64_t n_series = (int64_t)n_sb * n_dm[r];
        int64_t* ts = NULL;  /* two-step series of this range */
        if (two_step) {
            ts = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_series > 0 ? n_series : 1) * (size_t)(n_r > 0 ? n_r : 1));
            if (!ts) { free(d); free(y); return -2; }
            const int64_t rc = oracle_dedisperse_two_step(y, n_tab, n_chan, n_y, freq_mhz, t_samp_s, D, dm0[r], ddm[r],
                                                          n_dm[r], sub_chan[r], sub_k[r], sb_map, n_sb, n_r, ts);
            if (rc < 0) { free(ts); free(d); free(y); return rc == -1 ? -1 : -2; }
        }
#pragma omp parallel
        {
            int64_t* acc = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_r > 0 ? n_r : 1));
            double* snr = (double*)malloc(sizeof(double) * (size_t)(n_r > 0 ? n_r : 1));
#pragma omp for schedule(dynamic, 1)
            for (int64_t q = 0; q < n_series; q++) {
                int32_t s = (int32_t)(q / n_dm[r]), i = (int32_t)(q % n_dm[r]);
                if (ts)
                    memcpy(acc, ts + q * n_r, sizeof(int64_t) * (size_t)n_r);
                else
                    dedisperse_one(y, n_chan, n_y, sb_map + (int64_t)s * n_chan,
                                   d + (int64_t)i * n_chan, n_r, acc);
                if (series_or_null)
                    memcpy(series_or_null + series_base + q * n_r, acc, sizeof(int64_t) * (size_t)n_r);
                if (n_r == 0) continue;
                double mu, sd;
                oracle_stats(acc, n_r, &mu, &sd);
                if (!(sd > 0.0)) continue;
                for (int32_t k = 0; k < n_width[r]; k++) {
                    int32_t w = widths[w_base + k];
                    if (w > n_r) continue;
                    oracle_boxcar_snr(acc, n_r, w, mu, sd, snr);
                    for (int64_t t = 0; t + w <= n_r; t++) {
                        if (snr[t] > thr) {
                            int64_t slot;
#pragma omp atomic capture
                            slot = count++;
                            if (slot < cap) {
                                oracle_cand* o = cands + slot;
                                o->sb = s;
                                o->dm_index = dm_base + i;
                                o->downsamp = D;
                                o->width_native = w * D;
                                o->t_native = t * D + phase + t_offset_native;
                                o->dm = dm0[r] + (double)i * ddm[r];
                                o->snr = snr[t];
                            }
                        }
                    }
                }
            }
            free(acc);
            free(snr);
        }
        free(ts);
        free(d);
        free(y);
        dm_base += n_dm[r];
        w_base += n_width[r];
        series_base += n_series * n_r;
    }
    return count;
}

/* ------------------------------------------------------------------------
 * DM-width clustering of a candidate list (Sec. "AMBER", paragraph
 * "Clustering (optional)"), in the two steps the paper gives:
 *   1. among candidates of one SB at the same time and the same DM trial
 *      (different pulse widths) keep the one with the highest S/N;
 *   2. among the survivors of one SB at the same time, a group of
 *      neighbouring DM trials (dm_index k, k+1, k+2, ... with no gap) keeps
 *      only its highest-S/N candidate.
 * Readings (the paper is silent on them): "time" is the window start
 * t_native, compared exactly; clustering is per SB; DM neighbours are
 * consecutive global dm_index values (so a group may cross a DM-range
 * boundary); ties keep the smaller width in step 1, then the earlier record
 * of the input list, and the smaller dm_index in step 2.
 * Writes the kept records to out (in (sb, t, dm) order) and returns how many.
 * Returns -2 on allocation failure. */
static const oracle_cand* g_cl_in; /* qsort context (single-threaded) */

static int cl_cmp(const void* pa, const void* pb) {
    int64_t a = *(const int64_t*)pa, b = *(const int64_t*)pb;
    const oracle_cand *x = g_cl_in + a, *y = g_cl_in + b;
    if (x->sb != y->sb) return x->sb < y->sb ? -1 : 1;
    if (x->t_native != y->t_native) return x->t_native < y->t_native ? -1 : 1;
    if (x->dm_index != y->dm_index) return x->dm_index < y->dm_index ? -1 : 1;
    if (x->width_native != y->width_native) return x->width_native < y->width_native ? -1 : 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

int64_t oracle_cluster(const oracle_cand* in, int64_t n, oracle_cand* out) {
    if (n <= 0) return 0;
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int64_t* keep = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    if (!idx || !keep) { free(idx); free(keep); return -2; }
    for (int64_t k = 0; k < n; k++) idx[k] = k;
    g_cl_in = in;
    qsort(idx, (size_t)n, sizeof(int64_t), cl_cmp);
    /* step 1: one candidate per (sb, t, dm): the highest S/N; the sort order
     * puts smaller widths, then earlier records, first, and only a strictly
     * higher S/N replaces the one kept */
    int64_t m = 0;
    for (int64_t k = 0; k < n; k++) {
        const oracle_cand* c = in + idx[k];
        if (m > 0) {
            const oracle_cand* p = in + keep[m - 1];
            if (p->sb == c->sb && p->t_native == c->t_native && p->dm_index == c->dm_index) {
                if (c->snr > p->snr) keep[m - 1] = idx[k];
                continue;
            }
        }
        keep[m++] = idx[k];
    }
    /* step 2: runs of consecutive dm_index at one (sb, t) keep their highest
     * S/N; scanning in dm order, only a strictly higher S/N replaces */
    int64_t n_out = 0, best = -1, prev = -1;
    for (int64_t k = 0; k < m; k++) {
        const oracle_cand* c = in + keep[k];
        int joins = 0;
        if (prev >= 0) {
            const oracle_cand* p = in + prev;
            joins = p->sb == c->sb && p->t_native == c->t_native && c->dm_index == p->dm_index + 1;
        }
        if (!joins) {
            if (best >= 0) out[n_out++] = in[best];
            best = keep[k];
        } else if (c->snr > in[best].snr) {
            best = keep[k];
        }
        prev = keep[k];
    }
    if (best >= 0) out[n_out++] = in[best];
    free(idx);
    free(keep);
    return n_out;
}

/* ------------------------------------------------------------------------
 * RFI mitigation (Sec. "AMBER", "RFI mitigation (optional)"; Sec. "Fraction of
 * data lost to RFI"): a time-domain filter for bright wide-band low-DM RFI and
 * a frequency-domain filter for bright narrowband RFI, each applied
 * iteratively (three iterations each in ARTS) to ever cleaner samples.  The
 * filters' statistics are not given in the paper; readings:
 *   time domain, per TAB: the zero-DM series z[t] = sum_c x[c][t]; each
 *     iteration takes the mean mu and population std sigma of z over the
 *     unflagged samples and flags every unflagged t with z[t] - mu > thr_t*sigma
 *     (bright = positive excursions); flagged samples of every channel are
 *     replaced by the channel's mean over the unflagged samples, rounded half
 *     up;
 *   frequency domain, per TAB, on the time-cleaned data: the channel sums
 *     b[c] = sum_t x[c][t]; each iteration flags every unflagged channel with
 *     |b[c] - mu| > thr_f*sigma (mu, sigma over unflagged channels; two-sided:
 *     hot or dead channels); flagged channels are filled with the mean level
 *     of the unflagged channels, sum b / (channels * n_in) rounded half up.
 * Moments are exact integers: S1 < 2^64 and S2 as a 128-bit sum;
 * mu = S1/n and sigma = sqrt((n S2 - S1^2) / n^2), the population standard
 * deviation from its exact integer numerator, formed in FP64 only after the
 * numerator is complete.  Every flag decision compares lhs = z - mu (or
 * |b - mu|) against rhs = thr*sigma; decisions with |lhs - rhs| <= 1e-9 |rhs|
 * are counted in *near (the caller's report that a decision sat on the
 * threshold, where another FP64 evaluation order of the same statistic could
 * decide the other way).  x is modified in place ([n_tab][n_chan][pitch],
 * first n_in samples); tflags [n_tab][n_in] and cflags [n_tab][n_chan] get 1
 * for flagged samples / channels.  A threshold <= 0 disables its filter. */
static void rfi_moments(const uint64_t* v, const uint8_t* flag, int64_t n, int64_t* cnt, double* mu, double* sigma) {
    uint64_t s1 = 0;
    unsigned __int128 s2 = 0;
    int64_t k = 0;
    for (int64_t j = 0; j < n; j++)
        if (!flag[j]) {
            s1 += v[j];
            s2 += (unsigned __int128)v[j] * v[j];
            k++;
        }
    *cnt = k;
    if (k == 0) { *mu = 0; *sigma = 0; return; }
    /* n S2 - S1^2 >= 0 exactly (Cauchy-Schwarz), so no clamp is needed */
    const unsigned __int128 num = (unsigned __int128)k * s2 - (unsigned __int128)s1 * s1;
    *mu = (double)s1 / (double)k;
    *sigma = sqrt((double)num / ((double)k * (double)k));
}

/* lhs > rhs, counting near ties (|lhs - rhs| <= 1e-9 |rhs|) in *near */
static int rfi_exceeds(double lhs, double rhs, int64_t* near) {
    if (fabs(lhs - rhs) <= 1e-9 * fabs(rhs)) (*near)++;
    return lhs > rhs;
}

int64_t oracle_rfi_clean(uint8_t* x, int32_t n_tab, int32_t n_chan, int64_t n_in, int64_t pitch,
                         double time_thr, int32_t time_iters, double freq_thr, int32_t freq_iters,
                         uint8_t* tflags, uint8_t* cflags) {
    int64_t near = 0;
    uint64_t* z = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n_in > 0 ? n_in : 1));
    uint64_t* b = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n_chan);
    for (int32_t tab = 0; tab < n_tab; tab++) {
        uint8_t* xt = x + (int64_t)tab * n_chan * pitch;
        uint8_t* tf = tflags + (int64_t)tab * n_in;
        uint8_t* cf = cflags + (int64_t)tab * n_chan;
        memset(tf, 0, (size_t)n_in);
        memset(cf, 0, (size_t)n_chan);
        if (time_thr > 0) {
            for (int64_t t = 0; t < n_in; t++) {
                uint64_t s = 0;
                for (int32_t c = 0; c < n_chan; c++) s += xt[(int64_t)c * pitch + t];
                z[t] = s;
            }
            for (int32_t it = 0; it < time_iters; it++) {
                int64_t k;
                double mu, sigma;
                rfi_moments(z, tf, n_in, &k, &mu, &sigma);
                if (k == 0) break;
                for (int64_t t = 0; t < n_in; t++)
                    if (!tf[t] && rfi_exceeds((double)z[t] - mu, time_thr * sigma, &near)) tf[t] = 1;
            }
            int64_t n_ok = 0;
            for (int64_t t = 0; t < n_in; t++) n_ok += !tf[t];
            if (n_ok > 0 && n_ok < n_in)
                for (int32_t c = 0; c < n_chan; c++) {
                    uint8_t* row = xt + (int64_t)c * pitch;
                    uint64_t s = 0;
                    for (int64_t t = 0; t < n_in; t++)
                        if (!tf[t]) s += row[t];
                    const uint8_t m = (uint8_t)((2 * s + (uint64_t)n_ok) / (2 * (uint64_t)n_ok));
                    for (int64_t t = 0; t < n_in; t++)
                        if (tf[t]) row[t] = m;
                }
        }
        if (freq_thr > 0) {
            for (int32_t c = 0; c < n_chan; c++) {
                uint64_t s = 0;
                for (int64_t t = 0; t < n_in; t++) s += xt[(int64_t)c * pitch + t];
                b[c] = s;
            }
            for (int32_t it = 0; it < freq_iters; it++) {
                int64_t k;
                double mu, sigma;
                rfi_moments(b, cf, n_chan, &k, &mu, &sigma);
                if (k == 0) break;
                for (int32_t c = 0; c < n_chan; c++)
                    if (!cf[c] && rfi_exceeds(fabs((double)b[c] - mu), freq_thr * sigma, &near)) cf[c] = 1;
            }
            uint64_t s = 0;
            int64_t n_ok = 0;
            for (int32_t c = 0; c < n_chan; c++)
                if (!cf[c]) { s += b[c]; n_ok++; }
            if (n_ok > 0 && n_ok < n_chan && n_in > 0) {
                const uint64_t den = (uint64_t)n_ok * (uint64_t)n_in;
                const uint8_t v = (uint8_t)((2 * s + den) / (2 * den));
                for (int32_t c = 0; c < n_chan; c++)
                    if (cf[c]) memset(xt + (int64_t)c * pitch, v, (size_t)n_in);
            }
        }
    }
    free(z);
    free(b);
    return near;
}
