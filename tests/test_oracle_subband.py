"""Pins of the oracle's two-step subband dedispersion (Sec. "AMBER",
"Dedispersion"; Table "dedispersion setup": 32 subbands, subbanding DM step
32x the fine step), an approximation of brute force:

* subbands of one channel make it brute force exactly (no intra-subband delay);
* DM 0 gives the per-SB channel sum;
* an impulse in one channel lands where the exact-rational delays of both steps
  put it (subband reference = its top channel, coarse DM = block midpoint);
* the S/N of injected pulses stays close to brute force's at the paper's
  settings (the loss grows for pulses narrower than the intra-subband smearing)."""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
import synth

T = synth.ARTS_T_SAMP_S


def test_one_channel_subbands_are_brute_force():
    f = synth.channel_freqs(64)
    rng = np.random.default_rng(1)
    sb = rng.integers(0, 3, size=(2, 64)).astype(np.int32)
    ranges = [dict(dm0=10.0, ddm=1.3, n_dm=20, downsamp=1, widths=[1, 4])]
    n_out = 700
    n_in = n_out + int(oracle.delays(f, T, 10.0, 1.3, 20).max()) + 2
    x = synth.filterbank(3, 3, 64, n_in)
    _, _, exact = oracle.search(x, sb, f, T, ranges, 5.0, n_out, n_in=n_in, return_series=True)
    for K in (1, 4, 7):
        _, _, two = oracle.search(x, sb, f, T, [dict(ranges[0], subband=(1, K))], 5.0, n_out, n_in=n_in,
                                  return_series=True)
        assert (two[0] == exact[0]).all()


def test_dm_zero_is_the_channel_sum():
    f = synth.channel_freqs(96)
    sb = np.repeat(np.array([[0, 1, 2, 1, 0, 2], [2, 2, 1, 0, 0, 1]], np.int32), 16, axis=1)
    x = synth.filterbank(4, 3, 96, 300)
    _, _, two = oracle.search(x, sb, f, T, [dict(dm0=0.0, ddm=0.0, n_dm=5, downsamp=1, widths=[1],
                                                 subband=(16, 4))], 5.0, 250, n_in=300, return_series=True)
    want = np.zeros((2, 250), np.int64)
    for c in range(96):
        want += x[sb[:, c], c, :250]
    assert (two[0] == want[:, None, :]).all()


def _round_half_away(q):
    fl = q.numerator // q.denominator
    return fl + 1 if (q - fl) >= Fr(1, 2) else fl


def test_impulse_lands_at_the_two_step_delay():
    # 8 channels, 2 subbands of 4; 6 fine trials in blocks of K = 3
    f = np.array([1210.0 + 37.5 * c for c in range(8)])
    t_samp = 1e-3
    dm0, ddm, n_dm, G, K = 100.0, 10.0, 6, 4, 3
    n_out, n_in = 40, 400
    kdm = Fr(4148808, 1000)
    ff = [Fr(v).limit_denominator(10 ** 6) for v in f]
    f_top = max(ff)
    for c_hit in (0, 2, 5):
        x = np.zeros((1, 8, n_in), np.uint8)
        u0 = 150
        x[0, c_hit, u0] = 1
        _, _, two = oracle.search(x, np.zeros((1, 8), np.int32), f, t_samp,
                                  [dict(dm0=dm0, ddm=ddm, n_dm=n_dm, downsamp=1, widths=[1], subband=(G, K))],
                                  50.0, n_out, n_in=n_in, return_series=True)
        b = c_hit // G
        fb = max(ff[b * G:(b + 1) * G])
        for i in range(n_dm):
            q = i // K
            dmc = Fr(dm0) + (q * K + Fr(K - 1, 2)) * Fr(ddm)
            d1 = _round_half_away(kdm * dmc * (1 / ff[c_hit] ** 2 - 1 / fb ** 2) / Fr(t_samp).limit_denominator(10 ** 9))
            d2 = _round_half_away(kdm * (Fr(dm0) + i * Fr(ddm)) * (1 / fb ** 2 - 1 / f_top ** 2)
                                  / Fr(t_samp).limit_denominator(10 ** 9))
            t_hit = u0 - d1 - d2
            row = two[0][0, i]
            assert row.sum() == (1 if 0 <= t_hit < n_out else 0)
            if 0 <= t_hit < n_out:
                assert row[t_hit] == 1, (c_hit, i)


@pytest.mark.parametrize("dm,width,lo", [(300.0, 4, 0.85), (303.0, 4, 0.85), (306.2, 8, 0.88),
                                         (306.2, 2, 0.65), (306.2, 1, 0.55)])
def test_snr_loss_at_the_paper_settings(dm, width, lo):
    # 1536 channels, 32 subbands of 48, fine step 0.2, coarse step 6.4 (K = 32): trials 293.6..306.2 in
    # two coarse blocks, 293.6..299.8 (coarse DM 296.7) and 300.0..306.2 (coarse DM 303.1); pulses at
    # the second block's first trial (300.0), near its centre (303.0) and at its last trial (306.2)
    f = synth.channel_freqs(1536)
    ranges = [dict(dm0=293.6, ddm=0.2, n_dm=64, downsamp=1, widths=[1, 2, 4, 8, 16])]
    n_out = 2000
    n_in = n_out + int(oracle.delays(f, T, ranges[0]["dm0"], 0.2, 64).max()) + 64
    amp = synth.pulse_amplitude(30.0, 1536, width)
    x = synth.filterbank(5, 1, 1536, n_in, pulses=[dict(tab=0, start=800 + oracle.delays(f, T, dm, 1.0, 1)[0],
                                                        width=width, amp=amp)])
    sb = np.zeros((1, 1536), np.int32)
    a, _, _ = oracle.search(x, sb, f, T, ranges, 6.0, n_out, n_in=n_in, cap=1 << 20)
    b, _, _ = oracle.search(x, sb, f, T, [dict(ranges[0], subband=(48, 32))], 6.0, n_out, n_in=n_in, cap=1 << 20)
    ratio = b["snr"].max() / a["snr"].max()
    assert lo <= ratio <= 1.05, ratio
