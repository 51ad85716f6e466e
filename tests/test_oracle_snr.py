"""Pins for the oracle's statistics, boxcar S/N and candidate selection
(Sec. "Integration", "S/N evaluation", "Candidate selection").

The paper leaves the S/N method open; the reading (mean and population
standard deviation of the chunk's own series, sliding boxcar, S/N = (B - w
mu)/(sigma sqrt(w))) is pinned by: scipy's z-score (w = 1), the identity
S/N_w(t) = sum_{k<w} z(t+k) / sqrt(w) evaluated with numpy's convolution,
affine invariance, a closed-form spike whose S/N is exactly 8 (which also
pins the strict comparison), and unit variance on white noise.
"""
import numpy as np
import pytest
from scipy import stats as sstats

import oracle


def test_stats_match_numpy_population():
    rng = np.random.default_rng(0)
    s = rng.integers(-5000, 400000, size=1234)
    mu, sd = oracle.stats(s)
    assert mu == pytest.approx(np.mean(s), rel=1e-14)
    assert sd == pytest.approx(np.std(s, ddof=0), rel=1e-12)


@pytest.mark.parametrize("w", [1, 2, 5, 16, 64])
def test_boxcar_snr_equals_summed_zscore(w):
    rng = np.random.default_rng(w)
    s = rng.integers(190000, 200000, size=777).astype(np.int64)
    mu, sd = oracle.stats(s)
    got = oracle.boxcar_snr(s, w, mu, sd)
    z = sstats.zscore(s.astype(np.float64), ddof=0)
    want = np.convolve(z, np.ones(w), mode="valid") / np.sqrt(w)
    assert got.shape == (777 - w + 1,)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-9)


def test_affine_invariance():
    rng = np.random.default_rng(7)
    s = rng.integers(0, 1000, size=500).astype(np.int64)
    s2 = 3 * s + 12345
    for w in (1, 4, 32):
        a = oracle.boxcar_snr(s, w, *oracle.stats(s))
        b = oracle.boxcar_snr(s2, w, *oracle.stats(s2))
        np.testing.assert_allclose(a, b, atol=1e-10)


def test_exact_spike_and_strict_threshold():
    # 65 samples: one spike of 65, else 0.  mean = 1, sum of squared deviations
    # = 64*1 + 64^2 = 4160, variance = 64, sigma = 8; spike S/N = (65-1)/8 = 8.
    s = np.zeros(65, np.int64)
    s[30] = 65
    mu, sd = oracle.stats(s)
    assert (mu, sd) == (1.0, 8.0)
    snr = oracle.boxcar_snr(s, 1, mu, sd)
    assert snr[30] == 8.0
    # through the whole search: zero-delay plan, one channel, one TAB
    x = np.zeros((1, 1, 80), np.uint8)
    x[0, 0, 30] = 65
    plan = [dict(dm0=0.0, ddm=1.0, n_dm=1, downsamp=1, widths=[1])]
    got, n, _ = oracle.search(x, np.zeros((1, 1)), [1400.0], 1e-3, plan, 8.0, 65)
    assert n == 0                                      # "exceeds": 8.0 is not > 8.0
    got, n, _ = oracle.search(x, np.zeros((1, 1)), [1400.0], 1e-3, plan, 7.999, 65)
    assert n == 1 and got[0]["t_native"] == 30 and got[0]["snr"] == 8.0


def test_white_noise_unit_variance():
    rng = np.random.default_rng(11)
    s = np.rint(rng.normal(2.0e5, 600.0, size=200000)).astype(np.int64)
    mu, sd = oracle.stats(s)
    for w in (1, 4, 64):
        snr = oracle.boxcar_snr(s, w, mu, sd)
        # overlapping windows leave about n/w independent values: 4-sigma bounds
        tol = 4.0 * np.sqrt(2.0 * w / s.size)
        assert abs(snr.mean()) < 4.0 * np.sqrt(w / s.size) + 1e-9
        assert abs(snr.var() - 1.0) < tol
    snr1 = oracle.boxcar_snr(s, 1, mu, sd)
    assert abs(snr1.mean()) < 1e-9 and abs(snr1.var() - 1.0) < 1e-9


def test_constant_series_emits_nothing():
    x = np.full((1, 2, 50), 100, np.uint8)
    plan = [dict(dm0=0.0, ddm=1.0, n_dm=2, downsamp=1, widths=[1, 2])]
    got, n, _ = oracle.search(x, np.zeros((1, 2)), [1300.0, 1400.0], 1e-3, plan, -100.0, 40)
    assert n == 0
