"""Pins for the oracle's dispersion-delay table (Sec. "Dedispersion").

The paper prints no dispersion constant and no worked delay; the pins are the
physics (no delay at DM 0 or in the top channel, monotone in DM and 1/f^2),
exact rational arithmetic of the same law (rounding half away from zero), and
closed-form values worked by hand below.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

KDM = Fraction(4148808, 1000)  # s MHz^2 / (pc cm^-3), cold-plasma constant


def exact_delay(f, f_top, dm, t_samp, D):
    """Exact rational value of K*DM*(f^-2 - f_top^-2)/(D t_samp) for the binary
    doubles given, rounded half away from zero; also returns the distance of
    the fractional part from 1/2."""
    f, f_top, dm, t_samp = (Fraction(float(v)) for v in (f, f_top, dm, t_samp))
    x = KDM * dm * (1 / (f * f) - 1 / (f_top * f_top)) / (D * t_samp)
    assert x >= 0
    fl = x.numerator // x.denominator
    frac = x - fl
    r = fl + 1 if frac >= Fraction(1, 2) else fl
    return int(r), abs(float(frac) - 0.5)


def test_hand_worked_values():
    """Closed-form values worked by hand (tests/golden/delays_closed_form.txt)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "delays_closed_form.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 6
    for f, f_top, dm, t, D, real, rounded in rows:
        d = oracle.delays([float(f), float(f_top)], float(t), float(dm), 1.0, 1, downsamp=int(D))
        assert d.tolist() == [[int(rounded), 0]]
        exact, _ = exact_delay(float(f), float(f_top), float(dm), float(t), int(D))
        assert exact == int(rounded) and abs(exact - float(real)) <= 0.5


def test_zero_dm_and_top_channel():
    f = synth.channel_freqs(1536)
    d = oracle.delays(f, 81.92e-6, 0.0, 0.2, 64)
    assert (d[0] == 0).all()
    assert (d[:, -1] == 0).all()
    # any channel order: the top channel is the one with the largest frequency
    perm = np.random.default_rng(0).permutation(1536)
    dp = oracle.delays(f[perm], 81.92e-6, 0.0, 0.2, 64)
    assert (dp == d[:, perm]).all()


def test_monotone_and_nonnegative():
    f = synth.channel_freqs(1536)
    d = oracle.delays(f, 81.92e-6, 0.0, 0.2, 2048)
    assert (d >= 0).all()
    assert (np.diff(d, axis=0) >= 0).all()       # non-decreasing in DM
    assert (np.diff(d, axis=1) <= 0).all()       # non-increasing in frequency
    assert d.max() == d[-1, 0]


@pytest.mark.parametrize("n_chan,dm0,ddm,n_dm,D", [
    (128, 0.0, 1.0, 256, 1),
    (1536, 0.0, 0.2, 2048, 1),
    (1536, 409.6, 0.8, 1024, 2),
    (1536, 2867.2, 3.2, 667, 8),
])
def test_exact_rational_agreement(n_chan, dm0, ddm, n_dm, D):
    f = synth.channel_freqs(n_chan)
    t = 81.92e-6
    d, ties = oracle.delays(f, t, dm0, ddm, n_dm, D, return_ties=True)
    rng = np.random.default_rng(n_chan + n_dm)
    idx_i = rng.integers(0, n_dm, size=40)
    idx_c = rng.integers(0, n_chan, size=40)
    checked = 0
    for i, c in zip(idx_i.tolist() + [n_dm - 1], idx_c.tolist() + [0]):
        dm = dm0 + i * ddm            # same binary double as the oracle forms
        r, tie_dist = exact_delay(f[c], f.max(), dm, t, D)
        if tie_dist < 1e-9:
            continue
        assert d[i, c] == r, (i, c)
        checked += 1
    assert checked >= 30


def test_worked_maxima_for_arts_band():
    # Largest delay in the lowest channel centre, for the plans of the workloads.
    f128 = synth.channel_freqs(128)
    f1536 = synth.channel_freqs(1536)
    t = 81.92e-6
    for (f, dm0, ddm, n, D) in [(f128, 0, 1.0, 256, 1), (f1536, 0, 0.2, 2048, 1),
                                (f1536, 409.6, 0.8, 1024, 2), (f1536, 1228.8, 1.6, 1024, 4),
                                (f1536, 2867.2, 3.2, 667, 8)]:
        dm_last = dm0 + (n - 1) * ddm
        want, _ = exact_delay(f.min(), f.max(), dm_last, t, D)
        assert oracle.delays(f, t, dm0, ddm, n, D).max() == want


def test_downsampled_delay_tracks_native():
    f = synth.channel_freqs(1536)
    t = 81.92e-6
    d1 = oracle.delays(f, t, 409.6, 0.8, 64, 1)
    for D in (2, 4, 8):
        dD = oracle.delays(f, t, 409.6, 0.8, 64, D)
        assert np.abs(dD - d1 / D).max() <= 0.5 + 0.5 / D + 1e-9
