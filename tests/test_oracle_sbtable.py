"""Pins of the oracle's SB table (appendix "Synthesized Beams"), and the
library's table against it (host code; no GPU).

Hand-worked values use the appendix's Apertif-10 numbers (N_TAB = 12,
alpha = 0.80, B_max = 1296 m, B_cq = 144 m, f_max = 1500 MHz, 71 SBs)."""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle

GEOM = dict(f_max_mhz=1500.0, alpha=0.8, b_max_m=1296.0, b_cq_m=144.0)


def _table(freqs, n_sb=71, n_tab=12, G=1):
    return oracle.sb_table(n_tab, n_sb, freqs, GEOM["f_max_mhz"], GEOM["alpha"], GEOM["b_max_m"], GEOM["b_cq_m"], G)


def test_paper_counts():
    # the appendix's own counts follow from its formulas: 12 TABs (Apertif-10), 9 (Apertif-8), 71 SBs
    assert int(np.ceil(1296.0 / (0.80 * 144.0))) == 12
    assert int(np.ceil(1008.0 / (0.78 * 144.0))) == 9
    theta_sb = 0.80 * (299792458.0 / 1500e6) / 1296.0            # SB spacing at f_max, rad
    fov = (30.0 / 60.0) * np.pi / 180.0                           # 30 arcmin
    assert int(round(fov / theta_sb)) == 71


def _switches(row):
    return [k for k in range(1, len(row)) if row[k] != row[k - 1]]


def test_centre_and_inner_sbs():
    f = np.linspace(1200.0, 1520.0, 641)
    m = _table(f)
    assert (m[35] == 6).all()                       # n_SB = 0: central TAB (row N/2) everywhere
    for s in (34, 36):                               # |n_SB| = 1: the next TAB lands there only at f = 0
        assert len(set(m[s].tolist())) == 1
    assert m[36, 0] == 7 and m[34, 0] == 5


def test_hand_worked_switch_frequencies():
    # n_SB = 35: 35 mod 12 = 11 > 5 -> n_TAB = -1, n_gr = 3.
    # f_j = 1500 (3*1296 + (-1 - j)*0.8*144) / (3*1296 - 0.8*144); odd SB -> f_sw = 0.25 f_j + 0.75 f_{j+1}
    num = lambda j: Fr(3 * 1296) + Fr(-1 - j) * Fr(4, 5) * 144
    den = Fr(3 * 1296) - Fr(4, 5) * 144
    fj = lambda j: Fr(1500) * num(j) / den
    sw0 = float(Fr(1, 4) * fj(0) + Fr(3, 4) * fj(1))
    sw1 = float(Fr(1, 4) * fj(1) + Fr(3, 4) * fj(2))
    assert abs(sw0 - 1465.648854961832) < 1e-9 and abs(sw1 - 1419.8473282442748) < 1e-9
    f = np.array([sw0 + 0.01, sw0 - 0.01, sw1 + 0.01, sw1 - 0.01])
    m = _table(f)
    # rows n_TAB + 6: -1 above the first switch, -2 below it, -3 below the second
    assert m[70].tolist() == [5, 4, 4, 3]
    # n_SB = 5: n_TAB = 5, n_gr = 0, f_1 = 1500 * 4/5 = 1200, odd -> switch at 0.25*1500 + 0.75*1200 = 1275
    m = _table(np.array([1275.01, 1274.99]))
    assert m[40].tolist() == [11, 10]
    # n_SB = -4 (even): n_TAB = -4, f_1 = 1500 * 3/4 = 1125, switch at 0.75*1500 + 0.25*1125 = 1406.25 towards -3
    m = _table(np.array([1406.26, 1406.24]))
    assert m[31].tolist() == [2, 3]


def test_switches_step_one_tab_towards_the_centre():
    f = np.linspace(1220.0, 1520.0, 1536)
    m = _table(f)
    for s in range(71):
        nsb = s - 35
        for k in _switches(m[s][::-1]):              # walk down in frequency
            a, b = int(m[s][::-1][k - 1]), int(m[s][::-1][k])
            step = (b - a) % 12
            assert step == (11 if nsb > 0 else 1), (s, k, a, b)


def test_subband_quantisation():
    f = np.linspace(1220.0, 1520.0, 1536)
    g48 = _table(f, G=48)
    for b in range(0, 1536, 48):
        blk = g48[:, b:b + 48]
        assert (blk == blk[:, :1]).all()
        fc = np.array([f[b:b + 48].mean()])
        assert (blk[:, 0] == _table(fc)[:, 0]).all()


def test_library_matches_oracle():
    import paper_2205_12362_b300 as fdd
    for n_tab, n_sb, G, n_chan in [(12, 71, 1, 1536), (12, 71, 48, 1536), (8, 33, 1, 300), (12, 151, 16, 1536)]:
        f = np.linspace(1220.0, 1520.0, n_chan)
        got = fdd.sb_table(n_tab, n_sb, f, chan_per_subband=G)
        want = oracle.sb_table(n_tab, n_sb, f, 1500.0, 0.8, 1296.0, 144.0, G)
        assert (got == want).all(), (n_tab, n_sb, G)
    with pytest.raises(fdd.FddError):
        fdd.sb_table(11, 5, np.linspace(1220, 1520, 8))
