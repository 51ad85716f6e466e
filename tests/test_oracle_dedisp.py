"""Pins for the oracle's downsampling and SB-gather dedispersion
(Sec. "Downsampling", Sec. "Dedispersion", Sec. "Hierarchical beam forming").

Each pin is a property fixed by the definition, not a retyping of it:
special cases that reduce to numpy routines, linearity, shift covariance, an
exactly recovered injected pulse, and a scatter-form brute force on tiny
inputs (every input sample pushed to every output it feeds, the adjoint loop
order of the oracle's gather).
"""
import itertools

import numpy as np
import pytest

import oracle
import synth


def _rand_u8(rng, shape, hi=256):
    return rng.integers(0, hi, size=shape, dtype=np.int64).astype(np.uint8)


# ---------------------------------------------------------------- downsample
@pytest.mark.parametrize("D", [1, 2, 3, 4, 8])
def test_downsample_matches_reshape_sum(D):
    rng = np.random.default_rng(D)
    x = _rand_u8(rng, (3, 5, 203))
    y = oracle.downsample(x, D)
    n = 203 // D
    want = x[..., :n * D].astype(np.int64).reshape(3, 5, n, D).sum(-1)
    assert y.shape == (3, 5, n)
    assert (y == want).all()


def test_downsample_identity_and_saturation():
    rng = np.random.default_rng(1)
    x = _rand_u8(rng, (2, 4, 64))
    assert (oracle.downsample(x, 1) == x).all()
    full = np.full((1, 2, 64), 255, np.uint8)
    assert (oracle.downsample(full, 8) == 255 * 8).all()


def test_downsample_chunked_equals_one_shot():
    rng = np.random.default_rng(2)
    x = _rand_u8(rng, (1, 3, 240))
    D = 8
    one = oracle.downsample(x, D)
    parts = [oracle.downsample(np.ascontiguousarray(x[..., a:a + 80]), D) for a in (0, 80, 160)]
    assert (np.concatenate(parts, axis=-1) == one).all()


def test_downsample_respects_pitch():
    rng = np.random.default_rng(3)
    x = _rand_u8(rng, (2, 3, 48))
    y = oracle.downsample(x, 4, n_in=37)
    assert y.shape == (2, 3, 9)
    assert (y == x[..., :36].astype(np.int64).reshape(2, 3, 9, 4).sum(-1)).all()


# ---------------------------------------------------------------- dedisperse
def scatter_brute(y, sb_map, d, n_out):
    """Push every input sample y[tab][c][tau] into each S[s][i][tau - d[i][c]]
    that lies in [0, n_out) for every SB s with sb_map[s][c] == tab."""
    n_tab, n_chan, n_y = y.shape
    n_sb, n_dm = len(sb_map), len(d)
    S = [[[0] * n_out for _ in range(n_dm)] for _ in range(n_sb)]
    for tab, c, tau in itertools.product(range(n_tab), range(n_chan), range(n_y)):
        v = int(y[tab][c][tau])
        for s in range(n_sb):
            if sb_map[s][c] != tab:
                continue
            for i in range(n_dm):
                t = tau - int(d[i][c])
                if 0 <= t < n_out:
                    S[s][i][t] += v
    return np.array(S, dtype=np.int64)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_dedisperse_matches_scatter_brute_force(seed):
    rng = np.random.default_rng(seed)
    n_tab, n_chan, n_dm, n_sb, n_out = 3, 6, 5, 4, 17
    d = rng.integers(0, 9, size=(n_dm, n_chan))           # arbitrary (not monotone) delays
    n_y = n_out + int(d.max()) + int(rng.integers(0, 3))
    y = rng.integers(0, 2000, size=(n_tab, n_chan, n_y)).astype(np.uint32)
    sb_map = rng.integers(0, n_tab, size=(n_sb, n_chan))
    got = oracle.dedisperse(y, sb_map, d, n_out)
    assert (got == scatter_brute(y, sb_map, d, n_out)).all()


def test_dm_zero_is_channel_sum_per_sb():
    rng = np.random.default_rng(4)
    n_tab, n_chan, n_y = 4, 32, 300
    y = rng.integers(0, 256, size=(n_tab, n_chan, n_y)).astype(np.uint32)
    sb_map = rng.integers(0, n_tab, size=(5, n_chan))
    d = np.zeros((1, n_chan), np.int64)
    got = oracle.dedisperse(y, sb_map, d, n_y)
    for s in range(5):
        want = y[sb_map[s], np.arange(n_chan), :].astype(np.int64).sum(0)
        assert (got[s, 0] == want).all()


def test_linearity_and_shift_covariance():
    rng = np.random.default_rng(5)
    f = synth.channel_freqs(64)
    d = oracle.delays(f, 81.92e-6, 0.0, 2.0, 24)
    n_out = 200
    n_y = n_out + int(d.max()) + 8
    a = rng.integers(0, 128, size=(2, 64, n_y)).astype(np.uint32)
    b = rng.integers(0, 128, size=(2, 64, n_y)).astype(np.uint32)
    sb = rng.integers(0, 2, size=(3, 64))
    Sa, Sb = oracle.dedisperse(a, sb, d, n_out), oracle.dedisperse(b, sb, d, n_out)
    assert (oracle.dedisperse(a + b, sb, d, n_out) == Sa + Sb).all()
    k = 5   # delaying the input by k samples delays every output by k
    a_shift = np.zeros_like(a)
    a_shift[..., k:] = a[..., :-k]
    S_shift = oracle.dedisperse(a_shift, sb, d, n_out)
    assert (S_shift[..., k:] == Sa[..., :n_out - k]).all()


def test_injected_pulse_recovered_exactly_on_grid():
    # Zero background, one pulse of amplitude 7 placed along the delay curve
    # of trial 40: the series of trial 40 peaks at t0 with exactly 7 * n_chan.
    n_chan = 96
    f = synth.channel_freqs(n_chan)
    d = oracle.delays(f, 81.92e-6, 0.0, 1.0, 64)
    i0, t0, n_out = 40, 123, 400
    n_y = n_out + int(d.max()) + 1
    y = np.zeros((1, n_chan, n_y), np.uint32)
    y[0, np.arange(n_chan), t0 + d[i0]] = 7
    S = oracle.dedisperse(y, np.zeros((1, n_chan), np.int64), d, n_out)[0]
    assert S[i0, t0] == 7 * n_chan
    assert S.max() == 7 * n_chan
    peaks = np.argwhere(S == S.max())
    # every maximum is a trial whose delays equal trial 40's in all channels
    for i, t in peaks:
        assert t == t0 and (d[i] == d[i0]).all()


def test_sb_gather_single_tab_and_relabel():
    rng = np.random.default_rng(6)
    n_tab, n_chan = 4, 48
    f = synth.channel_freqs(n_chan)
    d = oracle.delays(f, 81.92e-6, 0.0, 3.0, 16)
    n_out = 150
    n_y = n_out + int(d.max()) + 3
    y = rng.integers(0, 256, size=(n_tab, n_chan, n_y)).astype(np.uint32)
    for k in range(n_tab):  # an SB that always picks TAB k is the single-beam search of TAB k
        S = oracle.dedisperse(y, np.full((1, n_chan), k), d, n_out)
        S1 = oracle.dedisperse(y[k:k + 1], np.zeros((1, n_chan), np.int64), d, n_out)
        assert (S == S1).all()
    sb = rng.integers(0, n_tab, size=(5, n_chan))
    perm = rng.permutation(n_tab)          # TAB t moves to slot perm[t]
    y_p = np.empty_like(y)
    y_p[perm] = y
    S = oracle.dedisperse(y, sb, d, n_out)
    S_p = oracle.dedisperse(y_p, perm[sb], d, n_out)
    assert (S == S_p).all()


def test_saturated_input_sum():
    n_chan = 1536
    d = np.zeros((2, n_chan), np.int64)
    y = np.full((1, n_chan, 10), 255 * 8, np.uint32)
    S = oracle.dedisperse(y, np.zeros((1, n_chan), np.int64), d, 10)
    assert (S == 255 * 8 * 1536).all() and S.max() < 2 ** 31
