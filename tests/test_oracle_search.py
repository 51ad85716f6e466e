"""End-to-end pins for the oracle's search on the small workloads:
injected-pulse recall at the right DM / time / width with the expected S/N,
silence on noise, agreement with the stage-by-stage functions, and the
native-sample bookkeeping of downsampled ranges."""
import numpy as np
import pytest

import oracle
import synth

T_SAMP = synth.ARTS_T_SAMP_S


def tiny_case(seed=1, amp=24.0, pulse=True):
    n_chan, n_out = 128, 4096
    f = synth.channel_freqs(n_chan)
    d = oracle.delays(f, T_SAMP, 0.0, 1.0, 256)
    n_in = n_out + int(d.max())
    t0 = 1500
    pulses = [dict(tab=0, start=t0 + oracle.delays(f, T_SAMP, 100.0, 1.0, 1)[0], width=4, amp=amp)] \
        if pulse else []
    x = synth.filterbank(seed, 1, n_chan, n_in, pulses=pulses)
    plan = [dict(dm0=0.0, ddm=1.0, n_dm=256, downsamp=1, widths=[1, 2, 4, 8, 16])]
    return x, f, plan, n_in, n_out, t0


def test_tiny_pulse_recovered():
    x, f, plan, n_in, n_out, t0 = tiny_case()
    got, n, _ = oracle.search(x, np.zeros((1, 128)), f, T_SAMP, plan, 8.0, n_out, n_in=n_in)
    assert n > 0 and n == len(got)
    best = got[np.argmax(got["snr"])]
    assert abs(int(best["dm_index"]) - 100) <= 2
    assert abs(int(best["t_native"]) - t0) <= 4
    assert 2 <= int(best["width_native"]) <= 8
    # ideal matched-filter S/N: 24 * sqrt(128 * 4) / 16 = 33.9
    assert 0.85 * 33.94 < best["snr"] < 1.15 * 33.94
    # every candidate is near the pulse in time (no noise candidates)
    assert (np.abs(got["t_native"] - t0) < 200).all()


def test_tiny_noise_silent():
    x, f, plan, n_in, n_out, _ = tiny_case(seed=5, pulse=False)
    _, n, _ = oracle.search(x, np.zeros((1, 128)), f, T_SAMP, plan, 8.0, n_out, n_in=n_in)
    assert n == 0


def test_search_equals_stage_functions_multi_range():
    rng = np.random.default_rng(3)
    n_tab, n_chan, n_sb = 3, 40, 4
    f = synth.channel_freqs(n_chan)
    plan = [dict(dm0=0.0, ddm=4.0, n_dm=6, downsamp=1, widths=[1, 2, 4]),
            dict(dm0=24.0, ddm=8.0, n_dm=5, downsamp=2, widths=[1, 3]),
            dict(dm0=64.0, ddm=16.0, n_dm=3, downsamp=4, widths=[2])]
    n_out = 301
    need = max(int(oracle.delays(f, T_SAMP, r["dm0"], r["ddm"], r["n_dm"], r["downsamp"]).max())
               * r["downsamp"] + (n_out // r["downsamp"]) * r["downsamp"] for r in plan)
    n_in = need + 5
    x = synth.filterbank(9, n_tab, n_chan, n_in)
    sb = rng.integers(0, n_tab, size=(n_sb, n_chan))
    thr = 1.5
    got, n, series = oracle.search(x, sb, f, T_SAMP, plan, thr, n_out, n_in=n_in,
                                   t_offset_native=1000, return_series=True)
    want = []
    dm_base = 0
    for r, S_r in zip(plan, series):
        D = r["downsamp"]
        y = oracle.downsample(x, D, n_in=n_in)
        d = oracle.delays(f, T_SAMP, r["dm0"], r["ddm"], r["n_dm"], D)
        S = oracle.dedisperse(y, sb, d, n_out // D)
        assert (S == S_r).all()
        for s in range(n_sb):
            for i in range(r["n_dm"]):
                mu, sd = oracle.stats(S[s, i])
                for w in r["widths"]:
                    snr = oracle.boxcar_snr(S[s, i], w, mu, sd)
                    for t in np.nonzero(snr > thr)[0]:
                        want.append((s, dm_base + i, w * D, t * D + 1000, snr[t]))
        dm_base += r["n_dm"]
    want.sort()
    assert n == len(want) == len(got)
    key = sorted(zip(got["sb"].tolist(), got["dm_index"].tolist(), got["width_native"].tolist(),
                     got["t_native"].tolist(), got["snr"].tolist()))
    assert key == want


def test_short_input_rejected():
    f = synth.channel_freqs(16)
    plan = [dict(dm0=0.0, ddm=10.0, n_dm=8, downsamp=1, widths=[1])]
    dmax = int(oracle.delays(f, T_SAMP, 0.0, 10.0, 8).max())
    x = np.zeros((1, 16, 100 + dmax - 1), np.uint8)
    with pytest.raises(ValueError):
        oracle.search(x, np.zeros((1, 16)), f, T_SAMP, plan, 8.0, 100)
