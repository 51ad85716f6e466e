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


def _stream_case():
    """A stream of several windows whose length is not a multiple of the
    largest downsampling factor (L = 500: 500 mod 8 = 4, as 12500 mod 8 in
    ARTS), with ranges at D = 1, 2, 3 and 8."""
    n_tab, n_chan, n_sb, L, W = 2, 48, 2, 500, 4
    f = synth.channel_freqs(n_chan)
    ranges = [dict(dm0=0.0, ddm=2.0, n_dm=8, downsamp=1, widths=[1, 2]),
              dict(dm0=16.0, ddm=4.0, n_dm=6, downsamp=2, widths=[1, 4]),
              dict(dm0=40.0, ddm=6.0, n_dm=5, downsamp=3, widths=[1, 2]),
              dict(dm0=70.0, ddm=8.0, n_dm=4, downsamp=8, widths=[1, 2, 4])]
    need = max((int(oracle.delays(f, T_SAMP, r["dm0"], r["ddm"], r["n_dm"], r["downsamp"]).max()) + 2)
               * r["downsamp"] for r in ranges) + 8
    x = synth.filterbank(21, n_tab, n_chan, W * L + need, pulses=[
        dict(tab=1, start=777 + oracle.delays(f, T_SAMP, 50.0, 1.0, 1)[0], width=3, amp=30.0)])
    sb = np.zeros((n_sb, n_chan), np.int32)
    sb[1, 20:] = 1
    return x, f, ranges, sb, L, W, need


def test_absolute_bins_windows_tile_the_one_shot_series():
    """Sec. "Downsampling" read with bins aligned to stream sample 0: the
    series of consecutive windows (bins starting in [wL, (w+1)L)) laid end to
    end equal the one-shot series of the whole stream, bin for bin, and a
    D = 8 range alternates 63 and 62 bins per 500-sample window."""
    x, f, ranges, sb, L, W, need = _stream_case()
    _, _, whole = oracle.search(x, sb, f, T_SAMP, ranges, 1e9, W * L, n_in=x.shape[2], return_series=True,
                                bins_absolute=True)
    parts = [[] for _ in ranges]
    for w in range(W):
        xw = np.ascontiguousarray(x[:, :, w * L:w * L + L + need])
        _, _, ser = oracle.search(xw, sb, f, T_SAMP, ranges, 1e9, L, n_in=L + need, t_offset_native=w * L,
                                  return_series=True, bins_absolute=True)
        for k, s_ in enumerate(ser):
            parts[k].append(s_)
    for k, r in enumerate(ranges):
        cat = np.concatenate(parts[k], axis=2)
        assert cat.shape == whole[k].shape
        assert (cat == whole[k]).all(), "range %d" % k
    assert [p.shape[2] for p in parts[3]] == [63, 62, 63, 62]
    assert [oracle.window_bins(w * L, L, 8) for w in range(2)] == [(0, 63), (4, 62)]


def test_absolute_bins_equal_a_shifted_plain_search():
    """One window in the absolute-bin mode equals, range by range, the plain
    search (bins from input sample 0) of the input advanced by the range's
    phase, with n_r bins and the stream position added to t_native."""
    x, f, ranges, sb, L, W, need = _stream_case()
    t0 = 1501               # stream position 1501: phases 0, 1, 2, 3 for D = 1, 2, 3, 8
    xw = np.ascontiguousarray(x[:, :, t0:t0 + L + need - 1])
    got, n, ser = oracle.search(xw, sb, f, T_SAMP, ranges, 5.0, L, n_in=xw.shape[2], t_offset_native=t0,
                                return_series=True, bins_absolute=True)
    dm_base = 0
    for k, r in enumerate(ranges):
        ph, nr = oracle.window_bins(t0, L, r["downsamp"])
        assert ph == (-t0) % r["downsamp"]
        xs = np.ascontiguousarray(xw[:, :, ph:])
        g2, _, s2 = oracle.search(xs, sb, f, T_SAMP, [r], 5.0, nr * r["downsamp"], n_in=xs.shape[2],
                                  t_offset_native=t0 + ph, return_series=True)
        assert (s2[0] == ser[k]).all()
        mine = got[(got["dm_index"] >= dm_base) & (got["dm_index"] < dm_base + r["n_dm"])]
        assert len(mine) == len(g2)
        assert (mine["t_native"] == g2["t_native"]).all() and (mine["dm_index"] - dm_base == g2["dm_index"]).all()
        dm_base += r["n_dm"]
