"""Per-beam streaming search (fdd_stream_*): a beam's chunks pushed in order
from device memory; every window's candidates equal the oracle's search of
that window's samples (t_native absolute, downsampling bins aligned to the
stream), the window schedule follows the max delay, and sequence errors are
refused on the host.  Windows of fdd_search_window laid end to end give the
dedispersed series of one oracle search of the whole stream, bit for bit.

Tolerances: S/N within 1e-4 relative of FP64; candidate sets equal after
ignoring candidates within 1e-3 of the threshold (tests/_cmp.py)."""
import numpy as np
import pytest

import oracle
import synth
from tests._cmp import compare_candidates, oracle_candidate_superset

pytestmark = pytest.mark.gpu

T_SAMP = synth.ARTS_T_SAMP_S


@pytest.fixture(scope="module")
def fdd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_12362_b300 as m
    return m


def _case(chunk=512, n_chunks=10):
    n_tab, n_chan, n_sb = 2, 64, 3
    f = synth.channel_freqs(n_chan)
    ranges = [dict(dm0=0.0, ddm=2.0, n_dm=48, downsamp=1, widths=[1, 2, 4]),
              dict(dm0=96.0, ddm=4.0, n_dm=24, downsamp=2, widths=[1, 4])]
    sb = np.zeros((n_sb, n_chan), np.int16)
    sb[1] = 1
    sb[2, 16:48] = 1
    total = n_chunks * chunk
    pulses = []
    for k in range(5):
        t0, dm = 250 + 900 * k, 15.0 + 35 * k
        pulses.append(dict(tab=k % n_tab, start=t0 + oracle.delays(f, T_SAMP, dm, 1.0, 1)[0], width=1 + k,
                           amp=26.0))
    x = synth.filterbank(77, n_tab, n_chan, total, pitch=total, pulses=pulses)
    return f, ranges, sb, x


def test_stream_windows_match_oracle(fdd):
    import torch
    chunk, n_chunks, thr = 512, 10, 7.0
    f, ranges, sb, x = _case(chunk, n_chunks)
    plan = fdd.Plan(2, 64, 3, f, T_SAMP, ranges, thr, sb)
    md, ws = plan.info(chunk)
    assert md == plan.max_delay and ws == plan.workspace_size(chunk + md, chunk, with_series=True)
    n_in = plan.window_sizes(chunk)[0]
    assert n_in >= chunk + md
    per_window = -(-n_in // chunk)           # chunks per window buffer
    st = fdd.Stream(plan, beam_id=5, chunk_len=chunk, cap=1 << 14)
    cands = torch.zeros((1 << 14, 8), dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    side = torch.cuda.Stream()
    # chunk buffers with a pitch larger than the chunk (rows not contiguous)
    buf = torch.zeros((2, 64, chunk + 48), dtype=torch.uint8, device="cuda")
    seen = []
    for k in range(n_chunks):
        buf[:, :, :chunk].copy_(torch.from_numpy(np.ascontiguousarray(x[:, :, k * chunk:(k + 1) * chunk])))
        use = side if k % 3 == 2 else None  # pushes alternate CUDA streams; order is kept by the object
        if use is not None:
            use.wait_stream(torch.cuda.current_stream())
        assert st.push(buf, k, stream=use) == 0
        t0 = st.results(cands, count)
        torch.cuda.synchronize()
        if k < per_window - 1:
            assert t0 == -1
            continue
        w = k - (per_window - 1)
        assert t0 == w * chunk
        n = int(count.item())
        gpu = fdd.decode_candidates(cands, n)
        ora, _ = oracle_candidate_superset(x[:, :, t0:t0 + n_in], sb, f, T_SAMP, ranges, thr, chunk, n_in,
                                           t_offset=t0, bins_absolute=True)
        compare_candidates(gpu, ora, thr)
        seen.append(n)
        assert st.results(cands, count) == -1  # taken already
    assert len(seen) == n_chunks - per_window + 1
    assert sum(seen) > 0
    st.close()


def test_stream_sequence_and_args(fdd):
    import torch
    chunk = 256
    f, ranges, sb, x = _case(chunk, 4)
    plan = fdd.Plan(2, 64, 3, f, T_SAMP, ranges, 7.0, sb)
    st = fdd.Stream(plan, beam_id=0, chunk_len=chunk)
    c = torch.zeros((2, 64, chunk), dtype=torch.uint8, device="cuda")
    assert st.push(c, 1) == fdd.FDD_ERR_SEQUENCE      # chunk 0 expected
    assert st.push(c, 0) == 0
    assert st.push(c, 0) == fdd.FDD_ERR_SEQUENCE      # duplicate
    assert st.push(c, 1) == 0
    with pytest.raises(ValueError):
        st.push(c[:, :, :chunk - 1], 2)
    torch.cuda.synchronize()
    st.close()


def _tiling_case():
    """A stream whose chunk length is not a multiple of the largest
    downsampling factor (500 = 62.5 x 8, like 12500 in ARTS), with D = 1, 3
    and 8."""
    n_tab, n_chan, n_sb, L, W = 2, 64, 3, 500, 5
    f = synth.channel_freqs(n_chan)
    ranges = [dict(dm0=0.0, ddm=2.0, n_dm=40, downsamp=1, widths=[1, 2, 4]),
              dict(dm0=80.0, ddm=5.0, n_dm=16, downsamp=3, widths=[1, 2]),
              dict(dm0=160.0, ddm=9.0, n_dm=12, downsamp=8, widths=[1, 2, 4])]
    sb = np.zeros((n_sb, n_chan), np.int16)
    sb[1] = 1
    sb[2, 16:48] = 1
    pulses = [dict(tab=k % n_tab, start=140 + 470 * k + oracle.delays(f, T_SAMP, dm, 1.0, 1)[0], width=2 + k,
                   amp=28.0) for k, dm in enumerate([20.0, 110.0, 200.0, 60.0])]
    return f, ranges, sb, pulses, L, W


def test_windows_tile_the_one_shot_oracle_series(fdd):
    """Sec. "Downsampling", bins aligned to the stream: the series of
    consecutive fdd_search_window windows (including the D = 8 range, whose
    windows alternate 63 and 62 bins) are the one-shot oracle series of the
    whole stream, cut at the windows' first bins, bit for bit."""
    import torch
    f, ranges, sb, pulses, L, W = _tiling_case()
    plan = fdd.Plan(2, 64, 3, f, T_SAMP, ranges, 7.0, sb)
    n_in, _, _ = plan.window_sizes(L)
    total = (W - 1) * L + n_in
    x = synth.filterbank(91, 2, 64, total, pitch=synth.padded_pitch(total), pulses=pulses)
    _, _, whole = oracle.search(x, sb, f, T_SAMP, ranges, 1e9, W * L, n_in=total, return_series=True,
                                bins_absolute=True)
    got = [[] for _ in ranges]
    for w in range(W):
        win = np.zeros((2, 64, synth.padded_pitch(n_in)), np.uint8)
        win[:, :, :n_in] = x[:, :, w * L:w * L + n_in]
        res = plan.search_window(torch.from_numpy(win).cuda(), n_in, L, w * L, want_series=True)
        torch.cuda.synchronize()
        for k, v in enumerate(plan.series_views(res.series, L, t0=w * L)):
            got[k].append(v.cpu().numpy())
    assert [g.shape[2] for g in got[2]] == [63, 62, 63, 62, 63]
    for k in range(len(ranges)):
        cat = np.concatenate(got[k], axis=2)
        assert cat.shape == whole[k].shape, (k, cat.shape, whole[k].shape)
        assert (cat == whole[k]).all(), "range %d" % k


def test_stream_with_phases_matches_oracle(fdd):
    """The per-beam stream on the same 500-sample chunks: every window's
    candidates equal the oracle's search of that window with bins aligned to
    the stream (t_native absolute)."""
    import torch
    f, ranges, sb, pulses, L, W = _tiling_case()
    thr = 7.0
    plan = fdd.Plan(2, 64, 3, f, T_SAMP, ranges, thr, sb)
    n_in, _, _ = plan.window_sizes(L)
    per_window = -(-n_in // L)
    n_chunks = per_window + W - 1
    x = synth.filterbank(92, 2, 64, n_chunks * L, pitch=n_chunks * L, pulses=pulses)
    st = fdd.Stream(plan, beam_id=1, chunk_len=L, cap=1 << 14)
    cands = torch.zeros((1 << 14, 8), dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    n_win = total = 0
    for k in range(n_chunks):
        c = torch.from_numpy(np.ascontiguousarray(x[:, :, k * L:(k + 1) * L])).cuda()
        assert st.push(c, k) == 0
        t0 = st.results(cands, count)
        torch.cuda.synchronize()
        if t0 < 0:
            continue
        n = int(count.item())
        gpu = fdd.decode_candidates(cands, n)
        ora, _ = oracle_candidate_superset(x[:, :, t0:t0 + n_in], sb, f, T_SAMP, ranges, thr, L, n_in,
                                           t_offset=t0, bins_absolute=True)
        compare_candidates(gpu, ora, thr)
        d8 = gpu[gpu["downsamp"] == 8]
        assert ((d8["t_native"] % 8) == 0).all()          # bins start at multiples of 8 of the stream
        n_win += 1
        total += n
    st.close()
    assert n_win == W and total > 0


@pytest.mark.parametrize("t0", [1501, 4000, 7])
def test_window_at_any_phase_matches_oracle(fdd, t0):
    """One fdd_search_window at stream positions whose bin phases are odd
    (1501: phases 1, 3, 5, 13 for D = 2, 4, 8, 16, read through the
    downsampler's unaligned path), aligned (4000) and tiny (7): series
    bit-exact and candidates equal to the oracle's window search."""
    import torch
    n_tab, n_chan, n_sb, L = 2, 64, 2, 700
    f = synth.channel_freqs(n_chan)
    ranges = [dict(dm0=0.0, ddm=2.0, n_dm=24, downsamp=1, widths=[1, 4]),
              dict(dm0=48.0, ddm=3.0, n_dm=16, downsamp=2, widths=[1, 2]),
              dict(dm0=96.0, ddm=5.0, n_dm=12, downsamp=4, widths=[1, 2]),
              dict(dm0=156.0, ddm=8.0, n_dm=8, downsamp=8, widths=[1, 2]),
              dict(dm0=220.0, ddm=12.0, n_dm=8, downsamp=16, widths=[1])]
    sb = np.zeros((n_sb, n_chan), np.int16)
    sb[1, 10:40] = 1
    thr = 6.0
    plan = fdd.Plan(n_tab, n_chan, n_sb, f, T_SAMP, ranges, thr, sb)
    n_in, _, _ = plan.window_sizes(L)
    pulses = [dict(tab=1, start=200 + oracle.delays(f, T_SAMP, 150.0, 1.0, 1)[0], width=8, amp=30.0)]
    x = synth.filterbank(93 + t0, n_tab, n_chan, n_in, pitch=synth.padded_pitch(n_in), pulses=pulses)
    res = plan.search_window(torch.from_numpy(x).cuda(), n_in, L, t0, want_series=True)
    torch.cuda.synchronize()
    ora, o_series = oracle_candidate_superset(x, sb, f, T_SAMP, ranges, thr, L, n_in, t_offset=t0,
                                              return_series=True, bins_absolute=True)
    for g, o in zip(plan.series_views(res.series, L, t0=t0), o_series):
        assert g.shape == o.shape
        assert (g.cpu().numpy() == o).all()
    gpu, n = res.candidates()
    compare_candidates(gpu, ora, thr)
    assert n > 0
