"""CUDA path vs the oracle, element by element, through the C ABI.

Tolerances: dedispersed series bit-exact (exact integer sums on both sides);
S/N within 1e-4 relative (floor 1) of the FP64 oracle; candidate sets equal
after ignoring candidates whose oracle S/N is within 1e-3 of the threshold
(see tests/_cmp.py)."""
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


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run_both(fdd, x, sb_map, freqs, ranges, thr, n_out, n_in, t_offset=0, cap=1 << 20):
    n_tab, n_chan, _ = x.shape
    plan = fdd.Plan(n_tab, n_chan, sb_map.shape[0], freqs, T_SAMP, ranges, thr, sb_map)
    res = plan.search(to_dev(x), n_in, n_out, t_offset=t_offset, cap=cap, want_series=True)
    import torch
    torch.cuda.synchronize()
    gpu, n = res.candidates()
    assert n == len(gpu), "GPU candidate buffer overflowed (cap %d, count %d)" % (cap, n)
    g_series = [s.cpu().numpy() for s in plan.series_views(res.series, n_out)]
    ora, o_series = oracle_candidate_superset(x, sb_map, freqs, T_SAMP, ranges, thr, n_out, n_in,
                                              t_offset=t_offset, return_series=True)
    return plan, gpu, g_series, ora, o_series


def tiny_config():
    n_chan, n_out = 128, 4096
    f = synth.channel_freqs(n_chan)
    d = oracle.delays(f, T_SAMP, 0.0, 1.0, 256)
    n_in = n_out + int(d.max())
    start = 1500 + oracle.delays(f, T_SAMP, 100.0, 1.0, 1)[0]
    x = synth.filterbank(1, 1, n_chan, n_in, pulses=[dict(tab=0, start=start, width=4, amp=24.0)])
    ranges = [dict(dm0=0.0, ddm=1.0, n_dm=256, downsamp=1, widths=[1, 2, 4, 8, 16])]
    return x, f, ranges, n_in, n_out


def test_tiny_plain_search(fdd):
    x, f, ranges, n_in, n_out = tiny_config()
    sb = np.zeros((1, 128), np.int16)
    plan, gpu, gs, ora, os_ = run_both(fdd, x, sb, f, ranges, 8.0, n_out, n_in)
    assert (gs[0] == os_[0]).all()
    assert compare_candidates(gpu, ora, 8.0) > 0
    best = gpu[np.argmax(gpu["snr"])]
    assert abs(int(best["dm_index"]) - 100) <= 2


def test_library_delay_table_matches_oracle(fdd):
    f = synth.channel_freqs(1536)
    ranges = [dict(dm0=0.0, ddm=0.2, n_dm=2048, downsamp=1, widths=[1]),
              dict(dm0=409.6, ddm=0.8, n_dm=1024, downsamp=2, widths=[1]),
              dict(dm0=2867.2, ddm=3.2, n_dm=667, downsamp=8, widths=[1])]
    plan = fdd.Plan(1, 1536, 1, f, T_SAMP, ranges, 8.0, np.zeros((1, 1536)))
    for r, rg in enumerate(ranges):
        want = oracle.delays(f, T_SAMP, rg["dm0"], rg["ddm"], rg["n_dm"], rg["downsamp"])
        assert (plan.delays(r) == want).all()
    assert plan.max_delay == max(int(oracle.delays(f, T_SAMP, rg["dm0"], rg["ddm"], rg["n_dm"],
                                                   rg["downsamp"]).max()) * rg["downsamp"] for rg in ranges)


@pytest.mark.parametrize("seed,n_chan,n_out", [(0, 37, 1001), (1, 64, 777), (2, 300, 2050), (3, 16, 96)])
def test_multi_range_sb_gather_ragged(fdd, seed, n_chan, n_out):
    rng = np.random.default_rng(seed)
    n_tab, n_sb = 3, 5
    f = synth.channel_freqs(n_chan)
    ranges = [dict(dm0=0.0, ddm=2.0, n_dm=19, downsamp=1, widths=[1, 2, 4, 64]),
              dict(dm0=38.0, ddm=4.0, n_dm=7, downsamp=2, widths=[1, 3, 8]),
              dict(dm0=66.0, ddm=6.0, n_dm=9, downsamp=3, widths=[2, 5]),
              dict(dm0=120.0, ddm=8.0, n_dm=33, downsamp=4, widths=[1, 16]),
              dict(dm0=384.0, ddm=16.0, n_dm=5, downsamp=8, widths=[1, 2, 500])]
    need = max(int(oracle.delays(f, T_SAMP, r["dm0"], r["ddm"], r["n_dm"], r["downsamp"]).max())
               * r["downsamp"] + (n_out // r["downsamp"]) * r["downsamp"] for r in ranges)
    n_in = need + int(rng.integers(0, 9))
    x = synth.filterbank(seed + 100, n_tab, n_chan, n_in)
    sb = rng.integers(0, n_tab, size=(n_sb, n_chan)).astype(np.int16)
    plan, gpu, gs, ora, os_ = run_both(fdd, x, sb, f, ranges, 3.0, n_out, n_in, t_offset=12345)
    for r in range(len(ranges)):
        assert gs[r].shape == os_[r].shape
        assert (gs[r] == os_[r]).all(), "series of range %d differ" % r
    assert compare_candidates(gpu, ora, 3.0) > 10


def test_swar_flush_saturated(fdd):
    # 600 channels of 255 (more than 257 channels per 16-bit lane) plus noise rows
    n_chan, n_out = 600, 700
    f = synth.channel_freqs(n_chan)
    ranges = [dict(dm0=0.0, ddm=1.0, n_dm=40, downsamp=1, widths=[1]),
              dict(dm0=40.0, ddm=2.0, n_dm=20, downsamp=8, widths=[1])]
    need = max(int(oracle.delays(f, T_SAMP, r["dm0"], r["ddm"], r["n_dm"], r["downsamp"]).max())
               * r["downsamp"] + n_out for r in ranges)
    x = np.full((2, n_chan, synth.padded_pitch(need)), 255, np.uint8)
    x[1] = synth.filterbank(5, 1, n_chan, need, pitch=x.shape[2])[0]
    sb = np.zeros((3, n_chan), np.int16)
    sb[1] = 1
    sb[2, ::2] = 1
    plan, gpu, gs, ora, os_ = run_both(fdd, x, sb, f, ranges, 8.0, n_out, need)
    assert (gs[0][0] == 255 * n_chan).all()
    assert (gs[1][0] == 255 * 8 * n_chan).all()
    for r in range(2):
        assert (gs[r] == os_[r]).all()
    compare_candidates(gpu, ora, 8.0)


@pytest.mark.parametrize("D", [1, 2, 3, 4, 8, 16])
def test_downsample_stage(fdd, D):
    rng = np.random.default_rng(D)
    n_in = 1000 + D
    x = rng.integers(0, 256, size=(3, 5, synth.padded_pitch(n_in)), dtype=np.int64).astype(np.uint8)
    out = fdd.downsample_u8(to_dev(x), n_in, D)
    got = out.cpu().numpy().view(np.uint16)[..., : n_in // D]
    want = oracle.downsample(x, D, n_in=n_in)
    assert (got == want).all()


def arts_single_sb():
    n_chan, n_out = 1536, synth.ARTS_CHUNK
    f = synth.channel_freqs(n_chan)
    d = oracle.delays(f, T_SAMP, 0.0, 0.2, 2048)
    n_in = n_out + int(d.max())
    prm = synth.random_pulses(2, 10, [0], 50.0, 400.0, [1, 2, 4, 8, 16, 32], 8.0, 50.0, 200, n_out - 200)
    pulses = []
    for p in prm:
        dm_grid = round(p["dm"] / 0.2) * 0.2
        start = p["t0"] + oracle.delays(f, T_SAMP, dm_grid, 1.0, 1)[0]
        pulses.append(dict(tab=0, start=start, width=p["width"],
                           amp=synth.pulse_amplitude(p["snr"], n_chan, p["width"])))
    x = synth.filterbank(2, 1, n_chan, n_in, pulses=pulses)
    ranges = [dict(dm0=0.0, ddm=0.2, n_dm=2048, downsamp=1, widths=[1, 2, 4, 8, 16, 32, 64])]
    return x, f, ranges, n_in, n_out, prm


def test_arts_single_sb_full_size(fdd):
    x, f, ranges, n_in, n_out, prm = arts_single_sb()
    plan, gpu, gs, ora, os_ = run_both(fdd, x, np.zeros((1, 1536), np.int16), f, ranges, 8.0, n_out, n_in)
    assert (gs[0] == os_[0]).all()
    assert plan.status() == 0                     # no raw-row (TMA) wait gave up
    n = compare_candidates(gpu, ora, 8.0)
    assert n > 0
    # recall: every injected pulse is found near its DM and time
    for p in prm:
        near = gpu[(np.abs(gpu["dm"] - p["dm"]) < 2.0) & (np.abs(gpu["t_native"] - p["t0"]) < 64)]
        assert len(near) > 0, p


@pytest.mark.parametrize("kernel", ["default", "sb_factored"])
def test_fused_71_sb_sampled(fdd, kernel):
    import torch
    n_tab, n_chan, n_sb, n_out = 12, 1536, 71, synth.ARTS_CHUNK
    f = synth.channel_freqs(n_chan)
    ranges = [dict(dm0=0.0, ddm=0.2, n_dm=2048, downsamp=1, widths=[1, 2, 4, 8, 16, 32, 64])]
    n_in = n_out + int(oracle.delays(f, T_SAMP, 0.0, 0.2, 2048).max())
    prm = synth.random_pulses(3, 5, [0, 3, 5, 8, 11], 50.0, 400.0, [1, 4, 16], 10.0, 40.0, 300, n_out - 300)
    pulses = [dict(tab=p["tab"], start=p["t0"] + oracle.delays(f, T_SAMP, p["dm"], 1.0, 1)[0],
                   width=p["width"], amp=synth.pulse_amplitude(p["snr"], n_chan, p["width"])) for p in prm]
    x = synth.filterbank(3, n_tab, n_chan, n_in, pulses=pulses)
    sb = synth.sb_map_piecewise(3, n_sb, n_chan, n_tab).astype(np.int16)
    plan = fdd.Plan(n_tab, n_chan, n_sb, f, T_SAMP, ranges, 8.0, sb)
    if kernel == "sb_factored":
        v = [v for v in fdd.variants() if v["kind"] == 2 and v["bytes_per_sample"] == 1][0]
        plan.set_config(0, v["index"])
        assert plan.get_config(0)["work_ratio"] < 0.3
    res = plan.search(to_dev(x), n_in, n_out, cap=1 << 21, want_series=True)
    torch.cuda.synchronize()
    assert plan.status() == 0                     # no tile-copy wait gave up
    gpu, n = res.candidates()
    assert n == len(gpu)
    series = plan.series_views(res.series, n_out)[0]
    # every SB at DM 0 (all delays 0) is its per-channel TAB selection summed
    dm0 = np.zeros((n_sb, n_out), np.int64)
    for c in range(n_chan):
        dm0 += x[sb[:, c], c, :n_out]
    assert (series[:, 0].cpu().numpy() == dm0).all()
    rng = np.random.default_rng(0)
    for s in sorted(set([0, 70] + rng.integers(1, 70, size=1).tolist())):
        ora, os_ = oracle_candidate_superset(x, sb[s:s + 1], f, T_SAMP, ranges, 8.0, n_out, n_in,
                                             return_series=True)
        dms = rng.integers(0, 2048, size=64)
        assert (series[s, dms].cpu().numpy() == os_[0][0, dms]).all()
        ora = ora.copy()
        ora["sb"] = s
        compare_candidates(gpu[gpu["sb"] == s], ora, 8.0)


def test_overflow_reports_true_count(fdd):
    import torch
    x, f, ranges, n_in, n_out = tiny_config()
    plan = fdd.Plan(1, 128, 1, f, T_SAMP, ranges, 3.0, np.zeros((1, 128)))
    full = plan.search(to_dev(x), n_in, n_out, cap=1 << 20)
    torch.cuda.synchronize()
    all_c, n = full.candidates()
    assert n > 100
    small = plan.search(to_dev(x), n_in, n_out, cap=50)
    torch.cuda.synchronize()
    part, n2 = small.candidates()
    assert n2 == n and len(part) == 50
    full_set = set(map(tuple, np.stack([all_c["dm_index"], all_c["width_native"], all_c["t_native"]], 1).tolist()))
    assert set(map(tuple, np.stack([part["dm_index"], part["width_native"], part["t_native"]], 1).tolist())) <= full_set


def test_host_errors(fdd):
    import torch
    x, f, ranges, n_in, n_out = tiny_config()
    plan = fdd.Plan(1, 128, 1, f, T_SAMP, ranges, 8.0, np.zeros((1, 128)))
    dx = to_dev(x)
    with pytest.raises(fdd.FddError) as e:
        plan.search(dx, n_in - 1, n_out)
    assert e.value.code == -2
    odd = torch.zeros((1, 128, x.shape[2] + 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(fdd.FddError) as e:
        plan.search(odd, n_in, n_out)
    assert e.value.code == -4
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(fdd.FddError) as e:
        plan.search(dx, n_in, n_out, workspace=ws)
    assert e.value.code == -7


def test_repeat_is_deterministic(fdd):
    import torch
    x, f, ranges, n_in, n_out = tiny_config()
    plan = fdd.Plan(1, 128, 1, f, T_SAMP, ranges, 6.0, np.zeros((1, 128)))
    dx = to_dev(x)
    a = plan.search(dx, n_in, n_out, want_series=True)
    b = plan.search(dx, n_in, n_out, want_series=True)
    torch.cuda.synchronize()
    assert torch.equal(a.series, b.series)
    ca, na = a.candidates()
    cb, nb = b.candidates()
    assert na == nb and (ca == cb).all()


def segment_lengths(sb, cap):
    """Lengths of the runs of channels on which every SB keeps one TAB, cut
    at `cap` channels (the SB-factored kernel's segments)."""
    n_chan = sb.shape[1]
    out, c0 = [], 0
    for c in range(1, n_chan + 1):
        if c == n_chan or c - c0 == cap or (sb[:, c] != sb[:, c - 1]).any():
            out.append(c - c0)
            c0 = c
    return out


def segments_whole_groups(sb, G):
    """True if every SB-factored segment (cut at 16 channels) is a run of
    whole channel groups of size G (the pattern-factored part's condition)."""
    n_chan, c0 = sb.shape[1], 0
    for n in segment_lengths(sb, 16):
        end = c0 + n
        if c0 % G or (end % G and end != n_chan):
            return False
        c0 = end
    return True


def variant_case():
    rng = np.random.default_rng(42)
    n_tab, n_chan, n_sb, n_out = 2, 70, 3, 1500
    f = synth.channel_freqs(n_chan)
    ranges = [dict(dm0=0.0, ddm=1.5, n_dm=45, downsamp=1, widths=[1, 4, 16]),
              dict(dm0=67.5, ddm=3.0, n_dm=37, downsamp=2, widths=[1, 8])]
    need = max(int(oracle.delays(f, T_SAMP, r["dm0"], r["ddm"], r["n_dm"], r["downsamp"]).max())
               * r["downsamp"] + n_out for r in ranges) + 3
    x = synth.filterbank(77, n_tab, n_chan, need)
    sb = rng.integers(0, n_tab, size=(n_sb, n_chan)).astype(np.int16)
    return x, f, ranges, sb, need, n_out


@pytest.fixture(scope="module")
def variant_oracle():
    x, f, ranges, sb, n_in, n_out = variant_case()
    ora, os_ = oracle_candidate_superset(x, sb, f, T_SAMP, ranges, 4.0, n_out, n_in, return_series=True)
    return ora, os_


def _all_variants():
    try:
        import paper_2205_12362_b300 as m
        return m.variants()
    except Exception:
        return []


@pytest.mark.parametrize("v", _all_variants(), ids=lambda v: "v%d_E%d_bd%d_t%d" % (
    v["index"], v["bytes_per_sample"], v["dm_per_block"], v["tile"]))
@pytest.mark.parametrize("cc", [0, 2, 8])
def test_every_kernel_variant(fdd, variant_oracle, v, cc):
    import torch
    if v.get("group", 0) and cc and (cc % v["group"] or cc < v["group"]):
        pytest.skip("stage size not a multiple of the channel group")
    x, f, ranges, sb, n_in, n_out = variant_case()
    if v["kind"] == 2 and cc and cc < max(segment_lengths(sb, 16)):
        pytest.skip("stage size shorter than a channel segment")
    if v["kind"] == 3 and not segments_whole_groups(sb, v["group"]):
        pytest.skip("segments of this SB table are not whole channel groups (test_sb_factored_pattern_part)")
    plan = fdd.Plan(x.shape[0], x.shape[1], sb.shape[0], f, T_SAMP, ranges, 4.0, sb)
    r = 0 if v["bytes_per_sample"] == 1 else 1
    try:
        plan.set_config(r, v["index"], cc)
    except fdd.FddError as e:
        # a given stage size may exceed a variant's shared memory on this steep-DM case (two
        # pattern-row buffers); the largest stage that fits (cc = 0) must always configure
        if cc == 0 or e.code != fdd.FDD_ERR_UNSUPPORTED:
            raise
        pytest.skip("stage size does not fit this variant's shared memory here")
    cfg = plan.get_config(r)
    assert cfg["variant"] == v["index"] and (cc == 0 or cfg["chan_per_stage"] == cc)
    res = plan.search(to_dev(x), n_in, n_out, want_series=True, cap=1 << 18)
    torch.cuda.synchronize()
    assert plan.status() == 0                     # no TMA tile wait gave up
    ora, os_ = variant_oracle
    g = plan.series_views(res.series, n_out)
    assert (g[r].cpu().numpy() == os_[r]).all()
    gpu, n = res.candidates()
    compare_candidates(gpu, ora, 4.0)


def test_wrong_width_variant_rejected(fdd):
    x, f, ranges, sb, n_in, n_out = variant_case()
    plan = fdd.Plan(x.shape[0], x.shape[1], sb.shape[0], f, T_SAMP, ranges, 4.0, sb)
    v16 = [v for v in fdd.variants() if v["bytes_per_sample"] == 2][0]
    with pytest.raises(fdd.FddError):
        plan.set_config(0, v16["index"])
    assert plan.get_config(0)["variant"] >= 0


def test_autotune_then_parity(fdd, variant_oracle):
    import torch
    x, f, ranges, sb, n_in, n_out = variant_case()
    plan = fdd.Plan(x.shape[0], x.shape[1], sb.shape[0], f, T_SAMP, ranges, 4.0, sb)
    dx = to_dev(x)
    cfgs = plan.autotune(dx, n_in, n_out, reps=2)
    assert all(c["tuned_ms"] > 0 for c in cfgs)
    res = plan.search(dx, n_in, n_out, want_series=True, cap=1 << 18)
    torch.cuda.synchronize()
    ora, os_ = variant_oracle
    for g, o in zip(plan.series_views(res.series, n_out), os_):
        assert (g.cpu().numpy() == o).all()
    gpu, n = res.candidates()
    compare_candidates(gpu, ora, 4.0)


# ---------------------------------------------------------------- batched search
def batch_case(seed, n_in_extra):
    rng = np.random.default_rng(seed)
    n_tab, n_chan, n_sb, n_out = 3, 96, 4, 2100
    f = synth.channel_freqs(n_chan)
    ranges = [dict(dm0=0.0, ddm=1.0, n_dm=70, downsamp=1, widths=[1, 2, 8]),
              dict(dm0=70.0, ddm=2.0, n_dm=33, downsamp=2, widths=[1, 4]),
              dict(dm0=136.0, ddm=4.0, n_dm=20, downsamp=4, widths=[2]),
              dict(dm0=216.0, ddm=8.0, n_dm=9, downsamp=8, widths=[1, 3])]
    need = max(int(oracle.delays(f, T_SAMP, r["dm0"], r["ddm"], r["n_dm"], r["downsamp"]).max())
               * r["downsamp"] + n_out for r in ranges)
    sb = np.random.default_rng(99).integers(0, n_tab, size=(n_sb, n_chan)).astype(np.int16)
    n_in = need + n_in_extra
    start = 800 + oracle.delays(f, T_SAMP, 40.0 + 3 * seed, 1.0, 1)[0]
    x = synth.filterbank(300 + seed, n_tab, n_chan, n_in, pulses=[dict(tab=seed % n_tab, start=start, width=4,
                                                                       amp=22.0)])
    return x, f, ranges, sb, n_in, n_out


# 1000: FDD_BATCH_SB_FACTORED, 1001: FDD_BATCH_SB_PERSISTENT (one launch for every job, range and slab)
@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 1000, 1001])
def test_batched_equals_single(fdd, variant):
    import torch
    cases = [batch_case(s, e) for s, e in [(0, 0), (1, 7), (2, 33)]]
    x0, f, ranges, sb, _, n_out = cases[0]
    plan = fdd.Plan(x0.shape[0], x0.shape[1], sb.shape[0], f, T_SAMP, ranges, 5.0, sb)
    plan.batch_prepare(n_out, variant)
    assert plan.batch_config()["variant"] == variant
    jobs, singles = [], []
    for k, (x, _, _, _, n_in, _) in enumerate(cases):
        dx = to_dev(x)
        jobs.append(plan.make_job(dx, n_in, n_out, t_offset=1000 * k, cap=1 << 16, want_series=(k != 1)))
        singles.append(plan.search(dx, n_in, n_out, t_offset=1000 * k, cap=1 << 16, want_series=True))
    res = plan.search_batch(jobs, n_out)
    torch.cuda.synchronize()
    for k, (r, s1) in enumerate(zip(res, singles)):
        if r.series is not None:
            assert torch.equal(r.series, s1.series), "job %d series" % k
        cb, nb = r.candidates()
        cs, ns = s1.candidates()
        assert nb == ns and (cb == cs).all(), "job %d candidates" % k
    # and against the oracle for one job
    x, f, ranges, sb, n_in, n_out = cases[2]
    ora, os_ = oracle_candidate_superset(x, sb, f, T_SAMP, ranges, 5.0, n_out, n_in, t_offset=2000,
                                         return_series=True)
    for g, o in zip(plan.series_views(res[2].series, n_out), os_):
        assert (g.cpu().numpy() == o).all()
    compare_candidates(res[2].candidates()[0], ora, 5.0)


@pytest.mark.parametrize("variant", [-1, 1000, 1001])
def test_batch_graph_and_update(fdd, variant):
    import torch
    cases = [batch_case(s, 0) for s in (3, 4)]
    x0, f, ranges, sb, n_in, n_out = cases[0]
    plan = fdd.Plan(x0.shape[0], x0.shape[1], sb.shape[0], f, T_SAMP, ranges, 5.0, sb)
    plan.batch_prepare(n_out, variant)
    dxs = [to_dev(c[0]) for c in cases]
    jobs = [plan.make_job(dx, c[4], n_out, t_offset=7, want_series=True) for dx, c in zip(dxs, cases)]
    ref = [plan.search(dx, c[4], n_out, t_offset=7, want_series=True) for dx, c in zip(dxs, cases)]
    g = fdd.Graph(plan, jobs, n_out)
    for _ in range(2):
        g.launch()
        torch.cuda.synchronize()
        for j, r in zip(jobs, ref):
            assert torch.equal(j.series, r.series)
            a, na = j.result().candidates()
            b, nb = r.candidates()
            assert na == nb and (a == b).all()
    # swap the inputs and shift the time offsets through an update
    jobs2 = [plan.make_job(dx, c[4], n_out, t_offset=5000, want_series=True) for dx, c in zip(dxs[::-1], cases[::-1])]
    g.update(jobs2)
    g.launch()
    torch.cuda.synchronize()
    for j, r in zip(jobs2, ref[::-1]):
        assert torch.equal(j.series, r.series)
        a, na = j.result().candidates()
        b, nb = r.candidates()
        assert na == nb
        assert (a["t_native"] - b["t_native"] == 5000 - 7).all()
    g.close()


def test_sb_factored_batches_on_two_streams(fdd):
    """SB-factored batches of one four-range plan run their ranges on two forked stream lanes (a
    side-stream pair per caller stream): two batches enqueued back to back on two different streams,
    with no synchronisation between them, each equal the single searches of their jobs; graphs
    created and destroyed repeatedly (each frees its capture stream's lanes) keep giving the same
    results."""
    import torch
    cases = [batch_case(s, 0) for s in (5, 6, 7, 8)]
    x0, f, ranges, sb, n_in, n_out = cases[0]
    plan = fdd.Plan(x0.shape[0], x0.shape[1], sb.shape[0], f, T_SAMP, ranges, 5.0, sb)
    plan.batch_prepare(n_out, fdd.FDD_BATCH_SB_FACTORED)
    dxs = [to_dev(c[0]) for c in cases]
    ref = [plan.search(dx, c[4], n_out, t_offset=11 * k, want_series=True)
           for k, (dx, c) in enumerate(zip(dxs, cases))]
    torch.cuda.synchronize()
    jobs = [plan.make_job(dx, c[4], n_out, t_offset=11 * k, want_series=True)
            for k, (dx, c) in enumerate(zip(dxs, cases))]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    for _ in range(2):
        for j in jobs:
            j.series.fill_(-1)
        torch.cuda.synchronize()
        plan.search_batch(jobs[:2], n_out, stream=s1)
        plan.search_batch(jobs[2:], n_out, stream=s2)
        torch.cuda.synchronize()
        assert plan.status() == 0
        for j, r in zip(jobs, ref):
            assert torch.equal(j.series, r.series)
            a, na = j.result().candidates()
            b, nb = r.candidates()
            assert na == nb and (a == b).all()
    for _ in range(6):
        g = fdd.Graph(plan, jobs[1:3], n_out)
        jobs[1].series.fill_(-1)
        jobs[2].series.fill_(-1)
        g.launch()
        torch.cuda.synchronize()
        g.close()
        for j, r in zip(jobs[1:3], ref[1:3]):
            assert torch.equal(j.series, r.series)


def test_batch_autotune_keeps_parity(fdd):
    import torch
    x, f, ranges, sb, n_in, n_out = batch_case(5, 0)
    plan = fdd.Plan(x.shape[0], x.shape[1], sb.shape[0], f, T_SAMP, ranges, 5.0, sb)
    dx = to_dev(x)
    job = plan.make_job(dx, n_in, n_out, want_series=True)
    cfg = plan.batch_autotune([job], n_out, reps=1)
    assert cfg["tuned_ms"] > 0 and cfg["grid"] > 0
    res = plan.search_batch([job], n_out)[0]
    ref = plan.search(dx, n_in, n_out, want_series=True)
    torch.cuda.synchronize()
    assert torch.equal(res.series, ref.series)


@pytest.mark.parametrize("variant", [-1, 1000, 1001])
def test_four_range_71_sb_batched_sampled(fdd, variant):
    """The 4-range 0-5000 plan over 71 SBs at full size, in the batched
    launch configuration the benchmark and serving loop use; one SB checked
    against the oracle on sampled series of every range and on all its
    candidates."""
    import torch
    n_tab, n_chan, n_sb, n_out = 12, 1536, 71, synth.ARTS_CHUNK
    f = synth.channel_freqs(n_chan)
    W = [1, 2, 4, 8, 16, 32, 64]
    ranges = [dict(dm0=0.0, ddm=0.2, n_dm=2048, downsamp=1, widths=W),
              dict(dm0=409.6, ddm=0.8, n_dm=1024, downsamp=2, widths=W),
              dict(dm0=1228.8, ddm=1.6, n_dm=1024, downsamp=4, widths=W),
              dict(dm0=2867.2, ddm=3.2, n_dm=667, downsamp=8, widths=W)]
    sb = synth.sb_map_piecewise(4, n_sb, n_chan, n_tab).astype(np.int16)
    plan = fdd.Plan(n_tab, n_chan, n_sb, f, T_SAMP, ranges, 8.0, sb)
    n_in = n_out + plan.max_delay
    s_chk = 17
    prm = [dict(dm=300.0, t0=3000, width=4, snr=30.0), dict(dm=900.0, t0=6000, width=8, snr=40.0),
           dict(dm=2000.0, t0=8000, width=16, snr=40.0), dict(dm=4000.0, t0=9000, width=32, snr=45.0)]
    tabs_of_sb = sorted(set(sb[s_chk].tolist()))
    pulses = [dict(tab=t, start=p["t0"] + oracle.delays(f, T_SAMP, p["dm"], 1.0, 1)[0], width=p["width"],
                   amp=synth.pulse_amplitude(p["snr"], n_chan, p["width"])) for p in prm for t in tabs_of_sb]
    x = synth.filterbank(4, n_tab, n_chan, n_in, pulses=pulses)
    dx = to_dev(x)
    plan.batch_prepare(n_out, variant)
    job = plan.make_job(dx, n_in, n_out, cap=1 << 22, want_series=True)
    res = plan.search_batch([job], n_out)[0]
    torch.cuda.synchronize()
    gpu, n = res.candidates()
    assert n == len(gpu)
    views = plan.series_views(res.series, n_out)
    ora, os_ = oracle_candidate_superset(x, sb[s_chk:s_chk + 1], f, T_SAMP, ranges, 8.0, n_out, n_in,
                                         return_series=True)
    rng = np.random.default_rng(4)
    for r in range(4):
        dms = rng.integers(0, ranges[r]["n_dm"], size=32)
        assert (views[r][s_chk, dms].cpu().numpy() == os_[r][0, dms]).all(), "range %d" % r
    ora = ora.copy()
    ora["sb"] = s_chk
    compare_candidates(gpu[gpu["sb"] == s_chk], ora, 8.0)
    for p in prm:   # every injected pulse is found in the checked SB
        near = gpu[(gpu["sb"] == s_chk) & (np.abs(gpu["dm"] - p["dm"]) < 0.02 * p["dm"] + 3)
                   & (np.abs(gpu["t_native"] - p["t0"]) < 4 * p["width"] + 16)]
        assert len(near) > 0, p


def test_sb_factored_piecewise_slabs(fdd):
    """SB-factored kernels on a piecewise TAB table (16-channel segments) with
    the partial-sum scratch capped so each range runs in several DM slabs;
    every series bit-exact, candidates equal, for every SB-factored variant."""
    import torch
    n_tab, n_chan, n_sb, n_out = 6, 168, 20, 2000
    f = synth.channel_freqs(n_chan)
    ranges = [dict(dm0=0.0, ddm=1.0, n_dm=100, downsamp=1, widths=[1, 2, 8]),
              dict(dm0=100.0, ddm=4.0, n_dm=41, downsamp=4, widths=[1, 4])]
    sb = synth.sb_map_piecewise(9, n_sb, n_chan, n_tab).astype(np.int16)
    sb[3, 40:47] = (sb[3, 40:47] + 1) % n_tab        # a few segments shorter than 16
    n_in = max(int(oracle.delays(f, T_SAMP, r["dm0"], r["ddm"], r["n_dm"], r["downsamp"]).max())
               * r["downsamp"] + n_out for r in ranges) + 5
    pulses = [dict(tab=k % n_tab, start=t0 + oracle.delays(f, T_SAMP, dm, 1.0, 1)[0], width=w, amp=40.0)
              for k, (t0, dm, w) in enumerate([(300, 30.0, 2), (900, 80.0, 4), (1500, 200.0, 8)])]
    x = synth.filterbank(21, n_tab, n_chan, n_in, pulses=pulses)
    ora, os_ = oracle_candidate_superset(x, sb, f, T_SAMP, ranges, 6.0, n_out, n_in, return_series=True)
    dx = to_dev(x)
    ran = set()
    for v in [v for v in fdd.variants() if v["kind"] == 2]:
        plan = fdd.Plan(n_tab, n_chan, n_sb, f, T_SAMP, ranges, 6.0, sb)
        plan.set_scratch_limit(1)                 # one DM block per slab
        r = 0 if v["bytes_per_sample"] == 1 else 1
        try:
            plan.set_config(r, v["index"])
        except fdd.FddError as e:
            assert e.code == -5                   # this DM step's staged rows do not fit the variant
            continue
        assert plan.get_config(r)["variant"] == v["index"]
        ran.add(v["bytes_per_sample"])
        res = plan.search(dx, n_in, n_out, want_series=True, cap=1 << 18)
        torch.cuda.synchronize()
        assert plan.status() == 0
        g = plan.series_views(res.series, n_out)
        for k in range(2):
            assert (g[k].cpu().numpy() == os_[k]).all(), (v, k)
        gpu, n = res.candidates()
        compare_candidates(gpu, ora, 6.0)
    assert ran == {1, 2}


def test_sb_factored_pattern_part(fdd):
    """SB-factored dedispersion whose segment partials come from the
    pattern-factored kernel in part mode (kind 3): piecewise TAB table with
    16- and 8-channel segments, the scratch capped to one DM block per slab
    (several slabs, a ragged last one), a ragged last tile; every series
    bit-exact against the oracle and candidates equal, for every such variant
    and stage size; the batched search in SB-factored mode equal to the single
    search with the same configuration."""
    import torch
    n_tab, n_chan, n_sb, n_out = 6, 176, 20, 1900
    f = synth.channel_freqs(n_chan)
    ranges = [dict(dm0=0.0, ddm=0.5, n_dm=150, downsamp=1, widths=[1, 2, 8]),
              dict(dm0=75.0, ddm=4.0, n_dm=30, downsamp=4, widths=[1, 4])]
    sb = synth.sb_map_piecewise(11, n_sb, n_chan, n_tab).astype(np.int16)
    sb[5, 32:40] = (sb[5, 32:40] + 1) % n_tab        # two 8-channel segments
    assert min(segment_lengths(sb, 16)) == 8
    n_in = max(int(oracle.delays(f, T_SAMP, r["dm0"], r["ddm"], r["n_dm"], r["downsamp"]).max())
               * r["downsamp"] + n_out for r in ranges) + 5
    pulses = [dict(tab=k % n_tab, start=t0 + oracle.delays(f, T_SAMP, dm, 1.0, 1)[0], width=w, amp=40.0)
              for k, (t0, dm, w) in enumerate([(300, 20.0, 2), (900, 60.0, 4), (1500, 150.0, 8)])]
    x = synth.filterbank(31, n_tab, n_chan, n_in, pulses=pulses)
    ora, os_ = oracle_candidate_superset(x, sb, f, T_SAMP, ranges, 6.0, n_out, n_in, return_series=True)
    dx = to_dev(x)
    vs = [v for v in fdd.variants() if v["kind"] == 3]
    assert vs and {v["group"] for v in vs} == {4, 8} and {v["bytes_per_sample"] for v in vs} == {1, 2}
    for v in vs:
        r = 0 if v["bytes_per_sample"] == 1 else 1   # raw rows, or the D = 4 range's 16-bit rows
        for cc in (0, 8, 16):
            plan = fdd.Plan(n_tab, n_chan, n_sb, f, T_SAMP, ranges, 6.0, sb)
            plan.set_scratch_limit(1)                 # one DM block per slab
            try:
                plan.set_config(r, v["index"], cc)
            except fdd.FddError as e:
                # the pattern rows of this steep DM step exceed shared memory at a given stage
                # size; the largest stage that fits (cc = 0) always configures
                assert cc != 0 and e.code == fdd.FDD_ERR_UNSUPPORTED
                continue
            cfg = plan.get_config(r)
            assert cfg["variant"] == v["index"] and (cc == 0 or cfg["chan_per_stage"] == cc)
            assert cfg["work_ratio"] < 0.5
            res = plan.search(dx, n_in, n_out, want_series=True, cap=1 << 18)
            torch.cuda.synchronize()
            assert plan.status() == 0
            g = plan.series_views(res.series, n_out)
            for k in range(2):
                assert (g[k].cpu().numpy() == os_[k]).all(), (v, cc, k)
            gpu, n = res.candidates()
            compare_candidates(gpu, ora, 6.0)
        plan = fdd.Plan(n_tab, n_chan, n_sb, f, T_SAMP, ranges, 6.0, sb)
        plan.set_scratch_limit(1)
        plan.set_config(r, v["index"], 0)
        res = plan.search(dx, n_in, n_out, want_series=True, cap=1 << 18)
        plan.batch_prepare(n_out, fdd.FDD_BATCH_SB_FACTORED)
        assert plan.get_config(r)["variant"] == v["index"]
        job = plan.make_job(dx, n_in, n_out, cap=1 << 18, want_series=True)
        bres = plan.search_batch([job], n_out)[0]
        torch.cuda.synchronize()
        assert plan.status() == 0
        assert torch.equal(bres.series, res.series)


def test_factored_downsampled_range(fdd):
    """The pattern-factored kernel on 16-bit (downsampled) rows: a single-SB
    plan whose D = 2 and D = 4 ranges run a pattern-factored variant built for
    16-bit samples (the lanes fold every 256 / D channels); every series
    bit-exact against the oracle, candidates equal."""
    import torch
    n_chan, n_out = 300, 1700
    f = synth.channel_freqs(n_chan)
    ranges = [dict(dm0=0.0, ddm=0.4, n_dm=70, downsamp=1, widths=[1, 4]),
              dict(dm0=28.0, ddm=0.8, n_dm=130, downsamp=2, widths=[1, 2, 8]),
              dict(dm0=132.0, ddm=1.6, n_dm=65, downsamp=4, widths=[1, 4])]
    n_in = max(int(oracle.delays(f, T_SAMP, r["dm0"], r["ddm"], r["n_dm"], r["downsamp"]).max())
               * r["downsamp"] + n_out for r in ranges) + 7
    pulses = [dict(tab=0, start=t0 + oracle.delays(f, T_SAMP, dm, 1.0, 1)[0], width=w, amp=12.0)
              for t0, dm, w in [(400, 60.0, 4), (1200, 170.0, 8)]]
    x = synth.filterbank(41, 1, n_chan, n_in, pulses=pulses)
    sb = np.zeros((1, n_chan), np.int16)
    ora, os_ = oracle_candidate_superset(x, sb, f, T_SAMP, ranges, 6.0, n_out, n_in, return_series=True)
    fv = [v for v in fdd.variants() if v["kind"] == 1 and v["group"] == 4 and v["dm_per_block"] == 64
          and v["tile"] == 256][0]
    plan = fdd.Plan(1, n_chan, 1, f, T_SAMP, ranges, 6.0, sb)
    for r in (1, 2):
        plan.set_config(r, fv["index"], 0)
        assert plan.get_config(r)["variant"] == fv["index"]
    res = plan.search(to_dev(x), n_in, n_out, want_series=True, cap=1 << 18)
    torch.cuda.synchronize()
    assert plan.status() == 0
    g = plan.series_views(res.series, n_out)
    for k in range(3):
        assert (g[k].cpu().numpy() == os_[k]).all(), k
    gpu, n = res.candidates()
    assert compare_candidates(gpu, ora, 6.0) > 0


def test_copy_rows(fdd):
    """fdd_copy_rows: rows from page-locked host memory into a strided
    device window and a device-to-device carry of row tails, equal to numpy
    slicing; ranges past a tensor are refused before the call."""
    import torch
    rows, L, pitch, keep = 37, 1000, 1312, 300
    host = torch.from_numpy(np.arange(rows * L, dtype=np.int64).astype(np.uint8).reshape(rows, L)).pin_memory()
    win = torch.zeros((rows, pitch), dtype=torch.uint8, device="cuda")
    fdd.copy_rows(win, keep, pitch, host, 0, L, L, rows)
    nxt = torch.zeros_like(win)
    fdd.copy_rows(nxt, 0, pitch, win, L, pitch, keep, rows)           # tail of each row to the head
    torch.cuda.synchronize()
    w = win.cpu().numpy()
    assert (w[:, keep:keep + L] == host.numpy()).all() and (w[:, :keep] == 0).all()
    assert (nxt.cpu().numpy()[:, :keep] == w[:, L:L + keep]).all()
    with pytest.raises(ValueError):
        fdd.copy_rows(win, keep + 100, pitch, host, 0, L, L, rows)    # last row past the window


def test_boxcar_width_sets(fdd):
    """Both boxcar forms: one warp per series (widths <= 512; 4, 8 and 16
    width slots) and one block per series (a width above 512), against the
    oracle, with chunk-crossing and series-end windows."""
    import torch
    n_chan, n_out = 96, 3100
    f = synth.channel_freqs(n_chan)
    ranges = [dict(dm0=0.0, ddm=2.0, n_dm=24, downsamp=1, widths=list(range(1, 11))),   # 10 widths
              dict(dm0=48.0, ddm=4.0, n_dm=12, downsamp=2, widths=[1, 600, 1024]),    # block path
              dict(dm0=96.0, ddm=8.0, n_dm=6, downsamp=4, widths=[3, 511])]           # 4 slots, wide
    n_in = max(int(oracle.delays(f, T_SAMP, r["dm0"], r["ddm"], r["n_dm"], r["downsamp"]).max())
               * r["downsamp"] + n_out for r in ranges) + 3
    pulses = [dict(tab=0, start=t0 + oracle.delays(f, T_SAMP, dm, 1.0, 1)[0], width=w, amp=30.0)
              for t0, dm, w in [(505, 20.0, 3), (1530, 70.0, 40), (2900, 120.0, 300)]]
    x = synth.filterbank(17, 1, n_chan, n_in, pulses=pulses)
    sb = np.zeros((1, n_chan), np.int16)
    plan, gpu, gs, ora, os_ = run_both(fdd, x, sb, f, ranges, 5.0, n_out, n_in)
    for g, o in zip(gs, os_):
        assert (g == o).all()
    assert compare_candidates(gpu, ora, 5.0) > 0


def test_boxcar_chunk_precheck(fdd):
    """The warp boxcar's chunk pre-check (widths up to 128: per 512-sample
    chunk, maxima of the 1-, 8- and 64-sample boxcars bound every width; a
    chunk whose bound stays under every threshold is skipped) against the
    oracle: power-of-two widths to 128 and a mixed set, pulses inside chunks,
    across a chunk boundary and at the series end, a low threshold so that
    noise chunks pass and fail the bound."""
    import torch
    n_chan, n_out = 96, 2900
    f = synth.channel_freqs(n_chan)
    ranges = [dict(dm0=0.0, ddm=2.0, n_dm=20, downsamp=1, widths=[1, 2, 4, 8, 16, 32, 64, 128]),
              dict(dm0=40.0, ddm=4.0, n_dm=12, downsamp=2, widths=[3, 6, 24, 72, 100])]
    n_in = max(int(oracle.delays(f, T_SAMP, r["dm0"], r["ddm"], r["n_dm"], r["downsamp"]).max())
               * r["downsamp"] + n_out for r in ranges) + 3
    pulses = [dict(tab=0, start=t0 + oracle.delays(f, T_SAMP, dm, 1.0, 1)[0], width=w, amp=a)
              for t0, dm, w, a in [(200, 10.0, 2, 40.0), (1000, 30.0, 60, 9.0), (2840, 60.0, 24, 14.0)]]
    x = synth.filterbank(23, 1, n_chan, n_in, pulses=pulses)
    sb = np.zeros((1, n_chan), np.int16)
    for thr in (4.5, 7.0):
        plan, gpu, gs, ora, os_ = run_both(fdd, x, sb, f, ranges, thr, n_out, n_in)
        for g, o in zip(gs, os_):
            assert (g == o).all()
        assert compare_candidates(gpu, ora, thr) > 0


def test_sb_factored_geometry_table(fdd):
    """SB-factored kernels on the SB table the library builds from the array
    geometry (Apertif-10, 71 SBs, TABs combined in 48-channel subbands):
    segments longer than 16 channels, sampled SBs against the oracle, DM 0 of
    every SB against a numpy gather-sum."""
    import torch
    n_tab, n_chan, n_sb, n_out = 12, 1536, 71, 2000
    f = synth.channel_freqs(n_chan)
    sb = fdd.sb_table(n_tab, n_sb, f, chan_per_subband=48)
    ranges = [dict(dm0=0.0, ddm=0.4, n_dm=96, downsamp=1, widths=[1, 4, 16])]
    n_in = n_out + int(oracle.delays(f, T_SAMP, 0.0, 0.4, 96).max()) + 3
    pulses = [dict(tab=k, start=900 + oracle.delays(f, T_SAMP, 20.0, 1.0, 1)[0], width=4, amp=12.0) for k in (0, 5, 11)]
    x = synth.filterbank(23, n_tab, n_chan, n_in, pulses=pulses)
    plan = fdd.Plan(n_tab, n_chan, n_sb, f, T_SAMP, ranges, 7.0, sb)
    cfg = None
    for v in [v for v in fdd.variants() if v["kind"] == 2 and v["bytes_per_sample"] == 1]:
        plan.set_config(0, v["index"])
        if plan.get_config(0)["chan_per_stage"] >= 48:   # a stage holds a whole 48-channel segment
            cfg = plan.get_config(0)
            break
    assert cfg is not None and abs(cfg["work_ratio"] - (12 * 1536 + 71 * 32) / (71 * 1536)) < 1e-6  # 32 segments
    res = plan.search(to_dev(x), n_in, n_out, want_series=True, cap=1 << 20)
    torch.cuda.synchronize()
    gpu, n = res.candidates()
    series = plan.series_views(res.series, n_out)[0]
    dm0 = np.zeros((n_sb, n_out), np.int64)
    for c in range(n_chan):
        dm0 += x[sb[:, c], c, :n_out]
    assert (series[:, 0].cpu().numpy() == dm0).all()
    for s in (0, 35, 52, 70):
        ora, os_ = oracle_candidate_superset(x, sb[s:s + 1], f, T_SAMP, ranges, 7.0, n_out, n_in, return_series=True)
        assert (series[s].cpu().numpy() == os_[0][0]).all()
        ora = ora.copy()
        ora["sb"] = s
        compare_candidates(gpu[gpu["sb"] == s], ora, 7.0)


@pytest.mark.parametrize("G,K", [(48, 32), (16, 16), (1, 32)])
def test_subband_two_step_matches_oracle(fdd, G, K):
    """Two-step subband dedispersion (approximate mode): series bit-exact and
    candidates equal to the oracle's two-step definition, on a multi-SB plan
    (SB map constant within 16-channel blocks) with a native and a
    downsampled range."""
    import torch
    n_tab, n_chan, n_sb, n_out = 3, 1536, 4, 3000
    f = synth.channel_freqs(n_chan)
    sb = synth.sb_map_piecewise(5, n_sb, n_chan, n_tab, sub=48).astype(np.int16)
    ranges = [dict(dm0=20.0, ddm=0.2, n_dm=128, downsamp=1, widths=[1, 2, 8]),
              dict(dm0=45.6, ddm=0.8, n_dm=64, downsamp=2, widths=[1, 4])]
    plan = fdd.Plan(n_tab, n_chan, n_sb, f, T_SAMP, ranges, 6.0, sb)
    exact_delay = plan.max_delay
    for r in range(2):
        plan.set_subband(r, G, K)
        assert plan.get_subband(r) == (G, K)
    assert plan.max_delay >= exact_delay - 2
    n_in = n_out + plan.max_delay + 5
    pulses = [dict(tab=k % n_tab, start=700 + 800 * k + oracle.delays(f, T_SAMP, dm, 1.0, 1)[0], width=w, amp=40.0)
              for k, (dm, w) in enumerate([(30.0, 4), (40.0, 2), (80.0, 8)])]
    x = synth.filterbank(31, n_tab, n_chan, n_in, pulses=pulses)
    res = plan.search(to_dev(x), n_in, n_out, want_series=True, cap=1 << 18)
    torch.cuda.synchronize()
    oranges = [dict(r, subband=(G, K)) for r in ranges]
    ora, os_ = oracle_candidate_superset(x, sb, f, T_SAMP, oranges, 6.0, n_out, n_in, return_series=True)
    g = plan.series_views(res.series, n_out)
    for k in range(2):
        assert (g[k].cpu().numpy() == os_[k]).all(), k
    gpu, n = res.candidates()
    assert compare_candidates(gpu, ora, 6.0) > 0
    # back to exact dedispersion
    for r in range(2):
        plan.set_subband(r, 0, 0)
    assert plan.max_delay == exact_delay


def test_subband_mode_refusals(fdd):
    n_chan = 96
    f = synth.channel_freqs(n_chan)
    sb = synth.sb_map_piecewise(2, 3, n_chan, 2, sub=16).astype(np.int16)
    ranges = [dict(dm0=0.0, ddm=1.0, n_dm=64, downsamp=1, widths=[1])]
    plan = fdd.Plan(2, n_chan, 3, f, T_SAMP, ranges, 6.0, sb)
    with pytest.raises(fdd.FddError):       # the SB map switches TAB inside a 32-channel subband
        plan.set_subband(0, 32, 32)
    plan.set_subband(0, 16, 32)
    with pytest.raises(fdd.FddError):       # batched searches stay exact
        plan.batch_prepare(1000)


def test_edge_cases_against_oracle(fdd):
    """Degenerate and limit shapes: one channel, one DM trial, an empty output,
    the largest downsampling factor, the channel and TAB limits."""
    import torch
    cases = []
    # one channel, one trial, widths longer than the series
    cases.append(dict(n_tab=1, n_chan=1, n_sb=1, n_out=300,
                      ranges=[dict(dm0=5.0, ddm=1.0, n_dm=1, downsamp=1, widths=[1, 7, 400])]))
    # the largest downsampling factor (257) next to a native range
    cases.append(dict(n_tab=2, n_chan=24, n_sb=2, n_out=257 * 9 + 5,
                      ranges=[dict(dm0=0.0, ddm=3.0, n_dm=5, downsamp=1, widths=[1, 2]),
                              dict(dm0=15.0, ddm=50.0, n_dm=3, downsamp=257, widths=[1, 2, 3])]))
    # the channel limit, few trials and samples
    cases.append(dict(n_tab=1, n_chan=16384, n_sb=1, n_out=600,
                      ranges=[dict(dm0=0.0, ddm=0.05, n_dm=4, downsamp=1, widths=[1, 4])]))
    # the TAB limit: 256 TABs, SBs picking across all of them
    cases.append(dict(n_tab=256, n_chan=32, n_sb=3, n_out=700,
                      ranges=[dict(dm0=0.0, ddm=2.0, n_dm=9, downsamp=1, widths=[1, 2])]))
    for k, cs in enumerate(cases):
        f = synth.channel_freqs(cs["n_chan"]) if cs["n_chan"] > 1 else np.array([1370.0])
        rng = np.random.default_rng(k)
        sb = rng.integers(0, cs["n_tab"], size=(cs["n_sb"], cs["n_chan"])).astype(np.int16)
        need = max(int(oracle.delays(f, T_SAMP, r["dm0"], r["ddm"], r["n_dm"], r["downsamp"]).max()) * r["downsamp"]
                   + (cs["n_out"] // r["downsamp"]) * r["downsamp"] for r in cs["ranges"])
        need += max(r["downsamp"] for r in cs["ranges"])
        x = synth.filterbank(40 + k, cs["n_tab"], cs["n_chan"], need)
        plan, gpu, gs, ora, os_ = run_both(fdd, x, sb, f, cs["ranges"], 4.0, cs["n_out"], need)
        for g, o in zip(gs, os_):
            assert (g == o).all(), k
        compare_candidates(gpu, ora, 4.0)
    # an empty output: nothing searched, nothing written
    f = synth.channel_freqs(16)
    plan = fdd.Plan(1, 16, 1, f, T_SAMP, [dict(dm0=0.0, ddm=1.0, n_dm=4, widths=[1])], 4.0, np.zeros((1, 16)))
    x = synth.filterbank(1, 1, 16, 200)
    res = plan.search(to_dev(x), 200, 0, cap=16)
    torch.cuda.synchronize()
    assert int(res.count.item()) == 0
