"""The serving runtime (continuous batching of real-time chunks from many
beams): every window's candidates equal those of a stand-alone window search
(fdd_search_window) of the same input, whatever the mix of windows it was
batched with; sequence errors, backpressure and HBM admission are reported on
the host.

Tolerance: identical candidate records (both paths run the same exact-integer
kernels; S/N bit-identical)."""
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


def stream_case(n_beams=3, n_chunks=9, chunk=512, dm_scale=1.0):
    n_tab, n_chan, n_sb = 2, 64, 3
    f = synth.channel_freqs(n_chan)
    ranges = [dict(dm0=0.0, ddm=2.0 * dm_scale, n_dm=48, downsamp=1, widths=[1, 2, 4]),
              dict(dm0=96.0 * dm_scale, ddm=4.0 * dm_scale, n_dm=24, downsamp=2, widths=[1, 4])]
    sb = np.zeros((n_sb, n_chan), np.int16)
    sb[1] = 1
    sb[2, 16:48] = 1
    total = n_chunks * chunk
    streams = []
    for b in range(n_beams):
        pulses = []
        for k in range(3):
            t0 = 300 + 1100 * k + 137 * b
            dm = (20.0 + 30 * k + 7 * b) * dm_scale
            pulses.append(dict(tab=(b + k) % n_tab, start=t0 + oracle.delays(f, T_SAMP, dm, 1.0, 1)[0],
                               width=2 + k, amp=26.0))
        streams.append(synth.filterbank(1000 + b, n_tab, n_chan, total, pitch=total, pulses=pulses))
    return f, ranges, sb, streams, chunk, n_chunks


def chunk_of(x, k, chunk):
    assert (k + 1) * chunk <= x.shape[2]
    return np.ascontiguousarray(x[:, :, k * chunk:(k + 1) * chunk])


def standalone(fdd, plan, x, w, chunk, n_in, cap=1 << 15):
    import torch
    win = np.zeros((x.shape[0], x.shape[1], synth.padded_pitch(n_in)), np.uint8)
    seg = x[:, :, w * chunk:w * chunk + n_in]
    win[:, :, :seg.shape[2]] = seg
    r = plan.search_window(torch.from_numpy(win).cuda(), n_in, chunk, w * chunk, cap=cap)
    torch.cuda.synchronize()
    return r.candidates()[0], win


@pytest.mark.parametrize("max_slots,variant", [(1, -1), (2, -1), (0, -1), (0, 1000), (2, 1001)])
def test_serving_results_match_standalone(fdd, max_slots, variant):
    """variant: the batched mode the server's batches run in (-1 the
    default, 1000 SB-factored launches, 1001 one persistent SB-factored
    launch per batch)."""
    # the persistent SB-factored kernel stages at most 1024 row chunks per channel stage: at 64 channels
    # that is DM steps up to about 0.5 per trial at full rate and 1 at D = 2
    f, ranges, sb, streams, chunk, n_chunks = stream_case(dm_scale=0.25 if variant == 1001 else 1.0)
    plan = fdd.Plan(2, 64, 3, f, T_SAMP, ranges, 6.0, sb)
    if variant >= 0:
        plan.batch_prepare(chunk, variant)
    srv = fdd.Server(plan, len(streams), chunk, max_slots=max_slots, cap_per_window=1 << 14)
    if variant >= 0:
        assert plan.batch_config()["variant"] == variant
    info = srv.info()
    n_in = info["window_len"]
    assert max_slots == 0 or info["n_slots"] == max_slots
    results = {}
    # interleave beams; poll only every other round so that windows of several
    # beams wait together and go out in shared batches; retry on backpressure
    for k in range(n_chunks):
        for b, x in enumerate(streams):
            while True:
                code = srv.push(b, k, chunk_of(x, k, chunk))
                if code == 0:
                    break
                assert code == fdd.FDD_ERR_BUSY
                srv.drain()
        if k % 2:
            srv.poll()
    srv.drain()
    for r, c in srv.results():
        results[(r["beam"], r["window"])] = (r, c)
    cpw = -(-n_in // chunk)
    n_windows = n_chunks - cpw + 1
    assert len(results) == len(streams) * n_windows
    mixed = False
    for (b, w), (r, c) in sorted(results.items()):
        assert r["t0_native"] == w * chunk and r["n_cands"] == len(c)
        mixed |= r["batch_jobs"] > 1
        ref, _ = standalone(fdd, plan, streams[b], w, chunk, n_in)
        assert len(ref) == len(c) and (ref == c).all(), "beam %d window %d differs from the stand-alone search" % (b, w)
    if max_slots != 1:
        assert mixed, "no window was batched with another"
    # one window holding an injected pulse (beam 1: t0 = 1537) against the oracle
    b, w = 1, 3
    _, win = standalone(fdd, plan, streams[b], w, chunk, n_in)
    ora, _ = oracle_candidate_superset(win, sb, f, T_SAMP, ranges, 6.0, chunk, n_in, t_offset=w * chunk,
                                       bins_absolute=True)
    compare_candidates(results[(b, w)][1], ora, 6.0)
    assert len(results[(b, w)][1]) > 0
    assert sum(len(c) for _, c in results.values()) > 0
    srv.close()


def test_serving_sequence_backpressure_and_reset(fdd):
    f, ranges, sb, streams, chunk, n_chunks = stream_case(n_beams=1, n_chunks=20)
    plan = fdd.Plan(2, 64, 3, f, T_SAMP, ranges, 6.0, sb)
    srv = fdd.Server(plan, 1, chunk, max_slots=1)
    x = streams[0]
    assert srv.push(0, 1, chunk_of(x, 1, chunk)) == fdd.FDD_ERR_SEQUENCE      # chunk 0 missing
    cpw = -(-srv.info()["window_len"] // chunk)
    k = 0
    busy_seen = False
    while k < n_chunks:           # never poll: windows pile up until the beam reports backpressure
        code = srv.push(0, k, chunk_of(x, k, chunk))
        if code == fdd.FDD_ERR_BUSY:
            busy_seen = True
            break
        assert code == 0
        k += 1
    assert busy_seen and k == cpw + 1
    assert k + 3 + cpw <= n_chunks
    assert srv.push(0, k - 1, chunk_of(x, k - 1, chunk)) == fdd.FDD_ERR_SEQUENCE  # duplicate
    srv.drain()
    assert srv.push(0, k, chunk_of(x, k, chunk)) == 0
    # a gap: resynchronise at a later chunk; its windows start from there
    srv.drain()
    assert srv.reset_beam(0, k + 3) == 0
    for j in range(k + 3, k + 3 + cpw):
        assert srv.push(0, j, chunk_of(x, j, chunk)) == 0
    srv.drain()
    got = {r["window"] for r, _ in srv.results()}
    assert {0, 1, 2, k + 3} <= got
    srv.close()


def test_admission_refused_without_hbm(fdd):
    f, ranges, sb, streams, chunk, _ = stream_case(n_beams=1)
    plan = fdd.Plan(2, 64, 3, f, T_SAMP, ranges, 6.0, sb)
    with pytest.raises(fdd.FddError) as e:
        fdd.Server(plan, 4, chunk, hbm_budget_bytes=1 << 20)
    assert e.value.code == -3


def test_plain_per_sb_serving_matches_batched(fdd):
    """The plain per-SB serving path (one single-SB search per SB and window)
    returns, window by window, the batched path's candidate records."""
    f, ranges, sb, streams, chunk, n_chunks = stream_case(n_beams=2, n_chunks=7)
    plan = fdd.Plan(2, 64, 3, f, T_SAMP, ranges, 6.0, sb)
    sb_plans = [fdd.Plan(2, 64, 1, f, T_SAMP, ranges, 6.0, sb[s:s + 1]) for s in range(3)]
    out = {}
    for name, kw in (("batched", {}), ("plain", dict(sb_plans=sb_plans))):
        srv = fdd.Server(plan, len(streams), chunk, max_slots=2, cap_per_window=1 << 14, **kw)
        for k in range(n_chunks):
            for b, x in enumerate(streams):
                while srv.push(b, k, chunk_of(x, k, chunk)) == fdd.FDD_ERR_BUSY:
                    srv.drain()
            srv.poll()
        srv.drain()
        out[name] = {(r["beam"], r["window"]): (r, c) for r, c in srv.results()}
        srv.close()
    assert set(out["plain"]) == set(out["batched"]) and len(out["plain"]) > 0
    total = 0
    for key, (r, c) in out["batched"].items():
        rp, cp = out["plain"][key]
        assert rp["n_cands"] == r["n_cands"] and rp["batch_jobs"] == 1
        assert len(cp) == len(c) and (cp == c).all(), "window %r differs between the two paths" % (key,)
        total += len(c)
    assert total > 0
    with pytest.raises(fdd.FddError):      # one plan per SB is required
        fdd.Server(plan, 1, chunk, sb_plans=sb_plans[:2])
