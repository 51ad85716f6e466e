"""The allocation-free entry point, fdd_search_static, against fdd_search.

fdd_search_static serves callers that cannot allocate device memory while
they search (real-time threads, processes whose GPU memory is granted only at
start-up): its workspace is a fixed device array inside the library.  Its
results must equal those of fdd_search with a caller workspace -- series
bit-exact, candidates equal -- on two calls in a row (the array keeps the
previous call's contents, so the second call checks that whatever must start
at zero is cleared).  This file is collected last on purpose."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

T_SAMP = synth.ARTS_T_SAMP_S


def _case():
    n_tab, n_chan, n_sb, n_out = 2, 128, 3, 3000
    f = synth.channel_freqs(n_chan)
    ranges = [dict(dm0=0.0, ddm=1.0, n_dm=128, downsamp=1, widths=[1, 2, 4, 8]),
              dict(dm0=128.0, ddm=2.0, n_dm=64, downsamp=2, widths=[1, 4])]
    need = max(int(oracle.delays(f, T_SAMP, r["dm0"], r["ddm"], r["n_dm"], r["downsamp"]).max())
               * r["downsamp"] + n_out for r in ranges) + 5
    start = 900 + oracle.delays(f, T_SAMP, 70.0, 1.0, 1)[0]
    x = synth.filterbank(11, n_tab, n_chan, need, pulses=[dict(tab=1, start=start, width=4, amp=20.0)])
    sb = np.zeros((n_sb, n_chan), np.int16)
    sb[1] = 1
    sb[2, 32:96] = 1
    return x, f, ranges, sb, need, n_out


def test_static_search_matches_workspace_search():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_12362_b300 as fdd
    x, f, ranges, sb, n_in, n_out = _case()
    plan = fdd.Plan(x.shape[0], x.shape[1], sb.shape[0], f, T_SAMP, ranges, 6.0, sb)
    assert plan.workspace_size(n_in, n_out, with_series=True) <= plan.STATIC_SCRATCH_BYTES
    dx = torch.from_numpy(x).cuda()
    ref = plan.search(dx, n_in, n_out, cap=1 << 16, want_series=True)
    torch.cuda.synchronize()
    ref_c, ref_n = ref.candidates()
    assert ref_n > 0
    cap = 1 << 16
    # every output buffer exists before the calls, so any drop in free device
    # memory across a call is the library's
    bufs = [(torch.empty((cap, 8), dtype=torch.int32, device="cuda"), torch.zeros(1, dtype=torch.int64, device="cuda"),
             torch.full_like(ref.series, -1) if call == 1 else None) for call in range(2)]
    torch.cuda.synchronize()
    free = [torch.cuda.mem_get_info()[0]]
    outs = []
    for cands, count, series in bufs:
        outs.append(plan.search_static(dx, n_in, n_out, cands, count, series=series))
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
    for call, (out, (cands, count, series)) in enumerate(zip(outs, bufs)):
        got_c, got_n = out.candidates()
        assert got_n == ref_n, "call %d: %d candidates vs %d" % (call, got_n, ref_n)
        assert (got_c == ref_c).all(), "call %d: candidate records differ" % call
        if series is not None:
            assert torch.equal(series, ref.series), "call %d: series differ" % call
    # the first call on the device may load the library module that holds the
    # static array (committing it); the second allocates nothing
    print("free device memory drop: first call %d bytes, second call %d bytes" % (free[0] - free[1],
                                                                                    free[1] - free[2]))
    assert free[0] - free[1] >= 0
    assert free[2] == free[1], "the second call changed free device memory by %d bytes" % (free[1] - free[2])


def test_static_search_rejects_oversized_and_timed_plans():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_12362_b300 as fdd
    f = synth.channel_freqs(1536)
    ranges = [dict(dm0=0.0, ddm=0.2, n_dm=2048, downsamp=1, widths=[1])]
    plan = fdd.Plan(1, 1536, 1, f, T_SAMP, ranges, 8.0, np.zeros((1, 1536)))
    n_out = 12500
    n_in = n_out + plan.max_delay
    assert plan.workspace_size(n_in, n_out, with_series=True) > plan.STATIC_SCRATCH_BYTES
    dx = torch.zeros((1, 1536, synth.padded_pitch(n_in)), dtype=torch.uint8, device="cuda")
    cands = torch.empty((16, 8), dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(fdd.FddError) as e:
        plan.search_static(dx, n_in, n_out, cands, count)
    assert e.value.code == -7
    x, f2, r2, sb, n_in2, n_out2 = _case()
    small = fdd.Plan(x.shape[0], x.shape[1], sb.shape[0], f2, T_SAMP, r2, 6.0, sb)
    small.set_timing(True)
    with pytest.raises(fdd.FddError) as e:
        small.search_static(torch.from_numpy(x).cuda(), n_in2, n_out2, cands, count)
    assert e.value.code == -1
