"""Per-beam streaming search (fdd_stream_*): a beam's chunks pushed in order
from device memory; every window's candidates equal the oracle's search of
that window's samples (t_native absolute), the window schedule follows the
max delay, and sequence errors are refused on the host.

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
    n_in = chunk + md
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
                                           t_offset=t0)
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
