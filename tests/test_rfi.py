"""RFI mitigation on the GPU (fdd_rfi_clean) against the oracle's, exactly:
cleaned samples, time flags and channel flags.  The oracle takes sigma from
the exact integer numerator n*S2 - S1^2; the kernel uses S2/n - mu^2 in FP64.
The two agree except where a decision sits within ~1e-11 (relative) of the
threshold; the oracle counts decisions within 1e-9 of it, and the inputs here
have none, so every flag and sample must match."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

T = synth.ARTS_T_SAMP_S


@pytest.fixture(scope="module")
def fdd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_12362_b300 as m
    return m


def _rfi_input(seed, n_tab, n_chan, n_in, pitch):
    x = synth.filterbank(seed, n_tab, n_chan, n_in, pitch=pitch)
    rng = np.random.default_rng(seed)
    for tab in range(n_tab):
        for t0 in rng.integers(0, n_in, 3):          # broadband spikes of several strengths
            x[tab, :, t0] = np.minimum(255, x[tab, :, t0].astype(int) + int(rng.integers(6, 90)))
        c0 = int(rng.integers(0, n_chan))
        x[tab, c0, :n_in] = np.minimum(255, x[tab, c0, :n_in].astype(int) + 30)   # narrowband
        x[tab, (c0 + 7) % n_chan, :n_in] = 0                                      # dead channel
    return x


@pytest.mark.parametrize("tt,ft", [(4.0, 4.0), (3.0, 0.0), (0.0, 3.5), (5.0, 2.5)])
def test_rfi_matches_oracle(fdd, tt, ft):
    import torch
    n_tab, n_chan, n_in, pitch = 3, 200, 5001, 5024
    x = _rfi_input(7, n_tab, n_chan, n_in, pitch)
    want, tf_o, cf_o, near = oracle.rfi_clean(x, n_in=n_in, time_thresh=tt, freq_thresh=ft, return_near=True)
    print("flag decisions within 1e-9 of the threshold: %d" % near)
    assert near == 0
    d = torch.from_numpy(x).cuda()
    tf = torch.zeros((n_tab, n_in), dtype=torch.uint8, device="cuda")
    cf = torch.zeros((n_tab, n_chan), dtype=torch.uint8, device="cuda")
    fdd.rfi_clean(d, n_in, time_thresh=tt, freq_thresh=ft, time_flags=tf, chan_flags=cf)
    torch.cuda.synchronize()
    assert (tf.cpu().numpy() == tf_o).all()
    assert (cf.cpu().numpy() == cf_o).all()
    got = d.cpu().numpy()
    assert (got[:, :, :n_in] == want[:, :, :n_in]).all()
    assert (got[:, :, n_in:] == x[:, :, n_in:]).all()      # the pitch padding is not touched
    if tt > 0:
        assert tf_o.sum() >= n_tab      # the spikes were found
    if ft > 0:
        assert cf_o.sum() >= 2 * n_tab


def test_rfi_then_search_matches_oracle(fdd):
    import torch
    from tests._cmp import compare_candidates, oracle_candidate_superset
    n_chan, n_out = 256, 3000
    f = synth.channel_freqs(n_chan)
    ranges = [dict(dm0=0.0, ddm=1.0, n_dm=96, downsamp=1, widths=[1, 2, 4, 8])]
    n_in = n_out + int(oracle.delays(f, T, 0.0, 1.0, 96).max()) + 3
    pulses = [dict(tab=0, start=1500 + oracle.delays(f, T, 60.0, 1.0, 1)[0], width=4, amp=20.0)]
    x = synth.filterbank(8, 1, n_chan, n_in, pulses=pulses)
    x[0, :, 400] = 250                       # broadband RFI at DM 0 would swamp the low DMs
    x[0, 33] = np.minimum(255, x[0, 33].astype(int) + 40)
    clean, _, _ = oracle.rfi_clean(x, n_in=n_in)
    d = torch.from_numpy(x).cuda()
    fdd.rfi_clean(d, n_in)
    plan = fdd.Plan(1, n_chan, 1, f, T, ranges, 7.0, np.zeros((1, n_chan), np.int16))
    res = plan.search(d, n_in, n_out, cap=1 << 16)
    torch.cuda.synchronize()
    gpu, n = res.candidates()
    ora, _ = oracle_candidate_superset(clean, np.zeros((1, n_chan), np.int32), f, T, ranges, 7.0, n_out, n_in)
    assert compare_candidates(gpu, ora, 7.0) > 0
    assert not ((gpu["t_native"] <= 400) & (gpu["t_native"] >= 392) & (gpu["dm_index"] < 3)).any()
