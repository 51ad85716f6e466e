"""The bounded wait of the TMA-staged kernels (tma.cuh): a wait on an
mbarrier that nothing arrives on gives up after its poll limit and the
kernel returns normally, and the device context stays usable -- a factored
search right after it still equals the oracle."""
import numpy as np
import pytest

import synth
from tests._cmp import compare_candidates
from tests.test_gpu_parity import fdd, tiny_config  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def test_wait_gives_up_and_context_stays_usable(fdd):
    assert fdd.selftest_bounded_wait(4096) is True
    assert fdd.selftest_bounded_wait(1) is True
    with pytest.raises(fdd.FddError):
        fdd.selftest_bounded_wait(0)
    x, f, ranges, n_in, n_out = tiny_config()
    sb = np.zeros((1, x.shape[1]), np.int16)
    # the factored kernel (TMA-staged, bounded waits) on the tiny workload
    v = [v for v in fdd.variants() if v["kind"] == 1 and v["group"] == 4][0]
    n_tab, n_chan, _ = x.shape
    plan = fdd.Plan(n_tab, n_chan, 1, f, synth.ARTS_T_SAMP_S, ranges, 8.0, sb)
    plan.set_config(0, v["index"])
    import torch
    from tests._cmp import oracle_candidate_superset
    res = plan.search(torch.from_numpy(np.ascontiguousarray(x)).cuda(), n_in, n_out, want_series=True)
    torch.cuda.synchronize()
    assert plan.status() == 0
    gpu, n = res.candidates()
    ora, os_ = oracle_candidate_superset(x, sb, f, synth.ARTS_T_SAMP_S, ranges, 8.0, n_out, n_in,
                                         return_series=True)
    assert (plan.series_views(res.series, n_out)[0].cpu().numpy() == os_[0]).all()
    assert compare_candidates(gpu, ora, 8.0) > 0
