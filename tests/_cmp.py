"""Comparison helpers for CUDA-vs-oracle parity tests.

Tolerances (stated in the tests that use them):
  * dedispersed series: bit-exact (integer sums);
  * S/N: |gpu - oracle| <= 1e-4 * max(1, |oracle|);
  * candidate sets: equal after ignoring candidates whose oracle S/N lies
    within 1e-3 of the threshold (FP32 vs FP64 may decide those either way).
"""
import numpy as np

import oracle

SNR_RTOL = 1e-4
THR_BAND = 1e-3


def oracle_candidate_superset(x, sb_map, freqs, t_samp, ranges, thr, n_out, n_in, t_offset=0,
                              return_series=False, bins_absolute=False):
    """Oracle candidates with S/N > thr - THR_BAND (a superset of what the
    GPU may legally return).  bins_absolute: x is a window of a stream at
    t_offset with downsampling bins aligned to the stream."""
    got, n, series = oracle.search(x, sb_map, freqs, t_samp, ranges, thr - THR_BAND, n_out, n_in=n_in,
                                   t_offset_native=t_offset, cap=1 << 22, return_series=return_series,
                                   bins_absolute=bins_absolute)
    assert n == len(got), "oracle candidate buffer overflowed"
    return got, series


def compare_candidates(gpu, ora, thr):
    """gpu: CAND_DTYPE array (binding), ora: oracle superset array."""
    key = lambda a: list(zip(a["sb"].tolist(), a["dm_index"].tolist(), a["width_native"].tolist(),
                             a["t_native"].tolist()))
    o_map = {k: (snr, dm, ds) for k, snr, dm, ds in zip(key(ora), ora["snr"].tolist(), ora["dm"].tolist(),
                                                       ora["downsamp"].tolist())}
    g_keys = key(gpu)
    assert len(set(g_keys)) == len(g_keys), "duplicate GPU candidates"
    # every GPU candidate is an oracle candidate of the superset, with matching S/N
    for k, snr, dm, ds in zip(g_keys, gpu["snr"].tolist(), gpu["dm"].tolist(), gpu["downsamp"].tolist()):
        assert k in o_map, "GPU candidate %r not found by the oracle" % (k,)
        osnr, odm, ods = o_map[k]
        assert abs(snr - osnr) <= SNR_RTOL * max(1.0, abs(osnr)), (k, snr, osnr)
        assert ds == ods
        assert abs(dm - odm) <= 1e-6 * max(1.0, abs(odm)) + 1e-4
    # every oracle candidate clearly above threshold is on the GPU
    g_set = set(g_keys)
    missing = [k for k, (osnr, _, _) in o_map.items() if osnr > thr + THR_BAND and k not in g_set]
    assert not missing, "GPU missed %d oracle candidates, e.g. %r" % (len(missing), missing[:3])
    return len(g_keys)
