"""CPU oracle for the ARTS single-pulse search hot path.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  It shares no code with
the CUDA library: the arithmetic lives in ``oracle.c`` (plain loops, FP64
delays and statistics, exact integer sums), reached here through ctypes.

Functions follow the paper's AMBER stages (Sec. "AMBER"): ``delays``
(Sec. "Dedispersion", cold-plasma law), ``downsample`` (Sec.
"Downsampling"), ``dedisperse`` (Sec. "Dedispersion" with the SB formation of
Sec. "Hierarchical beam forming"), ``stats`` / ``boxcar_snr`` (Sec.
"Integration", "S/N evaluation"), ``search`` (all stages plus Sec.
"Candidate selection") and ``cluster`` (the optional DM-width clustering of
Sec. "AMBER").  Pins for each live in tests/test_oracle_*.py.
"""
import ctypes
import os

import numpy as np

from .build import build as _build

_lib = None

CAND_DTYPE = np.dtype([("sb", np.int32), ("dm_index", np.int32), ("downsamp", np.int32),
                       ("width_native", np.int32), ("t_native", np.int64),
                       ("dm", np.float64), ("snr", np.float64)])
assert CAND_DTYPE.itemsize == 40

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double


def lib():
    global _lib
    if _lib is None:
        path = _build()
        L = ctypes.CDLL(path)
        L.oracle_set_threads.argtypes = [_I32]
        L.oracle_get_threads.restype = _I32
        L.oracle_delays.argtypes = [_I32, _P, _D, _D, _D, _I32, _I32, _P, _P]
        L.oracle_delays.restype = _I64
        L.oracle_downsample.argtypes = [_P, _I64, _I64, _I64, _I32, _P]
        L.oracle_dedisperse.argtypes = [_P, _I32, _I32, _I64, _P, _I32, _P, _I32, _I64, _P]
        L.oracle_stats.argtypes = [_P, _I64, _P, _P]
        L.oracle_boxcar_snr.argtypes = [_P, _I64, _I32, _D, _D, _P]
        L.oracle_search.argtypes = [_P, _I32, _I32, _I64, _I64, _P, _I32, _P, _D, _I32,
                                    _P, _P, _P, _P, _P, _P, _D, _I64, _I64, _P, _I64, _P, _P, _P, _I32]
        L.oracle_search.restype = _I64
        L.oracle_cluster.argtypes = [_P, _I64, _P]
        L.oracle_rfi_clean.argtypes = [_P, _I32, _I32, _I64, _I64, _D, _I32, _D, _I32, _P, _P]
        L.oracle_cluster.restype = _I64
        L.oracle_rfi_clean.restype = _I64
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(lib().oracle_get_threads())


def delays(freq_mhz, t_samp_s, dm0, ddm, n_dm, downsamp=1, return_ties=False):
    """Integer delay table int64[n_dm][n_chan] in units of downsamp*t_samp."""
    f = np.ascontiguousarray(freq_mhz, dtype=np.float64)
    out = np.empty((int(n_dm), f.size), dtype=np.int64)
    ties = np.zeros(1, dtype=np.int64)
    lib().oracle_delays(f.size, _ptr(f), float(t_samp_s), float(dm0), float(ddm), int(n_dm),
                        int(downsamp), _ptr(out), _ptr(ties))
    return (out, int(ties[0])) if return_ties else out


def downsample(x, downsamp, n_in=None):
    """x: uint8[rows][pitch] (or [.., pitch]); returns uint32[rows][n_in // D]."""
    x = np.ascontiguousarray(x, dtype=np.uint8)
    shape = x.shape
    pitch = shape[-1]
    rows = int(np.prod(shape[:-1])) if len(shape) > 1 else 1
    n_in = pitch if n_in is None else int(n_in)
    n_y = n_in // int(downsamp)
    y = np.empty((rows, n_y), dtype=np.uint32)
    lib().oracle_downsample(_ptr(x), rows, n_in, pitch, int(downsamp), _ptr(y))
    return y.reshape(tuple(shape[:-1]) + (n_y,))


def dedisperse(y, sb_map, delay_table, n_out):
    """y: uint32[n_tab][n_chan][n_y]; sb_map int[n_sb][n_chan];
    delay_table int64[n_dm][n_chan]; returns int64[n_sb][n_dm][n_out]."""
    y = np.ascontiguousarray(y, dtype=np.uint32)
    n_tab, n_chan, n_y = y.shape
    m = np.ascontiguousarray(sb_map, dtype=np.int32)
    d = np.ascontiguousarray(delay_table, dtype=np.int64)
    n_sb, n_dm = m.shape[0], d.shape[0]
    if n_out + int(d.max(initial=0)) > n_y:
        raise ValueError("input too short for this delay table")
    if m.min(initial=0) < 0 or m.max(initial=0) >= n_tab:
        raise ValueError("sb_map out of range")
    out = np.empty((n_sb, n_dm, int(n_out)), dtype=np.int64)
    lib().oracle_dedisperse(_ptr(y), n_tab, n_chan, n_y, _ptr(m), n_sb, _ptr(d), n_dm,
                            int(n_out), _ptr(out))
    return out


def stats(series):
    s = np.ascontiguousarray(series, dtype=np.int64)
    mu = np.zeros(1)
    sd = np.zeros(1)
    lib().oracle_stats(_ptr(s), s.size, _ptr(mu), _ptr(sd))
    return float(mu[0]), float(sd[0])


def boxcar_snr(series, width, mean, std):
    s = np.ascontiguousarray(series, dtype=np.int64)
    n = s.size - int(width) + 1
    out = np.empty(max(n, 0), dtype=np.float64)
    if n > 0:
        lib().oracle_boxcar_snr(_ptr(s), s.size, int(width), float(mean), float(std), _ptr(out))
    return out


def window_bins(t_offset_native, n_out, downsamp):
    """(phase, n_r) of a window whose input starts at stream sample
    t_offset_native, with bins aligned to stream sample 0 (oracle.c:
    oracle_search, bins_absolute): the bins that start in
    [t_offset, t_offset + n_out), read from input sample phase on."""
    j_first = -(-int(t_offset_native) // int(downsamp))
    j_end = -(-(int(t_offset_native) + int(n_out)) // int(downsamp))
    return j_first * int(downsamp) - int(t_offset_native), j_end - j_first


def search(x, sb_map, freq_mhz, t_samp_s, ranges, snr_thresh, n_out, n_in=None,
           t_offset_native=0, cap=1 << 20, return_series=False, bins_absolute=False):
    """Run the whole hot path on x: uint8[n_tab][n_chan][pitch].
    bins_absolute: x[..., 0] is stream sample t_offset_native and the
    downsampling bins are aligned to stream sample 0 (window_bins).

    ranges: list of dicts {dm0, ddm, n_dm, downsamp, widths} and optionally
    subband=(G, K): that range uses the two-step subband dedispersion of
    oracle.c (subbands of G channels, coarse DM blocks of K fine trials).
    Returns (candidates: structured array sorted by (sb, dm_index, width, t),
    total_count, series) where series is a list (one per range) of
    int64[n_sb][n_dm][n_out // D] or None.
    """
    x = np.ascontiguousarray(x, dtype=np.uint8)
    if x.ndim != 3:
        raise ValueError("x must be [n_tab][n_chan][pitch]")
    n_tab, n_chan, pitch = x.shape
    n_in = pitch if n_in is None else int(n_in)
    m = np.ascontiguousarray(sb_map, dtype=np.int32)
    if m.ndim != 2 or m.shape[1] != n_chan:
        raise ValueError("sb_map must be [n_sb][n_chan]")
    if m.min() < 0 or m.max() >= n_tab:
        raise ValueError("sb_map out of range")
    f = np.ascontiguousarray(freq_mhz, dtype=np.float64)
    dm0 = np.array([r["dm0"] for r in ranges], dtype=np.float64)
    ddm = np.array([r["ddm"] for r in ranges], dtype=np.float64)
    ndm = np.array([r["n_dm"] for r in ranges], dtype=np.int32)
    ds = np.array([r.get("downsamp", 1) for r in ranges], dtype=np.int32)
    nw = np.array([len(r["widths"]) for r in ranges], dtype=np.int32)
    ws = np.ascontiguousarray(np.concatenate([np.asarray(r["widths"], dtype=np.int32)
                                              for r in ranges]), dtype=np.int32)
    sub_g = np.array([int(r.get("subband", (0, 0))[0]) for r in ranges], dtype=np.int32)
    sub_k = np.array([int(r.get("subband", (0, 1))[1]) for r in ranges], dtype=np.int32)
    cands = np.zeros(max(int(cap), 1), dtype=CAND_DTYPE)
    series = None
    n_rs = [window_bins(t_offset_native, n_out, r.get("downsamp", 1))[1] if bins_absolute
            else int(n_out) // int(r.get("downsamp", 1)) for r in ranges]
    if return_series:
        total = sum(int(m.shape[0]) * int(r["n_dm"]) * nr for r, nr in zip(ranges, n_rs))
        series = np.empty(max(total, 1), dtype=np.int64)
    n = lib().oracle_search(_ptr(x), n_tab, n_chan, n_in, pitch, _ptr(m), m.shape[0], _ptr(f),
                            float(t_samp_s), len(ranges), _ptr(dm0), _ptr(ddm), _ptr(ndm),
                            _ptr(ds), _ptr(nw), _ptr(ws), float(snr_thresh), int(n_out),
                            int(t_offset_native), _ptr(cands), int(cap),
                            _ptr(series) if series is not None else None, _ptr(sub_g), _ptr(sub_k),
                            1 if bins_absolute else 0)
    if n == -1:
        raise ValueError("input too short for the DM plan")
    if n < 0:
        raise MemoryError("oracle allocation failed")
    got = cands[:min(int(n), int(cap))]
    got = np.sort(got, order=["sb", "dm_index", "width_native", "t_native"])
    out_series = None
    if series is not None:
        out_series = []
        off = 0
        for r, nr in zip(ranges, n_rs):
            k = m.shape[0] * int(r["n_dm"]) * nr
            out_series.append(series[off:off + k].reshape(m.shape[0], int(r["n_dm"]), nr))
            off += k
    return got, int(n), out_series


def cluster(cands):
    """DM-width clustering (oracle.c: oracle_cluster) of a structured array of
    candidates with the fields of CAND_DTYPE (any float type for dm/snr;
    records are taken in the given order, which decides exact ties).
    Returns the kept records as a CAND_DTYPE array sorted by (sb, dm_index,
    width_native, t_native)."""
    a = np.zeros(len(cands), dtype=CAND_DTYPE)
    for f in CAND_DTYPE.names:
        a[f] = cands[f]
    out = np.zeros(max(len(a), 1), dtype=CAND_DTYPE)
    n = lib().oracle_cluster(_ptr(a), len(a), _ptr(out))
    if n < 0:
        raise MemoryError("oracle allocation failed")
    return np.sort(out[:n], order=["sb", "dm_index", "width_native", "t_native"])


def sb_table(n_tab, n_sb, freq_mhz, f_max_mhz, alpha, b_max_m, b_cq_m, chan_per_subband=1):
    """TAB row per (SB, channel) from the array geometry (appendix "Synthesized
    beams"), written out in plain Python loops.  Returns int32[n_sb][n_chan].

    SB s has index n_SB = s - n_sb // 2.  At f_max it takes TAB n_TAB of grating
    response n_gr: n_TAB = n_SB mod N, minus N if above N/2 - 1, and
    n_gr = (n_SB - n_TAB) / N.  Going down in frequency, TAB k_j = n_TAB - j*sgn(n_SB)
    of the same grating response lands on the SB's position at
        f_j = f_max * (n_gr*B_max + k_j*alpha*B_cq) / (n_gr*B_max + n_TAB*alpha*B_cq),
    and the SB switches from k_j to k_{j+1} at 0.75 f_j + 0.25 f_{j+1} (even |n_SB|) or
    0.25 f_j + 0.75 f_{j+1} (odd |n_SB|).  A TAB index outside [-N/2, N/2 - 1] is the
    same TAB as the one N away (next grating response); the row is n_TAB + N/2 after
    that wrap.  With chan_per_subband = G > 1 every block of G channels takes the TAB
    chosen at the block's mean frequency."""
    freq = [float(f) for f in freq_mhz]
    n_chan = len(freq)
    N = int(n_tab)
    if N % 2:
        raise ValueError("the index convention needs an even number of TABs")
    out = np.zeros((n_sb, n_chan), dtype=np.int32)
    for s in range(n_sb):
        n_sb_idx = s - n_sb // 2
        n_t = n_sb_idx % N
        if n_t > N // 2 - 1:
            n_t -= N
        n_gr = (n_sb_idx - n_t) // N
        sgn = (n_sb_idx > 0) - (n_sb_idx < 0)
        w_hi, w_lo = (0.75, 0.25) if abs(n_sb_idx) % 2 == 0 else (0.25, 0.75)
        den = n_gr * b_max_m + n_t * alpha * b_cq_m

        def f_opt(j):
            return f_max_mhz * (n_gr * b_max_m + (n_t - j * sgn) * alpha * b_cq_m) / den

        def tab_at(f):
            if sgn == 0:
                return n_t
            j = 0
            while True:
                f_sw = w_hi * f_opt(j) + w_lo * f_opt(j + 1)
                if f >= f_sw or j > 4 * N + 64:
                    break
                j += 1
            return n_t - j * sgn

        def row(k):
            while k > N // 2 - 1:
                k -= N
            while k < -(N // 2):
                k += N
            return k + N // 2

        G = max(1, int(chan_per_subband))
        for b0 in range(0, n_chan, G):
            chans = range(b0, min(n_chan, b0 + G))
            f_c = sum(freq[c] for c in chans) / len(chans)
            r = row(tab_at(f_c))
            for c in chans:
                out[s, c] = r
    return out


def rfi_clean(x, n_in=None, time_thresh=4.0, time_iters=3, freq_thresh=4.0, freq_iters=3, return_near=False):
    """RFI mitigation (oracle.c: oracle_rfi_clean) of a copy of x
    (uint8[n_tab][n_chan][pitch]).  Returns (cleaned copy, time flags
    uint8[n_tab][n_in], channel flags uint8[n_tab][n_chan]), and with
    return_near=True also the number of flag decisions whose two sides were
    within 1e-9 (relative) of each other."""
    y = np.ascontiguousarray(x, dtype=np.uint8).copy()
    n_tab, n_chan, pitch = y.shape
    n_in = pitch if n_in is None else int(n_in)
    tf = np.zeros((n_tab, n_in), np.uint8)
    cf = np.zeros((n_tab, n_chan), np.uint8)
    near = lib().oracle_rfi_clean(_ptr(y), n_tab, n_chan, n_in, pitch, float(time_thresh), int(time_iters),
                                  float(freq_thresh), int(freq_iters), _ptr(tf), _ptr(cf))
    return (y, tf, cf, int(near)) if return_near else (y, tf, cf)
