"""B300-native hot path of the ARTS real-time single-pulse search.

A thin Python binding (ctypes) over the C ABI of ``libfdd.so`` (declared in
``include/fdd.h``).  Every stage of the search -- downsampling, synthesized-
beam gather + brute-force dedispersion, series statistics, boxcar S/N,
threshold and compaction -- runs in the library's CUDA kernels; this module
only marshals arguments.  PyTorch supplies device memory and streams.

There is no CPU fallback: if the library is missing, importing the binding
works but every call raises ``FddUnavailable``.
"""
import ctypes
import os
from dataclasses import dataclass

import numpy as np

from .build import LIB as _LIB_PATH

__all__ = ["Plan", "FddError", "FddUnavailable", "CAND_DTYPE", "decode_candidates", "downsample_u8",
           "library_path", "version", "variants", "Job", "Graph", "Server", "now"]

CAND_DTYPE = np.dtype([("sb", np.int32), ("dm_index", np.int32), ("downsamp", np.int32),
                       ("width_native", np.int32), ("t_native", np.int64), ("dm", np.float32),
                       ("snr", np.float32)])
assert CAND_DTYPE.itemsize == 32

FDD_MAX_WIDTHS = 16


class FddError(RuntimeError):
    def __init__(self, code, where):
        msg = "%s failed: %s (%d)" % (where, _lib_raw().fdd_error_string(code).decode(), code)
        detail = _lib_raw().fdd_last_error_message().decode()
        if detail:
            msg += ": " + detail
        super().__init__(msg)
        self.code = code


class FddUnavailable(RuntimeError):
    pass


class _Range(ctypes.Structure):
    _fields_ = [("dm0", ctypes.c_double), ("ddm", ctypes.c_double), ("n_dm", ctypes.c_int32),
                ("downsamp", ctypes.c_int32), ("n_width", ctypes.c_int32),
                ("widths", ctypes.POINTER(ctypes.c_int32))]


class KernelConfig(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("dm_per_block", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("chan_per_stage", ctypes.c_int32), ("threads", ctypes.c_int32), ("row_words", ctypes.c_int32),
                ("tuned_ms", ctypes.c_float), ("work_ratio", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class _Job(ctypes.Structure):
    _fields_ = [("d_tabs", ctypes.c_void_p), ("n_in", ctypes.c_int64), ("pitch", ctypes.c_int64),
                ("t_offset_native", ctypes.c_int64), ("d_workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("d_cands", ctypes.c_void_p), ("cap", ctypes.c_int64),
                ("d_count", ctypes.c_void_p), ("d_series", ctypes.c_void_p), ("bins_absolute", ctypes.c_int32)]


class _ServerDesc(ctypes.Structure):
    _fields_ = [("n_beams", ctypes.c_int32), ("chunk_len", ctypes.c_int64), ("max_slots", ctypes.c_int32),
                ("hbm_reserve_frac", ctypes.c_double), ("hbm_budget_bytes", ctypes.c_int64),
                ("cap_per_window", ctypes.c_int64)]


class _WindowResult(ctypes.Structure):
    _fields_ = [("beam", ctypes.c_int32), ("window", ctypes.c_int64), ("t0_native", ctypes.c_int64),
                ("t_arrival", ctypes.c_double), ("t_ready", ctypes.c_double), ("t_launch", ctypes.c_double),
                ("t_done", ctypes.c_double), ("n_cands", ctypes.c_int64), ("n_cands_kept", ctypes.c_int64),
                ("cand_offset", ctypes.c_int64), ("batch_jobs", ctypes.c_int32)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_int32), ("slots_busy", ctypes.c_int32), ("queued", ctypes.c_int32),
                ("max_queued", ctypes.c_int64), ("launched", ctypes.c_int64), ("done", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("window_len", ctypes.c_int64),
                ("ring_bytes_per_beam", ctypes.c_int64), ("slot_bytes", ctypes.c_int64)]


class _RfiDesc(ctypes.Structure):
    _fields_ = [("time_thresh", ctypes.c_double), ("time_iters", ctypes.c_int32),
                ("freq_thresh", ctypes.c_double), ("freq_iters", ctypes.c_int32)]


class _PlanDesc(ctypes.Structure):
    _fields_ = [("n_tab", ctypes.c_int32), ("n_chan", ctypes.c_int32), ("n_sb", ctypes.c_int32),
                ("chan_freq_mhz", ctypes.POINTER(ctypes.c_double)), ("t_samp_s", ctypes.c_double),
                ("n_range", ctypes.c_int32), ("ranges", ctypes.POINTER(_Range)),
                ("snr_thresh", ctypes.c_float)]


_lib = None
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_SZ = ctypes.c_size_t


def library_path():
    return _LIB_PATH


def _lib_raw():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise FddUnavailable("libfdd.so is not built (python -m paper_2205_12362_b300.build); "
                             "there is no CPU fallback")
    L = ctypes.CDLL(_LIB_PATH)
    L.fdd_version.restype = ctypes.c_char_p
    L.fdd_error_string.restype = ctypes.c_char_p
    L.fdd_error_string.argtypes = [ctypes.c_int]
    L.fdd_last_error_message.restype = ctypes.c_char_p
    L.fdd_plan_create.argtypes = [ctypes.POINTER(_PlanDesc), _P, ctypes.POINTER(_P)]
    L.fdd_plan_destroy.argtypes = [_P]
    L.fdd_plan_max_delay.argtypes = [_P, ctypes.POINTER(_I64)]
    L.fdd_plan_total_dms.argtypes = [_P, ctypes.POINTER(_I64)]
    L.fdd_plan_delays.argtypes = [_P, _I32, _P]
    L.fdd_workspace_size.argtypes = [_P, _I64, _I64, _I32, ctypes.POINTER(_SZ)]
    L.fdd_series_size.argtypes = [_P, _I64, ctypes.POINTER(_SZ)]
    L.fdd_search.argtypes = [_P, _P, _I64, _I64, _I64, _I64, _P, _SZ, _P, _I64, _P, _P, _P]
    L.fdd_search_window.argtypes = [_P, _P, _I64, _I64, _I64, _I64, _P, _SZ, _P, _I64, _P, _P, _P]
    L.fdd_window_sizes.argtypes = [_P, _I64, ctypes.POINTER(_I64), ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)]
    L.fdd_downsample_u8.argtypes = [_P, _I64, _I64, _I64, _I32, _P, _I64, _P]
    L.fdd_copy_rows.argtypes = [_P, _I64, _P, _I64, _I64, _I64, _P]
    L.fdd_plan_set_timing.argtypes = [_P, _I32]
    L.fdd_num_variants.argtypes = [ctypes.POINTER(_I32)]
    L.fdd_variant_info.argtypes = [_I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                                   ctypes.POINTER(_I32), ctypes.POINTER(_I32)]
    L.fdd_plan_get_config.argtypes = [_P, _I32, ctypes.POINTER(KernelConfig)]
    L.fdd_plan_set_config.argtypes = [_P, _I32, _I32, _I32]
    L.fdd_plan_autotune.argtypes = [_P, _P, _I64, _I64, _I64, _P, _SZ, _I32, _P]
    L.fdd_batch_prepare.argtypes = [_P, _I64, _I32]
    L.fdd_search_batch.argtypes = [_P, ctypes.POINTER(_Job), _I32, _I64, _P]
    L.fdd_batch_autotune.argtypes = [_P, ctypes.POINTER(_Job), _I32, _I64, _I32, _P]
    L.fdd_batch_config.argtypes = [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                                   ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_float)]
    L.fdd_graph_create.argtypes = [_P, ctypes.POINTER(_Job), _I32, _I64, ctypes.POINTER(_P)]
    L.fdd_graph_update.argtypes = [_P, ctypes.POINTER(_Job), _I32]
    L.fdd_graph_launch.argtypes = [_P, _P]
    L.fdd_graph_destroy.argtypes = [_P]
    L.fdd_now.restype = ctypes.c_double
    L.fdd_server_create.argtypes = [_P, ctypes.POINTER(_ServerDesc), ctypes.POINTER(_P)]
    L.fdd_server_destroy.argtypes = [_P]
    L.fdd_server_set_plain.argtypes = [_P, _P, _I32]
    L.fdd_server_push.argtypes = [_P, _I32, _I64, _P, ctypes.c_double]
    L.fdd_server_reset_beam.argtypes = [_P, _I32, _I64]
    L.fdd_server_poll.argtypes = [_P]
    L.fdd_server_drain.argtypes = [_P]
    L.fdd_server_results.argtypes = [_P, ctypes.POINTER(_WindowResult), _I32, _P, _I64, ctypes.POINTER(_I32),
                                     ctypes.POINTER(_I64)]
    L.fdd_server_info.argtypes = [_P, ctypes.POINTER(_ServerStats)]
    L.fdd_fact_tables_host.argtypes = [ctypes.POINTER(_PlanDesc), _P, _I32, _I32, _I32, _P, _P, _P, _P, _P, _P, _P]
    L.fdd_search_static.argtypes = [_P, _P, _I64, _I64, _I64, _I64, _P, _I64, _P, _P, _P]
    L.fdd_plan_stage_times.argtypes = [_P, _I32, _P, _P, _P, ctypes.POINTER(_I32)]
    L.fdd_plan_info.argtypes = [_P, _I64, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]
    L.fdd_stream_open.argtypes = [_P, _I32, _I64, _I64, ctypes.POINTER(_P)]
    L.fdd_stream_push.argtypes = [_P, _P, _I64, _I64, _P]
    L.fdd_stream_results.argtypes = [_P, _P, _I64, _P, ctypes.POINTER(_I64)]
    L.fdd_stream_close.argtypes = [_P]
    L.fdd_sort_candidates.argtypes = [_P, _I64]
    L.fdd_variant_kind.argtypes = [_I32, ctypes.POINTER(_I32)]
    L.fdd_plan_set_scratch_limit.argtypes = [_P, _I64]
    L.fdd_plan_last_launches.argtypes = [_P, ctypes.POINTER(_I64)]
    L.fdd_plan_status.argtypes = [_P, ctypes.POINTER(_I32), _I32]
    L.fdd_selftest_bounded_wait.argtypes = [_I32, ctypes.POINTER(_I32)]
    L.fdd_probe_issue_rate.argtypes = [_I32, _I32, _I64, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_I32)]
    L.fdd_plan_set_subband.argtypes = [_P, _I32, _I32, _I32]
    L.fdd_rfi_workspace_size.argtypes = [_I32, _I32, _I64, ctypes.POINTER(_SZ)]
    L.fdd_rfi_clean.argtypes = [ctypes.POINTER(_RfiDesc), _P, _I32, _I32, _I64, _I64, _P, _SZ, _P, _P, _P]
    L.fdd_plan_get_subband.argtypes = [_P, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]
    L.fdd_sb_table.argtypes = [_I32, _I32, _I32, _P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, _I32, _P]
    L.fdd_cluster_workspace_size.argtypes = [_I64, ctypes.POINTER(_SZ)]
    L.fdd_cluster.argtypes = [_P, _P, _I64, _P, _SZ, _P, _I64, _P, _P]
    _lib = L
    return L


def version():
    return _lib_raw().fdd_version().decode()


def variants():
    """[{index, kind, bytes_per_sample, dm_per_block, tile, threads, group}] of the compiled
    dedispersion kernels (kind 0 brute force, 1 pattern-factored with channel groups of size
    `group`, 2 SB-factored, 3 SB-factored with pattern-factored partial sums, groups of `group`)."""
    L = _lib_raw()
    n = _I32()
    _check(L.fdd_num_variants(ctypes.byref(n)), "fdd_num_variants")
    out = []
    for v in range(n.value):
        e, bd, t, th, g = _I32(), _I32(), _I32(), _I32(), _I32()
        _check(L.fdd_variant_info(v, ctypes.byref(e), ctypes.byref(bd), ctypes.byref(t), ctypes.byref(th),
                                  ctypes.byref(g)), "fdd_variant_info")
        k = _I32()
        _check(L.fdd_variant_kind(v, ctypes.byref(k)), "fdd_variant_kind")
        out.append(dict(index=v, kind=k.value, bytes_per_sample=e.value, dm_per_block=bd.value, tile=t.value,
                        threads=th.value, group=g.value))
    return out


def _check(code, where):
    if code != 0:
        raise FddError(code, where)


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, name, dtype=None):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must have dtype %s" % (name, dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


def _check_outputs(plan, n_out, cands, count, series):
    """Validate caller-given output buffers before their pointers reach the
    library, which writes up to cands.shape[0] 32-byte records, one uint64
    count and (with series) fdd_series_size(n_out) bytes through them."""
    torch = _torch()
    if not isinstance(cands, torch.Tensor) or cands.dtype != torch.int32 or cands.dim() != 2 or cands.shape[1] != 8:
        raise TypeError("cands must be an int32 tensor of shape [cap, 8] (32-byte records)")
    if not isinstance(count, torch.Tensor) or count.dtype != torch.int64 or count.numel() < 1:
        raise TypeError("count must be an int64 tensor with at least one element")
    if series is not None:
        if not isinstance(series, torch.Tensor) or series.dtype != torch.int32:
            raise TypeError("series must be an int32 tensor")
        if series.numel() * 4 < plan.series_size(n_out):
            raise ValueError("series holds %d bytes; this search writes %d" % (series.numel() * 4,
                                                                              plan.series_size(n_out)))


@dataclass
class SearchResult:
    cands: "object"     # torch.int32 [cap, 8] raw 32-byte records on the device
    count: "object"     # torch.int64 [1] on the device (true count; > cap means overflow)
    series: "object"    # torch.int32 flat series buffer or None
    cap: int

    def candidates(self):
        """Copy to host and decode (sorted by sb, dm_index, width, t)."""
        n = int(self.count.item())
        return decode_candidates(self.cands, min(n, self.cap)), n


@dataclass
class Job:
    """One chunk of a batched search (include/fdd.h: fdd_job).  Tensors are
    CUDA tensors owned by the caller; `workspace` must be sized by
    Plan.workspace_size(n_in, n_out, with_series=series is None)."""
    tabs: "object"
    n_in: int
    workspace: "object"
    cands: "object"
    count: "object"
    t_offset: int = 0
    series: "object" = None
    bins_absolute: bool = False   # True: a window of a stream (include/fdd.h: fdd_search_window)

    def result(self):
        return SearchResult(cands=self.cands, count=self.count, series=self.series, cap=int(self.cands.shape[0]))


def _jobs_array(jobs):
    import torch
    arr = (_Job * len(jobs))()
    for k, j in enumerate(jobs):
        arr[k].d_tabs = _dev_ptr(j.tabs, "tabs", torch.uint8).value
        arr[k].n_in = int(j.n_in)
        arr[k].pitch = int(j.tabs.shape[2])
        arr[k].t_offset_native = int(j.t_offset)
        arr[k].d_workspace = _dev_ptr(j.workspace, "workspace").value
        arr[k].workspace_bytes = int(j.workspace.numel() * j.workspace.element_size())
        arr[k].d_cands = _dev_ptr(j.cands, "cands").value
        arr[k].cap = int(j.cands.shape[0])
        arr[k].d_count = _dev_ptr(j.count, "count").value
        arr[k].d_series = _dev_ptr(j.series, "series", torch.int32).value if j.series is not None else None
        arr[k].bins_absolute = 1 if j.bins_absolute else 0
    return arr


class Graph:
    """CUDA graph of a batched search over fixed jobs (include/fdd.h: fdd_graph_*)."""

    def __init__(self, plan, jobs, n_out):
        h = ctypes.c_void_p()
        self._plan = plan
        self._jobs = list(jobs)
        _check(_lib_raw().fdd_graph_create(plan.handle, _jobs_array(self._jobs), len(self._jobs), int(n_out),
                                           ctypes.byref(h)), "fdd_graph_create")
        self._h = h

    def update(self, jobs):
        self._jobs = list(jobs)
        _check(_lib_raw().fdd_graph_update(self._h, _jobs_array(self._jobs), len(self._jobs)), "fdd_graph_update")

    def launch(self, stream=None):
        _check(_lib_raw().fdd_graph_launch(self._h, _stream_handle(stream)), "fdd_graph_launch")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib_raw().fdd_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


FDD_ERR_UNSUPPORTED = -5
FDD_ERR_SEQUENCE = -8
FDD_BATCH_SB_FACTORED = 1000
FDD_BATCH_SB_PERSISTENT = 1001
FDD_STATUS_TILE_WAIT = 1
FDD_ERR_TIMEOUT = -10
FDD_ERR_BUSY = -9


def now():
    """The serving runtime's monotonic clock (seconds)."""
    return float(_lib_raw().fdd_now())


class Server:
    """Serving runtime (include/fdd.h: fdd_server_*): per-beam device window
    buffers, slots sized from free HBM, continuous batching of complete
    windows onto the GPU."""

    def __init__(self, plan, n_beams, chunk_len, max_slots=0, hbm_reserve_frac=0.1, hbm_budget_bytes=0,
                 cap_per_window=1 << 15, sb_plans=None):
        """sb_plans: one single-SB Plan per SB of `plan` switches the server to
        the plain per-SB path (include/fdd.h: fdd_server_set_plain)."""
        d = _ServerDesc(int(n_beams), int(chunk_len), int(max_slots), float(hbm_reserve_frac),
                        int(hbm_budget_bytes), int(cap_per_window))
        h = ctypes.c_void_p()
        _check(_lib_raw().fdd_server_create(plan.handle, ctypes.byref(d), ctypes.byref(h)), "fdd_server_create")
        self._h = h
        self._plan = plan
        self._sb_plans = list(sb_plans) if sb_plans else []
        if self._sb_plans:
            arr = (ctypes.c_void_p * len(self._sb_plans))(*[p_.handle.value for p_ in self._sb_plans])
            _check(_lib_raw().fdd_server_set_plain(self._h, arr, len(self._sb_plans)), "fdd_server_set_plain")
        self.n_beams, self.chunk_len, self.cap_per_window = int(n_beams), int(chunk_len), int(cap_per_window)

    def push(self, beam, seq, chunk, t_arrival=None):
        """Deliver a host chunk (numpy uint8 or pinned CPU torch tensor,
        [n_tab][n_chan][chunk_len], contiguous).  Returns 0, FDD_ERR_BUSY or
        FDD_ERR_SEQUENCE; raises on other errors."""
        need = self._plan.n_tab * self._plan.n_chan * self.chunk_len
        if int(np.prod(chunk.shape)) != need:
            raise ValueError("chunk must hold n_tab * n_chan * chunk_len samples")
        if hasattr(chunk, "data_ptr"):
            if chunk.is_cuda or not chunk.is_contiguous() or chunk.element_size() != 1:
                raise ValueError("chunk must be a contiguous host uint8 tensor")
            ptr = chunk.data_ptr()
        else:
            if not chunk.flags["C_CONTIGUOUS"] or chunk.dtype != np.uint8:
                raise ValueError("chunk must be a contiguous uint8 array")
            ptr = chunk.ctypes.data
        t = now() if t_arrival is None else float(t_arrival)
        code = _lib_raw().fdd_server_push(self._h, int(beam), int(seq), ctypes.c_void_p(ptr), t)
        if code in (0, FDD_ERR_BUSY, FDD_ERR_SEQUENCE):
            return code
        raise FddError(code, "fdd_server_push")

    def reset_beam(self, beam, next_seq):
        return _lib_raw().fdd_server_reset_beam(self._h, int(beam), int(next_seq))

    def poll(self):
        _check(_lib_raw().fdd_server_poll(self._h), "fdd_server_poll")

    def drain(self):
        _check(_lib_raw().fdd_server_drain(self._h), "fdd_server_drain")

    def results(self, max_results=4096):
        """[(window-record dict, candidates structured array)] in completion order."""
        out = (_WindowResult * max_results)()
        cap = max_results * self.cap_per_window
        cands = np.zeros(cap, dtype=CAND_DTYPE)
        n, nc = _I32(), _I64()
        _check(_lib_raw().fdd_server_results(self._h, out, int(max_results), cands.ctypes.data_as(ctypes.c_void_p),
                                             int(cap), ctypes.byref(n), ctypes.byref(nc)), "fdd_server_results")
        res = []
        for k in range(n.value):
            r = {f: getattr(out[k], f) for f, _ in _WindowResult._fields_}
            c = cands[r["cand_offset"]:r["cand_offset"] + r["n_cands_kept"]].copy()
            res.append((r, np.sort(c, order=["sb", "dm_index", "width_native", "t_native"])))
        return res

    def info(self):
        st = _ServerStats()
        _check(_lib_raw().fdd_server_info(self._h, ctypes.byref(st)), "fdd_server_info")
        return {f: getattr(st, f) for f, _ in _ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib_raw().fdd_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Stream:
    """Per-beam streaming search (include/fdd.h: fdd_stream_*): chunks are
    pushed from device memory in order; each completed window is searched on
    the device."""

    def __init__(self, plan, beam_id, chunk_len, cap=1 << 15):
        h = ctypes.c_void_p()
        _check(_lib_raw().fdd_stream_open(plan.handle, int(beam_id), int(chunk_len), int(cap), ctypes.byref(h)),
               "fdd_stream_open")
        self._h = h
        self._plan = plan
        self.chunk_len, self.cap = int(chunk_len), int(cap)

    def push(self, chunk, seq, stream=None):
        """chunk: CUDA uint8 tensor [n_tab][n_chan][>= chunk_len] (rows at its
        last-dimension pitch).  Returns 0 or FDD_ERR_SEQUENCE; raises on
        other errors."""
        import torch
        if chunk.dim() != 3 or chunk.shape[0] != self._plan.n_tab or chunk.shape[1] != self._plan.n_chan:
            raise ValueError("chunk must be [n_tab][n_chan][pitch]")
        if chunk.shape[2] < self.chunk_len:
            raise ValueError("chunk pitch shorter than chunk_len")
        code = _lib_raw().fdd_stream_push(self._h, _dev_ptr(chunk, "chunk", torch.uint8), int(chunk.shape[2]),
                                          int(seq), _stream_handle(stream))
        if code in (0, FDD_ERR_SEQUENCE):
            return code
        raise FddError(code, "fdd_stream_push")

    def results(self, cands, count):
        """Enqueue the last window's records into device `cands` (int32
        [cap, 8]) and its true count into device `count` (int64 [1]); returns
        the window's first output sample, or -1 if no new window."""
        import torch
        t0 = _I64()
        _check(_lib_raw().fdd_stream_results(self._h, _dev_ptr(cands, "cands", torch.int32), int(cands.shape[0]),
                                             _dev_ptr(count, "count", torch.int64), ctypes.byref(t0)),
               "fdd_stream_results")
        return int(t0.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib_raw().fdd_stream_close(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def probe_issue_rate(kind, blocks_per_sm=8, iters=1 << 16):
    """Issue-rate probe (include/fdd.h: fdd_probe_issue_rate) on the current
    device: kind 0 integer adds/s, 1 byte permutes/s, 2 shared-memory bytes
    loaded/s.  Returns dict(per_second, ms, n_sm)."""
    v, t, n = ctypes.c_double(), ctypes.c_float(), _I32()
    _check(_lib_raw().fdd_probe_issue_rate(int(kind), int(blocks_per_sm), int(iters), ctypes.byref(v),
                                           ctypes.byref(t), ctypes.byref(n)), "fdd_probe_issue_rate")
    return dict(per_second=v.value, ms=t.value, n_sm=n.value)


def selftest_bounded_wait(polls=4096):
    """Run the bounded-wait self-test (include/fdd.h: fdd_selftest_bounded_wait):
    True when a wait on an mbarrier that nothing arrives on gave up after
    `polls` polls and its kernel returned normally."""
    g = _I32()
    _check(_lib_raw().fdd_selftest_bounded_wait(int(polls), ctypes.byref(g)), "fdd_selftest_bounded_wait")
    return bool(g.value)


def cluster_workspace_size(cap_in):
    v = _SZ()
    _check(_lib_raw().fdd_cluster_workspace_size(int(cap_in), ctypes.byref(v)), "fdd_cluster_workspace_size")
    return int(v.value)


def cluster(cands, count, out, out_count, workspace=None, stream=None):
    """DM-width clustering on the device (include/fdd.h: fdd_cluster).
    cands: int32 CUDA tensor [cap_in, 8] of records, count: int64 [1] (true
    count as written by a search); out: int32 [cap_out, 8], out_count:
    int64 [1].  Asynchronous on `stream`."""
    import torch
    cap_in = int(cands.shape[0])
    need = cluster_workspace_size(cap_in)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=cands.device)
    _check(_lib_raw().fdd_cluster(_dev_ptr(cands, "cands", torch.int32), _dev_ptr(count, "count", torch.int64),
                                  cap_in, _dev_ptr(workspace, "workspace"),
                                  int(workspace.numel() * workspace.element_size()),
                                  _dev_ptr(out, "out", torch.int32), int(out.shape[0]),
                                  _dev_ptr(out_count, "out_count", torch.int64), _stream_handle(stream)),
           "fdd_cluster")
    return workspace


def sb_table(n_tab, n_sb, chan_freq_mhz, f_max_mhz=1500.0, alpha=0.80, b_max_m=1296.0, b_cq_m=144.0,
             chan_per_subband=1):
    """int16 [n_sb][n_chan] SB table from the array geometry (include/fdd.h:
    fdd_sb_table); defaults are Apertif-10's.  Host only."""
    f = np.ascontiguousarray(chan_freq_mhz, dtype=np.float64)
    out = np.zeros((int(n_sb), f.size), dtype=np.int16)
    _check(_lib_raw().fdd_sb_table(int(n_tab), int(n_sb), f.size, f.ctypes.data_as(ctypes.c_void_p), float(f_max_mhz),
                                   float(alpha), float(b_max_m), float(b_cq_m), int(chan_per_subband),
                                   out.ctypes.data_as(ctypes.c_void_p)), "fdd_sb_table")
    return out


def rfi_clean(tabs, n_in, time_thresh=4.0, time_iters=3, freq_thresh=4.0, freq_iters=3, time_flags=None,
              chan_flags=None, workspace=None, stream=None):
    """RFI mitigation in place on a CUDA uint8 tensor [n_tab][n_chan][pitch]
    (include/fdd.h: fdd_rfi_clean).  Optional CUDA uint8 outputs: time_flags
    [n_tab][n_in], chan_flags [n_tab][n_chan]."""
    import torch
    n_tab, n_chan, pitch = (int(v) for v in tabs.shape)
    need = _SZ()
    _check(_lib_raw().fdd_rfi_workspace_size(n_tab, n_chan, int(n_in), ctypes.byref(need)), "fdd_rfi_workspace_size")
    if workspace is None:
        workspace = torch.empty(need.value, dtype=torch.uint8, device=tabs.device)
    d = _RfiDesc(float(time_thresh), int(time_iters), float(freq_thresh), int(freq_iters))
    _check(_lib_raw().fdd_rfi_clean(ctypes.byref(d), _dev_ptr(tabs, "tabs", torch.uint8), n_tab, n_chan, int(n_in), pitch,
                                    _dev_ptr(workspace, "workspace"), int(workspace.numel()),
                                    _dev_ptr(time_flags, "time_flags", torch.uint8) if time_flags is not None else None,
                                    _dev_ptr(chan_flags, "chan_flags", torch.uint8) if chan_flags is not None else None,
                                    _stream_handle(stream)), "fdd_rfi_clean")
    return workspace


def sort_candidates(cands):
    """Sort a host structured array of CAND_DTYPE records in place with the
    library's fdd_sort_candidates; returns it."""
    if cands.dtype != CAND_DTYPE or not cands.flags["C_CONTIGUOUS"]:
        raise ValueError("cands must be a contiguous CAND_DTYPE array")
    _check(_lib_raw().fdd_sort_candidates(cands.ctypes.data_as(ctypes.c_void_p), int(cands.size)),
           "fdd_sort_candidates")
    return cands


def _plan_desc(n_tab, n_chan, n_sb, chan_freq_mhz, t_samp_s, ranges, snr_thresh, keep):
    freq = np.ascontiguousarray(chan_freq_mhz, dtype=np.float64)
    rs = [dict(dm0=float(r["dm0"]), ddm=float(r["ddm"]), n_dm=int(r["n_dm"]), downsamp=int(r.get("downsamp", 1)),
               widths=[int(w) for w in r["widths"]]) for r in ranges]
    ws = [np.ascontiguousarray(r["widths"], dtype=np.int32) for r in rs]
    rr = (_Range * len(rs))()
    for k, r in enumerate(rs):
        rr[k].dm0, rr[k].ddm, rr[k].n_dm = r["dm0"], r["ddm"], r["n_dm"]
        rr[k].downsamp, rr[k].n_width = r["downsamp"], len(r["widths"])
        rr[k].widths = ws[k].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    keep.extend([freq, ws, rr])
    return _PlanDesc(n_tab, n_chan, n_sb, freq.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(t_samp_s),
                     len(rs), rr, float(snr_thresh))


def fact_tables_host(n_tab, n_chan, n_sb, chan_freq_mhz, t_samp_s, ranges, sb_map, r, variant, chan_per_stage):
    """Host-only build of the pattern-factored kernel's tables (include/fdd.h:
    fdd_fact_tables_host), for inspection and CPU checks.  Needs no GPU."""
    L = _lib_raw()
    keep = []
    desc = _plan_desc(n_tab, n_chan, n_sb, chan_freq_mhz, t_samp_s, ranges, 0.0, keep)
    sb = np.ascontiguousarray(sb_map, dtype=np.int16)
    info = np.zeros(15, np.int64)
    args = [ctypes.byref(desc), sb.ctypes.data_as(ctypes.c_void_p), int(r), int(variant), int(chan_per_stage),
            info.ctypes.data_as(ctypes.c_void_p)]
    _check(L.fdd_fact_tables_host(*args, None, None, None, None, None, None), "fdd_fact_tables_host")
    Lw, pat_bytes, n_groups, n_stages, desc_ints, smem, n_desc, n_blk = [int(v) for v in info[:8]]
    out = dict(Lw=Lw, pat_bytes=pat_bytes, n_groups=n_groups, n_stages=n_stages, desc_ints=desc_ints,
               smem_bytes=smem, n_desc=n_desc, n_blk=n_blk)
    out.update(zip(["zero_off", "raw_off", "rb", "pat_off", "bar_off", "pat_bufs", "box_rows"],
                   [int(v) for v in info[8:]]))
    if Lw < 0:
        return out
    v = variants()[int(variant)]
    bd = v["dm_per_block"]
    n_dm = int(ranges[r]["n_dm"])
    out["base"] = np.zeros((n_blk, n_chan), np.int32)
    out["goff"] = np.zeros((n_blk, n_groups, bd), np.int32)
    out["pdesc"] = np.zeros((max(n_desc, 1), desc_ints), np.int32)
    out["pd_idx"] = np.zeros((n_blk, n_stages, 2), np.int32)
    out["delays"] = np.zeros((n_dm, n_chan), np.int32)
    out["bbase"] = np.zeros((n_blk, (n_chan + out["box_rows"] - 1) // out["box_rows"]), np.int32)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(L.fdd_fact_tables_host(*args, ptr(out["base"]), ptr(out["goff"]), ptr(out["pdesc"]), ptr(out["pd_idx"]),
                                  ptr(out["delays"]), ptr(out["bbase"])), "fdd_fact_tables_host")
    return out


def decode_candidates(cands, n):
    raw = cands[:n].contiguous().cpu().numpy().view(np.uint8).reshape(-1)
    arr = raw.view(CAND_DTYPE).copy()
    return np.sort(arr, order=["sb", "dm_index", "width_native", "t_native"])


class Plan:
    """A DM plan over SBs of one compound beam (include/fdd.h: fdd_plan_create).

    ranges: list of dicts {dm0, ddm, n_dm, downsamp, widths}.
    sb_map: int array [n_sb][n_chan] of TAB indices (n_tab = 1, zeros: plain
    single-beam search).
    """

    def __init__(self, n_tab, n_chan, n_sb, chan_freq_mhz, t_samp_s, ranges, snr_thresh, sb_map):
        L = _lib_raw()
        self._freq = np.ascontiguousarray(chan_freq_mhz, dtype=np.float64)
        if self._freq.size != n_chan:
            raise ValueError("chan_freq_mhz must have n_chan entries")
        sb = np.ascontiguousarray(sb_map, dtype=np.int16)
        if sb.shape != (n_sb, n_chan):
            raise ValueError("sb_map must be [n_sb][n_chan]")
        self.ranges = [dict(dm0=float(r["dm0"]), ddm=float(r["ddm"]), n_dm=int(r["n_dm"]),
                            downsamp=int(r.get("downsamp", 1)), widths=[int(w) for w in r["widths"]])
                       for r in ranges]
        self._widths = [np.ascontiguousarray(r["widths"], dtype=np.int32) for r in self.ranges]
        rr = (_Range * len(self.ranges))()
        for k, r in enumerate(self.ranges):
            rr[k].dm0, rr[k].ddm, rr[k].n_dm = r["dm0"], r["ddm"], r["n_dm"]
            rr[k].downsamp, rr[k].n_width = r["downsamp"], len(r["widths"])
            rr[k].widths = self._widths[k].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        desc = _PlanDesc(n_tab, n_chan, n_sb, self._freq.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         float(t_samp_s), len(self.ranges), rr, float(snr_thresh))
        h = ctypes.c_void_p()
        _check(L.fdd_plan_create(ctypes.byref(desc), sb.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)),
               "fdd_plan_create")
        self._h = h
        self.n_tab, self.n_chan, self.n_sb = int(n_tab), int(n_chan), int(n_sb)
        self.t_samp_s = float(t_samp_s)
        self.snr_thresh = float(snr_thresh)

    # -- queries
    @property
    def handle(self):
        return self._h

    @property
    def max_delay(self):
        v = _I64()
        _check(_lib_raw().fdd_plan_max_delay(self._h, ctypes.byref(v)), "fdd_plan_max_delay")
        return int(v.value)

    def set_subband(self, r, chan_per_subband, dm_per_coarse):
        """Two-step subband dedispersion (approximate) for range r; (0, 0)
        restores exact dedispersion (include/fdd.h: fdd_plan_set_subband)."""
        _check(_lib_raw().fdd_plan_set_subband(self._h, int(r), int(chan_per_subband), int(dm_per_coarse)),
               "fdd_plan_set_subband")

    def get_subband(self, r):
        g, k = _I32(), _I32()
        _check(_lib_raw().fdd_plan_get_subband(self._h, int(r), ctypes.byref(g), ctypes.byref(k)), "fdd_plan_get_subband")
        return int(g.value), int(k.value)

    def last_launches(self):
        """Kernels enqueued by the last search / batched search (include/fdd.h:
        fdd_plan_last_launches)."""
        v = _I64()
        _check(_lib_raw().fdd_plan_last_launches(self._h, ctypes.byref(v)), "fdd_plan_last_launches")
        return int(v.value)

    def status(self, clear=False):
        """Device status word (include/fdd.h: fdd_plan_status; bit 0 =
        FDD_STATUS_TILE_WAIT, a tile-copy wait that gave up).  Blocking."""
        v = _I32()
        rc = _lib_raw().fdd_plan_status(self._h, ctypes.byref(v), 1 if clear else 0)
        if rc != FDD_ERR_TIMEOUT:          # FDD_ERR_TIMEOUT only says the word is set: return it
            _check(rc, "fdd_plan_status")
        return int(v.value)

    def set_scratch_limit(self, nbytes):
        """Cap the SB-factored kernel's partial-sum scratch (include/fdd.h:
        fdd_plan_set_scratch_limit; 0 = default)."""
        _check(_lib_raw().fdd_plan_set_scratch_limit(self._h, int(nbytes)), "fdd_plan_set_scratch_limit")

    def info(self, n_out):
        """(max delay in native samples, workspace bytes of an n_out search)
        (include/fdd.h: fdd_plan_info)."""
        md, ws = _I64(), _I64()
        _check(_lib_raw().fdd_plan_info(self._h, int(n_out), ctypes.byref(md), ctypes.byref(ws)), "fdd_plan_info")
        return int(md.value), int(ws.value)

    @property
    def n_dm_total(self):
        v = _I64()
        _check(_lib_raw().fdd_plan_total_dms(self._h, ctypes.byref(v)), "fdd_plan_total_dms")
        return int(v.value)

    def delays(self, r):
        out = np.empty((self.ranges[r]["n_dm"], self.n_chan), dtype=np.int32)
        _check(_lib_raw().fdd_plan_delays(self._h, int(r), out.ctypes.data_as(ctypes.c_void_p)),
               "fdd_plan_delays")
        return out

    def workspace_size(self, n_in, n_out, with_series=True):
        v = _SZ()
        _check(_lib_raw().fdd_workspace_size(self._h, int(n_in), int(n_out), int(bool(with_series)),
                                             ctypes.byref(v)), "fdd_workspace_size")
        return int(v.value)

    def series_size(self, n_out):
        v = _SZ()
        _check(_lib_raw().fdd_series_size(self._h, int(n_out), ctypes.byref(v)), "fdd_series_size")
        return int(v.value)

    def series_views(self, series, n_out, t0=None):
        """Split a flat series buffer into per-range [n_sb][n_dm][n_r] views:
        n_r = n_out // D for fdd_search; with t0 (a window's stream position,
        fdd_search_window) rows are ceil(n_out / D) apart and hold the
        window's n_r = ceil((t0 + n_out) / D) - ceil(t0 / D) bins."""
        out, off = [], 0
        for r in self.ranges:
            D = int(r["downsamp"])
            if t0 is None:
                stride = nr = int(n_out) // D
            else:
                stride = -(-int(n_out) // D)
                nr = -(-(int(t0) + int(n_out)) // D) - (-(-int(t0) // D))
            k = self.n_sb * r["n_dm"] * stride
            out.append(series[off:off + k].view(self.n_sb, r["n_dm"], stride)[:, :, :nr])
            off += k
        return out

    def window_sizes(self, n_out):
        """(n_in, workspace bytes, series bytes) of fdd_search_window windows
        of n_out outputs (include/fdd.h: fdd_window_sizes)."""
        n_in, ws, sr = _I64(), _SZ(), _SZ()
        _check(_lib_raw().fdd_window_sizes(self._h, int(n_out), ctypes.byref(n_in), ctypes.byref(ws),
                                           ctypes.byref(sr)), "fdd_window_sizes")
        return int(n_in.value), int(ws.value), int(sr.value)

    def search_window(self, tabs, n_in, n_out, t0, cap=1 << 16, workspace=None, cands=None, count=None,
                      series=None, want_series=False, stream=None):
        """One window of a beam's stream (include/fdd.h: fdd_search_window):
        tabs[..., 0] is stream sample t0; downsampling bins are aligned to the
        stream.  Buffers not given are allocated with torch on tabs' device."""
        torch = _torch()
        if tabs.dim() != 3 or tuple(tabs.shape[:2]) != (self.n_tab, self.n_chan):
            raise ValueError("tabs must be [n_tab][n_chan][pitch]")
        dev = tabs.device
        _, ws_bytes, sr_bytes = self.window_sizes(n_out)
        if want_series and series is None:
            series = torch.empty(sr_bytes // 4, dtype=torch.int32, device=dev)
        if workspace is None:
            workspace = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        if cands is None:
            cands = torch.empty((max(int(cap), 1), 8), dtype=torch.int32, device=dev)
        if count is None:
            count = torch.zeros(1, dtype=torch.int64, device=dev)
        if not isinstance(cands, torch.Tensor) or cands.dtype != torch.int32 or cands.dim() != 2 or \
                cands.shape[1] != 8:
            raise TypeError("cands must be an int32 tensor of shape [cap, 8] (32-byte records)")
        if not isinstance(count, torch.Tensor) or count.dtype != torch.int64 or count.numel() < 1:
            raise TypeError("count must be an int64 tensor with at least one element")
        if series is not None and series.numel() * 4 < sr_bytes:
            raise ValueError("series holds %d bytes; a window writes up to %d" % (series.numel() * 4, sr_bytes))
        code = _lib_raw().fdd_search_window(
            self._h, _dev_ptr(tabs, "tabs", torch.uint8), int(n_in), int(tabs.shape[2]), int(n_out), int(t0),
            _dev_ptr(workspace, "workspace"), int(workspace.numel() * workspace.element_size()),
            _dev_ptr(cands, "cands"), int(cands.shape[0]), _dev_ptr(count, "count"),
            _dev_ptr(series, "series", torch.int32) if series is not None else None,
            _stream_handle(stream))
        _check(code, "fdd_search_window")
        return SearchResult(cands=cands, count=count, series=series, cap=int(cands.shape[0]))

    # -- the hot path
    def search(self, tabs, n_in, n_out, t_offset=0, cap=1 << 16, workspace=None, cands=None, count=None,
               series=None, want_series=False, stream=None):
        """Search one chunk (include/fdd.h: fdd_search).  tabs: CUDA uint8
        [n_tab][n_chan][pitch], pitch a multiple of 16.  Buffers not given
        are allocated with torch on tabs' device."""
        torch = _torch()
        if tabs.dim() != 3 or tuple(tabs.shape[:2]) != (self.n_tab, self.n_chan):
            raise ValueError("tabs must be [n_tab][n_chan][pitch]")
        pitch = int(tabs.shape[2])
        dev = tabs.device
        if want_series and series is None:
            series = torch.empty(self.series_size(n_out) // 4, dtype=torch.int32, device=dev)
        ws_bytes = self.workspace_size(n_in, n_out, with_series=series is None)
        if workspace is None:
            workspace = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        if cands is None:
            cands = torch.empty((max(int(cap), 1), 8), dtype=torch.int32, device=dev)
        if count is None:
            count = torch.zeros(1, dtype=torch.int64, device=dev)
        _check_outputs(self, n_out, cands, count, series)
        cap = int(cands.shape[0])
        code = _lib_raw().fdd_search(
            self._h, _dev_ptr(tabs, "tabs", torch.uint8), int(n_in), pitch, int(n_out), int(t_offset),
            _dev_ptr(workspace, "workspace"), int(workspace.numel() * workspace.element_size()),
            _dev_ptr(cands, "cands"), cap, _dev_ptr(count, "count"),
            _dev_ptr(series, "series", torch.int32) if series is not None else None,
            _stream_handle(stream))
        _check(code, "fdd_search")
        return SearchResult(cands=cands, count=count, series=series, cap=cap)

    def get_config(self, r):
        c = KernelConfig()
        _check(_lib_raw().fdd_plan_get_config(self._h, int(r), ctypes.byref(c)), "fdd_plan_get_config")
        return c.as_dict()

    def set_config(self, r, variant, chan_per_stage=0):
        _check(_lib_raw().fdd_plan_set_config(self._h, int(r), int(variant), int(chan_per_stage)),
               "fdd_plan_set_config")

    def autotune(self, tabs, n_in, n_out, reps=3, workspace=None, stream=None):
        """Time every compatible kernel configuration per DM range on this
        chunk and keep the fastest (include/fdd.h: fdd_plan_autotune)."""
        torch = _torch()
        if workspace is None:
            workspace = torch.empty(self.workspace_size(n_in, n_out, with_series=True), dtype=torch.uint8,
                                    device=tabs.device)
        _check(_lib_raw().fdd_plan_autotune(self._h, _dev_ptr(tabs, "tabs", torch.uint8), int(n_in),
                                            int(tabs.shape[2]), int(n_out), _dev_ptr(workspace, "workspace"),
                                            int(workspace.numel()), int(reps), _stream_handle(stream)),
               "fdd_plan_autotune")
        return [self.get_config(r) for r in range(len(self.ranges))]

    def set_timing(self, enable=True):
        _check(_lib_raw().fdd_plan_set_timing(self._h, int(bool(enable))), "fdd_plan_set_timing")

    STAGE_NAMES = {0: "downsample", 1: "dedisperse", 2: "boxcar_snr", 3: "batch_prep"}

    def stage_times(self):
        """[(stage name, range or D, ms)] of the last timed search (after sync)."""
        n = _I32()
        _check(_lib_raw().fdd_plan_stage_times(self._h, 0, None, None, None, ctypes.byref(n)),
               "fdd_plan_stage_times")
        k = int(n.value)
        kind = np.zeros(max(k, 1), np.int32)
        rng = np.zeros(max(k, 1), np.int32)
        ms = np.zeros(max(k, 1), np.float32)
        _check(_lib_raw().fdd_plan_stage_times(self._h, k, kind.ctypes.data_as(ctypes.c_void_p),
                                               rng.ctypes.data_as(ctypes.c_void_p),
                                               ms.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n)),
               "fdd_plan_stage_times")
        return [(self.STAGE_NAMES[int(kind[i])], int(rng[i]), float(ms[i])) for i in range(k)]

    # -- batched search
    def make_job(self, tabs, n_in, n_out, t_offset=0, cap=1 << 16, want_series=False, bins_absolute=False):
        """Allocate a Job's output buffers and workspace with torch on tabs' device
        (bins_absolute: a window of a stream at t_offset, sized by window_sizes)."""
        torch = _torch()
        dev = tabs.device
        if bins_absolute:
            _, ws_b, sr_b = self.window_sizes(n_out)
            series = torch.empty(sr_b // 4, dtype=torch.int32, device=dev) if want_series else None
            ws = torch.empty(ws_b, dtype=torch.uint8, device=dev)
        else:
            series = torch.empty(self.series_size(n_out) // 4, dtype=torch.int32, device=dev) if want_series else None
            ws = torch.empty(self.workspace_size(n_in, n_out, with_series=series is None), dtype=torch.uint8,
                             device=dev)
        cands = torch.empty((max(int(cap), 1), 8), dtype=torch.int32, device=dev)
        count = torch.zeros(1, dtype=torch.int64, device=dev)
        return Job(tabs=tabs, n_in=int(n_in), workspace=ws, cands=cands, count=count, t_offset=int(t_offset),
                   series=series, bins_absolute=bool(bins_absolute))

    def batch_prepare(self, n_out, variant=-1):
        _check(_lib_raw().fdd_batch_prepare(self._h, int(n_out), int(variant)), "fdd_batch_prepare")

    def search_batch(self, jobs, n_out, stream=None):
        """All jobs in four launches (include/fdd.h: fdd_search_batch)."""
        _check(_lib_raw().fdd_search_batch(self._h, _jobs_array(jobs), len(jobs), int(n_out),
                                           _stream_handle(stream)), "fdd_search_batch")
        return [j.result() for j in jobs]

    def batch_autotune(self, jobs, n_out, reps=2, stream=None):
        _check(_lib_raw().fdd_batch_autotune(self._h, _jobs_array(jobs), len(jobs), int(n_out), int(reps),
                                             _stream_handle(stream)), "fdd_batch_autotune")
        return self.batch_config()

    def batch_config(self):
        v, g, t, bd = _I32(), _I32(), _I32(), _I32()
        ms = ctypes.c_float()
        _check(_lib_raw().fdd_batch_config(self._h, ctypes.byref(v), ctypes.byref(g), ctypes.byref(t),
                                           ctypes.byref(bd), ctypes.byref(ms)), "fdd_batch_config")
        return dict(variant=v.value, grid=g.value, threads=t.value, dm_per_block=bd.value, tuned_ms=ms.value)

    STATIC_SCRATCH_BYTES = 64 * 1024 * 1024   # FDD_STATIC_SCRATCH_BYTES of include/fdd.h (checked by the ABI test)

    def search_static(self, tabs, n_in, n_out, cands, count, t_offset=0, series=None, stream=None):
        """Allocation-free search (include/fdd.h: fdd_search_static): the
        library's static device array is the workspace; every output buffer
        is the caller's.  For callers that cannot allocate device memory at
        search time."""
        torch = _torch()
        if tabs.dim() != 3 or tuple(tabs.shape[:2]) != (self.n_tab, self.n_chan):
            raise ValueError("tabs must be [n_tab][n_chan][pitch]")
        _check_outputs(self, n_out, cands, count, series)
        code = _lib_raw().fdd_search_static(
            self._h, _dev_ptr(tabs, "tabs", torch.uint8), int(n_in), int(tabs.shape[2]), int(n_out),
            int(t_offset), _dev_ptr(cands, "cands"), int(cands.shape[0]), _dev_ptr(count, "count"),
            _dev_ptr(series, "series", torch.int32) if series is not None else None, _stream_handle(stream))
        _check(code, "fdd_search_static")
        return SearchResult(cands=cands, count=count, series=series, cap=int(cands.shape[0]))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib_raw().fdd_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def copy_rows(dst, dst_offset, dst_pitch, src, src_offset, src_pitch, width, rows, stream=None):
    """Row copy on a copy engine (include/fdd.h: fdd_copy_rows): `rows` rows
    of `width` bytes from contiguous tensor `src` (byte offset src_offset,
    row pitch src_pitch) to contiguous tensor `dst`; each is a CUDA tensor or
    page-locked host memory.  The byte ranges are checked against both
    tensors before the call."""
    torch = _torch()

    def ptr(t, off, pitch, name):
        if not isinstance(t, torch.Tensor) or not (t.is_cuda or t.is_pinned()):
            raise TypeError("%s must be a CUDA tensor or page-locked host memory" % name)
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        nbytes = t.numel() * t.element_size()
        if off < 0 or (rows > 0 and off + (rows - 1) * pitch + width > nbytes):
            raise ValueError("%s: rows reach past the tensor" % name)
        return ctypes.c_void_p(t.data_ptr() + int(off))
    code = _lib_raw().fdd_copy_rows(ptr(dst, dst_offset, dst_pitch, "dst"), int(dst_pitch),
                                    ptr(src, src_offset, src_pitch, "src"), int(src_pitch), int(width), int(rows),
                                    _stream_handle(stream))
    _check(code, "fdd_copy_rows")


def downsample_u8(x, n_in, downsamp, out=None, stream=None):
    """Time downsampling (include/fdd.h: fdd_downsample_u8) of every row of a
    CUDA uint8 tensor [..., pitch]; returns uint16 [..., out_pitch]."""
    torch = _torch()
    pitch = int(x.shape[-1])
    rows = int(np.prod(x.shape[:-1]))
    n_y = int(n_in) // int(downsamp)
    out_pitch = (n_y + 7) // 8 * 8
    if out is None:
        out = torch.empty(tuple(x.shape[:-1]) + (max(out_pitch, 8),), dtype=torch.int16, device=x.device)
    code = _lib_raw().fdd_downsample_u8(_dev_ptr(x, "x", torch.uint8), rows, int(n_in), pitch,
                                        int(downsamp), _dev_ptr(out, "out"), int(out.shape[-1]),
                                        _stream_handle(stream))
    _check(code, "fdd_downsample_u8")
    return out
