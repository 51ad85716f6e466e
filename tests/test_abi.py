"""CPU-side checks of the C ABI: the library builds, loads, exports every
function include/fdd.h declares, and rejects bad plans on the host before any
device work."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "fdd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fdd_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2205_12362_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = header_functions()
    for must in ("fdd_plan_create", "fdd_plan_destroy", "fdd_plan_info", "fdd_search", "fdd_workspace_size",
                 "fdd_downsample_u8", "fdd_stream_open", "fdd_stream_push", "fdd_stream_results",
                 "fdd_stream_close", "fdd_sort_candidates", "fdd_error_string"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_error_strings_and_version(lib):
    lib.fdd_error_string.restype = ctypes.c_char_p
    lib.fdd_version.restype = ctypes.c_char_p
    assert lib.fdd_error_string(0) == b"ok"
    assert b"short" in lib.fdd_error_string(-2).lower() or b"input" in lib.fdd_error_string(-2).lower()
    assert b"gave up" in lib.fdd_error_string(-10)          # FDD_ERR_TIMEOUT
    for code in range(-10, 0):                                # every code has its own text
        assert lib.fdd_error_string(code) != b"unknown error"
    assert b"sm_103a" in lib.fdd_version()


def test_host_rejects_bad_plans(lib):
    import paper_2205_12362_b300 as fdd
    f = np.linspace(1220, 1520, 8)
    good = [dict(dm0=0.0, ddm=1.0, n_dm=4, downsamp=1, widths=[1, 2])]
    with pytest.raises(fdd.FddError) as e:   # TAB index out of range
        fdd.Plan(2, 8, 1, f, 81.92e-6, good, 8.0, np.full((1, 8), 2))
    assert e.value.code == -1
    with pytest.raises(fdd.FddError):        # negative DM step
        fdd.Plan(1, 8, 1, f, 81.92e-6, [dict(dm0=0.0, ddm=-1.0, n_dm=4, widths=[1])], 8.0, np.zeros((1, 8)))
    with pytest.raises(fdd.FddError):        # width beyond the limit
        fdd.Plan(1, 8, 1, f, 81.92e-6, [dict(dm0=0.0, ddm=1.0, n_dm=4, widths=[5000])], 8.0, np.zeros((1, 8)))
    with pytest.raises(fdd.FddError) as e:   # box sums that could leave int32 (16384 ch x 255 x D 257 x w 1024)
        fdd.Plan(1, 16384, 1, np.linspace(1220, 1520, 16384), 81.92e-6,
                 [dict(dm0=0.0, ddm=1.0, n_dm=1, downsamp=257, widths=[1024])], 8.0, np.zeros((1, 16384)))
    assert e.value.code == -5
    with pytest.raises(fdd.FddError):        # non-positive frequency
        fdd.Plan(1, 8, 1, np.zeros(8), 81.92e-6, good, 8.0, np.zeros((1, 8)))
    with pytest.raises(ValueError):          # sb_map shape
        fdd.Plan(1, 8, 2, f, 81.92e-6, good, 8.0, np.zeros((1, 8)))


def test_candidate_record_layout():
    import paper_2205_12362_b300 as fdd
    assert fdd.CAND_DTYPE.itemsize == 32
    assert [fdd.CAND_DTYPE.fields[k][1] for k in ("sb", "dm_index", "downsamp", "width_native",
                                                  "t_native", "dm", "snr")] == [0, 4, 8, 12, 16, 24, 28]


def test_variant_table():
    import paper_2205_12362_b300 as fdd
    vs = fdd.variants()
    assert len(vs) >= 4
    assert {v["bytes_per_sample"] for v in vs} == {1, 2}
    for v in vs:
        assert v["dm_per_block"] % 4 == 0 and v["threads"] % 32 == 0
        # factored tiles are 64 * NW samples (2 per lane and word); every tile start stays on a
        # 16-byte boundary of the input rows, as the TMA copies need
        assert v["tile"] > 0 and v["tile"] % (64 if v["kind"] == 1 else 128) == 0


def test_sort_candidates_host_helper():
    """fdd_sort_candidates (host) orders records by (sb, dm_index, width,
    t) exactly as numpy's lexicographic sort of the same fields."""
    import paper_2205_12362_b300 as m
    rng = np.random.default_rng(3)
    a = np.zeros(5000, dtype=m.CAND_DTYPE)
    a["sb"] = rng.integers(0, 4, a.size)
    a["dm_index"] = rng.integers(0, 30, a.size)
    a["width_native"] = rng.choice([1, 2, 4, 8], a.size)
    a["t_native"] = rng.integers(-5, 10 ** 10, a.size)
    a["snr"] = rng.random(a.size)
    want = np.sort(a.copy(), order=["sb", "dm_index", "width_native", "t_native"])
    got = m.sort_candidates(a)
    keys = ["sb", "dm_index", "width_native", "t_native"]
    for k in keys:
        assert (got[k] == want[k]).all()
    assert sorted(got["snr"].tolist()) == sorted(want["snr"].tolist())
    m.sort_candidates(np.zeros(0, dtype=m.CAND_DTYPE))


def test_static_scratch_size_matches_header():
    """The binding's STATIC_SCRATCH_BYTES is the header's FDD_STATIC_SCRATCH_BYTES."""
    import paper_2205_12362_b300 as fdd
    text = open(os.path.join(ROOT, "include", "fdd.h")).read()
    m = re.search(r"#define\s+FDD_STATIC_SCRATCH_BYTES\s+\((\d+)u\s*\*\s*(\d+)u\s*\*\s*(\d+)u\)", text)
    assert m, "FDD_STATIC_SCRATCH_BYTES not found in include/fdd.h"
    assert fdd.Plan.STATIC_SCRATCH_BYTES == int(m.group(1)) * int(m.group(2)) * int(m.group(3))


def test_copy_rows_rejects_bad_arguments(lib):
    """fdd_copy_rows refuses null pointers and pitches below the width on the
    host, before any CUDA call."""
    f = lib.fdd_copy_rows
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                  ctypes.c_void_p]
    buf = ctypes.create_string_buffer(64)
    p = ctypes.cast(buf, ctypes.c_void_p)
    assert f(None, 16, p, 16, 8, 2, None) == -1
    assert f(p, 16, None, 16, 8, 2, None) == -1
    assert f(p, 4, p, 16, 8, 2, None) == -1          # destination pitch below the width
    assert f(p, 16, p, 4, 8, 2, None) == -1          # source pitch below the width
    assert f(p, 16, p, 16, -1, 2, None) == -1
