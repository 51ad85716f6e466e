"""Pins of the oracle's DM-width clustering (Sec. "AMBER", "Clustering
(optional)": at one time and DM keep the best width; then neighbouring DM
trials keep their best candidate).

Pinned by a hand-worked example and by an independent restatement: the kept
records are exactly the maxima of the connected components of the graph
whose edges join candidates of the same SB and time whose DM indices differ
by at most one (brute force, pure Python), on random lists full of ties."""
import numpy as np
import pytest

import oracle


def _recs(rows):
    a = np.zeros(len(rows), dtype=oracle.CAND_DTYPE)
    for k, (sb, dm, w, t, snr) in enumerate(rows):
        a[k]["sb"], a[k]["dm_index"], a[k]["width_native"], a[k]["t_native"], a[k]["snr"] = sb, dm, w, t, snr
        a[k]["downsamp"], a[k]["dm"] = 1, 0.5 * dm
    return a


def _key(a):
    return [(int(r["sb"]), int(r["dm_index"]), int(r["width_native"]), int(r["t_native"]), float(r["snr"]))
            for r in a]


def test_hand_worked_example():
    rows = [
        # SB 0, t 100: DM 10 has three widths -> width 2 (S/N 9.0) survives step 1
        (0, 10, 1, 100, 8.5), (0, 10, 2, 100, 9.0), (0, 10, 4, 100, 8.7),
        # DM 11: a tie between widths 1 and 4 -> the smaller width
        (0, 11, 4, 100, 9.5), (0, 11, 1, 100, 9.5),
        (0, 12, 2, 100, 9.2),
        # DM 14 is not a neighbour of 12 (13 is empty): its own cluster
        (0, 14, 1, 100, 8.1),
        # another time: its own cluster even though DM 11 is occupied at t 100
        (0, 11, 1, 101, 10.0),
        # SB 1: an S/N tie between neighbouring DMs -> the smaller DM
        (1, 11, 1, 100, 8.2), (1, 10, 1, 100, 8.2),
        # consecutive global DM indices across a range boundary join
        (0, 2047, 8, 200, 12.0), (0, 2048, 16, 200, 12.5),
    ]
    got = _key(oracle.cluster(_recs(rows)))
    want = sorted([(0, 11, 1, 100, 9.5), (0, 14, 1, 100, 8.1), (0, 11, 1, 101, 10.0), (1, 10, 1, 100, 8.2),
                   (0, 2048, 16, 200, 12.5)])
    assert sorted(got) == want


def _components_brute(a):
    """Maxima of connected components; edges: same (sb, t), |d dm| <= 1."""
    n = len(a)
    seen = [False] * n
    kept = []
    for s in range(n):
        if seen[s]:
            continue
        comp, stack = [], [s]
        seen[s] = True
        while stack:
            u = stack.pop()
            comp.append(u)
            for v in range(n):
                if not seen[v] and a[v]["sb"] == a[u]["sb"] and a[v]["t_native"] == a[u]["t_native"] \
                        and abs(int(a[v]["dm_index"]) - int(a[u]["dm_index"])) <= 1:
                    seen[v] = True
                    stack.append(v)
        # highest S/N; ties: smaller DM, then smaller width, then earlier record
        best = min(comp, key=lambda k: (-float(a[k]["snr"]), int(a[k]["dm_index"]), int(a[k]["width_native"]), k))
        kept.append(best)
    return kept


@pytest.mark.parametrize("seed", range(12))
def test_equals_connected_component_maxima(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 160))
    rows = []
    for _ in range(n):
        rows.append((int(rng.integers(0, 3)), int(rng.integers(0, 12)), int(rng.choice([1, 2, 4, 8])),
                     int(rng.integers(0, 4)), float(rng.choice([8.25, 8.5, 9.0, 9.5, 11.0]))))
    a = _recs(rows)
    got = sorted(_key(oracle.cluster(a)))
    want = sorted(_key(a[_components_brute(a)]))
    assert got == want


def test_exact_duplicates_and_trivial_cases():
    a = _recs([(0, 5, 2, 7, 9.0), (0, 5, 2, 7, 9.0)])
    assert len(oracle.cluster(a)) == 1
    assert len(oracle.cluster(_recs([]))) == 0
    one = _recs([(3, 1, 4, 99, 8.01)])
    assert _key(oracle.cluster(one)) == _key(one)


def test_idempotent_and_subset():
    rng = np.random.default_rng(99)
    rows = [(int(rng.integers(0, 2)), int(rng.integers(0, 40)), int(rng.choice([1, 2, 4])), int(rng.integers(0, 6)),
             float(rng.uniform(8, 20))) for _ in range(600)]
    a = _recs(rows)
    c1 = oracle.cluster(a)
    assert set(_key(c1)) <= set(_key(a))
    assert sorted(_key(oracle.cluster(c1))) == sorted(_key(c1))
    # no two kept records of one (sb, t) are DM neighbours
    s = {(r[0], r[3], r[1]) for r in _key(c1)}
    assert not any((sb, t, dm + 1) in s for sb, t, dm in s)
