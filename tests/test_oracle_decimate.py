"""Pins of the oracle's Visvalingam-Whyatt decimation (Sec. 3.1).

* hand-worked cases (tests/golden/vw_cases.txt): areas, neighbour updates,
  ties, the strict tolerance;
* collinear points vanish for any positive tolerance, end points stay,
  polylines of fewer than 3 points are untouched;
* the same keep masks as a naive implementation that rescans every point
  after each elimination (same float32 arithmetic), on random polylines;
* a larger tolerance keeps a subset (the elimination order is one ranking);
* at termination every kept interior point spans at least the tolerance
  with its kept neighbours;
* on 0.1 m-sampled synthetic roads the default tolerance removes 10-15x of
  the points, the reduction the paper reports.
"""
import os

import numpy as np

from oracle.oracle import decimate
from paper_2408_01584_b300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "vw_cases.txt")
CASES = {"A": [(0, 0), (1, 1), (2, 0), (3, 0.25), (4, 0)], "B": [(0, 0), (1, 0), (2, 0), (3, 1), (4, 0)]}
DEFAULT_TOL = 1e-3     # m^2, the library default of decimate_scene (the paper gives no tolerance)


def _one(pts, tol):
    p = np.array(pts, np.float32)
    return decimate(np.array([0, len(p)]), p[:, 0], p[:, 1], tol)


def test_golden_hand_worked_cases():
    n = 0
    for line in open(GOLDEN):
        if not line.strip() or line.startswith("#"):
            continue
        name, tol, *keep = line.split()
        np.testing.assert_array_equal(_one(CASES[name], float(tol)), np.array(keep, np.uint8), err_msg=line)
        n += 1
    assert n == 10


def test_collinear_ends_and_short_polylines():
    line = [(k, 2.0 * k) for k in range(12)]
    np.testing.assert_array_equal(_one(line, 1e-6), [1] + [0] * 10 + [1])
    np.testing.assert_array_equal(_one(line, 0.0), [1] * 12)
    x = np.array([0, 1, 5, 5, 7], np.float32)
    y = np.array([0, 1, 5, 6, 9], np.float32)
    np.testing.assert_array_equal(decimate(np.array([0, 1, 3, 5]), x, y, 100.0), [1, 1, 1, 1, 1])


def _area32(a, b, c):
    dx1, dy1 = np.float32(b[0] - a[0]), np.float32(b[1] - a[1])
    dx2, dy2 = np.float32(c[0] - a[0]), np.float32(c[1] - a[1])
    return np.float32(0.5) * np.float32(abs(np.float32(dx1 * dy2) - np.float32(dx2 * dy1)))


def _naive(p, tol):
    """Rescan all interior points after each elimination."""
    alive = list(range(len(p)))
    area = {}
    last = np.float32(0)
    while len(alive) > 2:
        best = None
        for k in range(1, len(alive) - 1):
            i = alive[k]
            a = _area32(p[alive[k - 1]], p[i], p[alive[k + 1]])
            a = max(a, area.get(i, a)) if i in area else a
            if best is None or (a, i) < best:
                best = (a, i)
        if not best[0] < tol:
            break
        last = best[0]
        k = alive.index(best[1])
        alive.pop(k)
        # the published rule: recomputed neighbours never drop below the last eliminated area
        for j in (alive[k - 1], alive[k] if k < len(alive) else None):
            if j is not None and 0 < alive.index(j) < len(alive) - 1:
                kk = alive.index(j)
                area[j] = max(_area32(p[alive[kk - 1]], p[j], p[alive[kk + 1]]), last)
    keep = np.zeros(len(p), np.uint8)
    keep[alive] = 1
    return keep


def test_matches_naive_rescan_on_random_polylines():
    rng = np.random.default_rng(0)
    for case in range(150):
        n = int(rng.integers(3, 25))
        steps = rng.normal(size=(n, 2)) * np.array([1.0, 0.3])
        p = np.cumsum(steps, axis=0).astype(np.float32)
        if case % 3 == 0:
            p = np.round(p * 4) / 4                          # many equal areas: ties by index
        tol = float(rng.choice([0.01, 0.1, 0.5, 2.0]))
        got = decimate(np.array([0, n]), p[:, 0], p[:, 1], tol)
        np.testing.assert_array_equal(got, _naive([tuple(q) for q in p], np.float32(tol)), err_msg=f"case {case}")


def test_nested_and_terminal_property_on_synthetic_roads():
    sc = scenes.make_scene(np.array([4]), np.array([6000]), 9, n_poly=12, spacing=0.1)
    off = np.concatenate([[0], np.nonzero(np.diff(sc.road_poly))[0] + 1, [sc.num_road]]).astype(np.int32)
    prev = None
    for tol in (0.001, 0.01, 0.1):
        keep = decimate(off, sc.road_x, sc.road_y, tol)
        if prev is not None:
            assert ((keep == 1) <= (prev == 1)).all()          # a larger tolerance keeps a subset
        prev = keep
        for p in range(len(off) - 1):
            idx = np.arange(off[p], off[p + 1])[keep[off[p]:off[p + 1]] == 1]
            assert keep[off[p]] == 1 and keep[off[p + 1] - 1] == 1
            pts = np.stack([sc.road_x[idx], sc.road_y[idx]], 1)
            for k in range(1, len(idx) - 1):
                assert _area32(pts[k - 1], pts[k], pts[k + 1]) >= np.float32(tol)


def test_default_tolerance_gives_the_papers_reduction():
    sc = scenes.make_scene(np.array([8]), np.array([24000]), 3, n_poly=24, spacing=0.1)
    off = np.concatenate([[0], np.nonzero(np.diff(sc.road_poly))[0] + 1, [sc.num_road]]).astype(np.int32)
    keep = decimate(off, sc.road_x, sc.road_y, DEFAULT_TOL)
    ratio = len(keep) / keep.sum()
    print(f"VW at {DEFAULT_TOL} m^2 on 0.1 m roads: {len(keep)} -> {int(keep.sum())} points ({ratio:.1f}x)")
    assert 10.0 <= ratio <= 15.0
