"""Pins of the oracle's collision tests against independent geometry.

Agents are convex boxes (Sec. 3.2 "Convex objects only"); the oracle decides
overlap with a separating-axis penetration depth.  Here the same decisions
are made by polygon clipping (Sutherland-Hodgman area) and by parametric
segment clipping (Liang-Barsky), written in the test in float64.
"""
import math

import numpy as np

from oracle.oracle import box_box, box_seg


def _corners(b):
    cx, cy, th, L, W = b
    c, s = math.cos(th), math.sin(th)
    pts = []
    for sx, sy in ((1, 1), (-1, 1), (-1, -1), (1, -1)):
        lx, ly = sx * L / 2, sy * W / 2
        pts.append((cx + c * lx - s * ly, cy + s * lx + c * ly))
    return pts  # counter-clockwise


def _clip(subject, clipper):
    """Sutherland-Hodgman: subject polygon clipped by a convex CCW polygon."""
    out = subject
    for k in range(len(clipper)):
        a, b = clipper[k], clipper[(k + 1) % len(clipper)]
        inp, out = out, []
        if not inp:
            break

        def inside(p):
            return (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0]) >= 0

        def cross(p, q):
            x1, y1, x2, y2 = a[0], a[1], b[0], b[1]
            x3, y3, x4, y4 = p[0], p[1], q[0], q[1]
            den = (x1 - x2) * (y3 - y4) - (y1 - y2) * (x3 - x4)
            t = ((x1 - x3) * (y3 - y4) - (y1 - y3) * (x3 - x4)) / den
            return (x1 + t * (x2 - x1), y1 + t * (y2 - y1))

        s = inp[-1]
        for e in inp:
            if inside(e):
                if not inside(s):
                    out.append(cross(s, e))
                out.append(e)
            elif inside(s):
                out.append(cross(s, e))
            s = e
    return out


def _area(poly):
    if len(poly) < 3:
        return 0.0
    x = np.array([p[0] for p in poly])
    y = np.array([p[1] for p in poly])
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


def test_box_box_matches_clipping_area():
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(4000):
        p = [rng.uniform(-3, 3), rng.uniform(-3, 3), rng.uniform(-math.pi, math.pi),
             rng.uniform(1, 6), rng.uniform(0.5, 3)]
        q = [rng.uniform(-3, 3), rng.uniform(-3, 3), rng.uniform(-math.pi, math.pi),
             rng.uniform(1, 6), rng.uniform(0.5, 3)]
        pen = box_box(p, q)
        area = _area(_clip(_corners(p), _corners(q)))
        if abs(pen) < 1e-6:
            continue          # grazing contact: both answers are rounding
        assert (pen > 0) == (area > 1e-12), (p, q, pen, area)
        checked += 1
    assert checked > 3900


def test_box_box_symmetry_and_axis_aligned_intervals():
    rng = np.random.default_rng(5)
    for _ in range(500):
        p = [rng.uniform(-3, 3), rng.uniform(-3, 3), rng.uniform(-4, 4), rng.uniform(1, 6), rng.uniform(0.5, 3)]
        q = [rng.uniform(-3, 3), rng.uniform(-3, 3), rng.uniform(-4, 4), rng.uniform(1, 6), rng.uniform(0.5, 3)]
        assert abs(box_box(p, q) - box_box(q, p)) < 1e-12
    # axis aligned: depth = min over x, y of the interval overlap
    for _ in range(500):
        L1, W1, L2, W2 = rng.uniform(1, 5, 4)
        dx, dy = rng.uniform(-6, 6, 2)
        ox = (L1 + L2) / 2 - abs(dx)
        oy = (W1 + W2) / 2 - abs(dy)
        got = box_box([0, 0, 0, L1, W1], [dx, dy, 0, L2, W2])
        assert abs(got - min(ox, oy)) < 1e-12
    # touching is not a collision (strict), a hair of overlap is
    assert box_box([0, 0, 0, 4, 2], [4, 0, 0, 4, 2]) <= 0
    assert box_box([0, 0, 0, 4, 2], [4 - 1e-6, 0, 0, 4, 2]) > 0
    assert box_box([0, 0, 0, 4, 2], [4 + 1e-6, 0, 0, 4, 2]) < 0


def _seg_inside_length(b, s):
    """Liang-Barsky: length of segment s inside box b (box frame clipping)."""
    cx, cy, th, L, W = b
    c, sn = math.cos(th), math.sin(th)

    def to_box(x, y):
        dx, dy = x - cx, y - cy
        return c * dx + sn * dy, -sn * dx + c * dy

    x0, y0 = to_box(s[0], s[1])
    x1, y1 = to_box(s[2], s[3])
    dx, dy = x1 - x0, y1 - y0
    t0, t1 = 0.0, 1.0
    for p, q in ((-dx, x0 + L / 2), (dx, L / 2 - x0), (-dy, y0 + W / 2), (dy, W / 2 - y0)):
        if p == 0:
            if q < 0:
                return 0.0
            continue
        r = q / p
        if p < 0:
            t0 = max(t0, r)
        else:
            t1 = min(t1, r)
    return max(0.0, t1 - t0) * math.hypot(dx, dy)


def test_box_segment_matches_liang_barsky():
    rng = np.random.default_rng(17)
    checked = 0
    for _ in range(4000):
        b = [rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(-math.pi, math.pi), rng.uniform(2, 6), rng.uniform(1, 3)]
        p0 = rng.uniform(-5, 5, 2)
        ang = rng.uniform(-math.pi, math.pi)
        ln = rng.uniform(0.2, 4)
        s = [p0[0], p0[1], p0[0] + ln * math.cos(ang), p0[1] + ln * math.sin(ang)]
        pen = box_seg(b, s)
        inside = _seg_inside_length(b, s)
        if abs(pen) < 1e-6:
            continue
        assert (pen > 0) == (inside > 1e-9), (b, s, pen, inside)
        checked += 1
    assert checked > 3900


def test_box_segment_special_cases():
    box = [0, 0, 0, 4, 2]
    # segment fully inside
    assert box_seg(box, [-0.5, 0, 0.5, 0]) > 0
    # crossing the box, endpoints outside
    assert box_seg(box, [-5, 0.3, 5, 0.3]) > 0
    # parallel to the long side, 1 mm outside
    assert box_seg(box, [-5, 1.001, 5, 1.001]) < 0
    # lying on the boundary: touching only
    assert box_seg(box, [-5, 1.0, 5, 1.0]) <= 0
    # diagonal passing near a corner outside
    assert box_seg(box, [2.5, 0.0, 3.5, 2.0]) < 0
