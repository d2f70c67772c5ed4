"""CPU check of the LiDAR kernel's arc angle (arc_atan2 in
csrc/lidar_kernel.cuh): its polynomial, read from the source, evaluated in
float32 with the kernel's steps, stays within 1e-6 rad of atan2 over every
octant, far inside the LIDAR_PAD margin that widens each obstacle's ray range
(Sec. 3.2 "Sensor modalities": rays are tested only inside the arcs the
obstacles subtend, so the margin must cover the angle's error)."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2408_01584_b300", "csrc", "lidar_kernel.cuh")


def _source():
    return open(SRC).read()


def _coefficients():
    body = re.search(r"float arc_atan2\(float y, float x\) \{(.*?)\n\}", _source(), re.S).group(1)
    first = float(re.search(r"float p = ([-0-9.e]+)f;", body).group(1))
    rest = [float(v) for v in re.findall(r"p = fmaf\(p, t, ([-0-9.e]+)f\);", body)]
    return [first] + rest          # highest power of t first (Horner order)


def arc_atan2(y, x):
    f = np.float32
    y, x = f(y), f(x)
    ax, ay = np.abs(x), np.abs(y)
    mx, mn = np.maximum(ax, ay), np.minimum(ax, ay)
    a = np.where(mx > 0, mn / np.where(mx > 0, mx, f(1)), f(0)).astype(f)
    t = (a * a).astype(f)
    c = _coefficients()
    p = np.full_like(a, f(c[0]))
    for k in c[1:]:
        p = (p.astype(np.float64) * t + k).astype(f)      # one rounding, like fmaf
    r = (p * a).astype(f)
    r = np.where(ay > ax, (f(np.pi / 2) - r).astype(f), r)
    r = np.where(x < 0, (f(np.pi) - r).astype(f), r)
    return np.copysign(r, y)


def test_polynomial_is_read():
    c = _coefficients()
    assert len(c) == 7 and abs(c[-1] - 1.0) < 1e-4          # atan(a) / a -> 1 as a -> 0


def test_error_inside_the_ray_margin():
    pad = float(re.search(r"LIDAR_PAD = ([0-9.e-]+)f;", _source()).group(1))
    rng = np.random.default_rng(0)
    ang = np.concatenate([rng.uniform(-np.pi, np.pi, 400_000),
                          np.arange(-8, 9) * np.pi / 4])           # octant edges included
    rad = rng.uniform(0.1, 60.0, ang.size)
    x, y = (rad * np.cos(ang)).astype(np.float32), (rad * np.sin(ang)).astype(np.float32)
    got = arc_atan2(y, x).astype(np.float64)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    err = np.abs(np.angle(np.exp(1j * (got - ref))))
    assert err.max() < 1e-6 and err.max() < pad / 10, err.max()


def test_special_directions():
    for (y, x), ref in {(0.0, 1.0): 0.0, (1.0, 0.0): np.pi / 2, (0.0, -1.0): np.pi, (-1.0, 0.0): -np.pi / 2,
                        (1.0, 1.0): np.pi / 4, (-1.0, -1.0): -3 * np.pi / 4}.items():
        assert abs(float(arc_atan2(np.array([y]), np.array([x]))[0]) - ref) < 1e-6
