"""Pins of the oracle's bicycle model (App. B) against closed forms.

None of these re-type the oracle's update: each compares many Euler steps
with a closed-form trajectory, or one step with a hand-derived golden value.
"""
import math
import os

import numpy as np
import pytest

from oracle import OracleConfig
from oracle.oracle import bicycle

HERE = os.path.dirname(os.path.abspath(__file__))
CFG = OracleConfig(dt=0.1, v_max=30.0)


def _roll(state, actions, L):
    s = np.array(state, np.float64).reshape(1, 4)
    out = [s[0].copy()]
    for a in actions:
        s = bicycle(CFG, s, np.array(a, np.float64).reshape(1, 2), L)
        out.append(s[0].copy())
    return np.array(out)


def test_golden_single_steps():
    rows = []
    with open(os.path.join(HERE, "golden", "bicycle_cases.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            lhs, rhs = line.split("|")
            rows.append((np.array(lhs.split(), float), np.array(rhs.split(), float)))
    assert len(rows) >= 7
    for inp, exp in rows:
        got = bicycle(CFG, inp[:4].reshape(1, 4), inp[4:6].reshape(1, 2), inp[6])[0]
        np.testing.assert_allclose(got, exp, rtol=0, atol=1e-12)


@pytest.mark.parametrize("theta", [0.0, 0.7, -2.1])
def test_straight_line_constant_accel_exact(theta):
    # delta = 0, constant a, no clipping: the mid-step speed makes Euler exact,
    # x_n = x_0 + cos(theta) (v0 n dt + a (n dt)^2 / 2)
    v0, a, n, dt = 3.0, 1.5, 60, CFG.dt
    traj = _roll([1.0, -2.0, theta, v0], [(a, 0.0)] * n, 4.5)
    k = np.arange(n + 1)
    s = v0 * k * dt + 0.5 * a * (k * dt) ** 2
    np.testing.assert_allclose(traj[:, 0], 1.0 + math.cos(theta) * s, atol=1e-10)
    np.testing.assert_allclose(traj[:, 1], -2.0 + math.sin(theta) * s, atol=1e-10)
    np.testing.assert_allclose(traj[:, 2], theta, atol=0)
    np.testing.assert_allclose(traj[:, 3], v0 + a * k * dt, atol=1e-12)


def test_straight_line_varying_accel():
    # x_n = x_0 + cos(theta) dt sum_k (v_k + a_k dt / 2), v_n = v_0 + dt sum a_k
    rng = np.random.default_rng(3)
    acc = rng.uniform(-2, 2, 40)
    v0, th, dt = 8.0, 0.4, CFG.dt
    traj = _roll([0.0, 0.0, th, v0], [(a, 0.0) for a in acc], 4.5)
    v = v0 + dt * np.concatenate([[0.0], np.cumsum(acc)])
    vbar = v[:-1] + 0.5 * acc * dt
    s = np.concatenate([[0.0], np.cumsum(vbar * dt)])
    np.testing.assert_allclose(traj[:, 3], v, atol=1e-12)
    np.testing.assert_allclose(traj[:, 0], math.cos(th) * s, atol=1e-10)
    np.testing.assert_allclose(traj[:, 1], math.sin(th) * s, atol=1e-10)


@pytest.mark.parametrize("delta", [0.05, 0.3, -0.6])
def test_constant_steer_arc(delta):
    # a = 0, constant delta and v: heading grows by dth = v cos(beta) tan(delta) dt / L
    # per step and x_n = x_0 + v dt sin(n dth/2)/sin(dth/2) cos(theta0 + beta + (n-1) dth/2)
    v, L, th0, n, dt = 7.0, 4.5, 0.3, 50, CFG.dt
    traj = _roll([2.0, 5.0, th0, v], [(0.0, delta)] * n, L)
    beta = math.atan(0.5 * math.tan(delta))
    dth = v * math.cos(beta) * math.tan(delta) * dt / L
    k = np.arange(n + 1)
    gain = np.where(k == 0, 0.0, np.sin(k * dth / 2) / math.sin(dth / 2))
    ang = th0 + beta + (k - 1) * dth / 2
    np.testing.assert_allclose(traj[:, 2], th0 + k * dth, atol=1e-12)
    np.testing.assert_allclose(traj[:, 0], 2.0 + v * dt * gain * np.cos(ang), atol=1e-9)
    np.testing.assert_allclose(traj[:, 1], 5.0 + v * dt * gain * np.sin(ang), atol=1e-9)
    # every position lies on one circle of radius v dt / (2 sin(dth/2))
    rad = v * dt / (2 * abs(math.sin(dth / 2)))
    # centre: perpendicular bisector construction from the first three points
    p = traj[:3, :2]
    ax, ay, bx, by, cx, cy = p[0, 0], p[0, 1], p[1, 0], p[1, 1], p[2, 0], p[2, 1]
    d = 2 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by))
    ux = ((ax**2 + ay**2) * (by - cy) + (bx**2 + by**2) * (cy - ay) + (cx**2 + cy**2) * (ay - by)) / d
    uy = ((ax**2 + ay**2) * (cx - bx) + (bx**2 + by**2) * (ax - cx) + (cx**2 + cy**2) * (bx - ax)) / d
    r = np.hypot(traj[:, 0] - ux, traj[:, 1] - uy)
    np.testing.assert_allclose(r, rad, rtol=1e-9)


def test_arc_radius_limit():
    # as dt -> 0 the circle radius tends to L / (cos(beta) tan(delta))
    v, L, delta = 5.0, 4.5, 0.25
    beta = math.atan(0.5 * math.tan(delta))
    cfg = OracleConfig(dt=1e-4, v_max=30.0)
    s = np.array([[0.0, 0.0, 0.0, v]])
    pts = []
    for _ in range(3):
        pts.append(s[0, :2].copy())
        s = bicycle(cfg, s, np.array([[0.0, delta]]), L)
    dth = v * math.cos(beta) * math.tan(delta) * 1e-4 / L
    rad = v * 1e-4 / (2 * math.sin(dth / 2))
    assert abs(rad - L / (math.cos(beta) * math.tan(delta))) < 1e-6 * rad


def test_speed_clip_saturates_exactly():
    traj = _roll([0.0, 0.0, 0.0, 25.0], [(40.0, 0.0)] * 5, 4.5)
    assert traj[-1, 3] == 30.0
    traj = _roll([0.0, 0.0, 0.0, -25.0], [(-40.0, 0.1)] * 5, 4.5)
    assert traj[-1, 3] == -30.0
    # speed stays put once saturated while the position keeps moving at v_max
    traj = _roll([0.0, 0.0, 0.0, 30.0], [(5.0, 0.0)] * 3, 4.5)
    np.testing.assert_allclose(traj[:, 0], [0.0, 3.0, 6.0, 9.0], atol=1e-12)


def test_length_scales_turn_rate():
    # the yaw rate is inversely proportional to L (App. B: theta-dot has L in the denominator)
    a = _roll([0.0, 0.0, 0.0, 10.0], [(0.0, 0.2)], 4.0)
    b = _roll([0.0, 0.0, 0.0, 10.0], [(0.0, 0.2)], 8.0)
    assert abs(a[1, 2] - 2 * b[1, 2]) < 1e-14
    np.testing.assert_allclose(a[1, :2], b[1, :2], atol=0)
