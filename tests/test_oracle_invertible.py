"""Pins of the oracle's simplified invertible model and expert-action
inversion (Sec. 3.2 "Agent dynamics").

* straight line with constant acceleration: x_n = x_0 + cos(theta) (v_0 n dt
  + a (n dt)^2 / 2), exactly (the double integrator integrates a constant
  acceleration without error);
* constant curvature at constant speed: the positions lie on the closed-form
  polygon inscribed in a circle of radius v dt / (2 sin(phi / 2)), phi =
  s v dt, which tends to 1 / s; the heading change is curvature x distance;
* the paper's two properties: the model ignores the vehicle length, and it is
  invertible: random actions -> trajectory -> inverted actions recover the
  actions, and replaying them recovers the trajectory;
* the kinematic bicycle's inversion recovers (a, delta) of App. B
  trajectories without speed clipping;
* degenerate and wrapped cases: a vehicle at rest gets curvature 0;
  headings wrapped to (-pi, pi] invert like unwrapped ones.
"""
import math

import numpy as np

from oracle import OracleConfig
from oracle.oracle import bicycle, invert

INV = OracleConfig(dynamics=1)
BIC = OracleConfig(dynamics=0)


def _roll(cfg, s0, acts, L):
    out = [np.array(s0, dtype=np.float64)]
    for a in acts:
        out.append(bicycle(cfg, out[-1], a, L))
    return np.stack(out)


def test_straight_line_constant_acceleration_is_exact():
    th, v0, a, n, dt = 0.4, 4.0, 1.3, 25, INV.dt
    s0 = np.array([[3.0, -2.0, th, v0]])
    traj = _roll(INV, s0, np.tile([[a, 0.0]], (n, 1, 1)), 4.5)
    t = np.arange(n + 1) * dt
    dist = v0 * t + 0.5 * a * t ** 2
    np.testing.assert_allclose(traj[:, 0, 0], 3.0 + math.cos(th) * dist, rtol=0, atol=1e-12)
    np.testing.assert_allclose(traj[:, 0, 1], -2.0 + math.sin(th) * dist, rtol=0, atol=1e-12)
    np.testing.assert_allclose(traj[:, 0, 3], v0 + a * t, rtol=0, atol=1e-12)
    assert (traj[:, 0, 2] == th).all()


def test_constant_curvature_polygon_and_heading():
    th0, v, s, n, dt = 0.3, 8.0, 0.05, 40, INV.dt
    traj = _roll(INV, np.array([[0.0, 0.0, th0, v]]), np.tile([[0.0, s]], (n, 1, 1)), 4.5)
    phi = s * v * dt                           # heading change per step = curvature x distance
    k = np.arange(n + 1)
    chord = v * dt
    ex = chord * np.sin(k * phi / 2) / np.sin(phi / 2) * np.cos(th0 + (k - 1) * phi / 2)
    ey = chord * np.sin(k * phi / 2) / np.sin(phi / 2) * np.sin(th0 + (k - 1) * phi / 2)
    np.testing.assert_allclose(traj[:, 0, 0], ex, atol=1e-10)
    np.testing.assert_allclose(traj[:, 0, 1], ey, atol=1e-10)
    np.testing.assert_allclose(traj[:, 0, 2], th0 + k * phi, atol=1e-12)
    # every point on one circle of radius chord / (2 sin(phi / 2)) -> 1 / s
    r = chord / (2 * math.sin(phi / 2))
    c = np.array([0.0, 0.0]) + r * np.array([-math.sin(th0 - phi / 2), math.cos(th0 - phi / 2)])
    np.testing.assert_allclose(np.hypot(traj[:, 0, 0] - c[0], traj[:, 0, 1] - c[1]), r, atol=1e-9)
    assert abs(r - 1 / s) < 1e-2 * (1 / s)


def test_heading_change_is_curvature_times_distance():
    rng = np.random.default_rng(1)
    s0 = np.column_stack([rng.uniform(-50, 50, 64), rng.uniform(-50, 50, 64), rng.uniform(-3, 3, 64),
                          rng.uniform(2, 15, 64)])
    a, s = rng.uniform(-3, 3, 64), rng.uniform(-0.2, 0.2, 64)
    n, dt = 17, INV.dt
    traj = _roll(INV, s0, np.tile(np.column_stack([a, s])[None], (n, 1, 1)), 4.5)
    dist = s0[:, 3] * n * dt + 0.5 * a * (n * dt) ** 2
    np.testing.assert_allclose(traj[-1, :, 2] - s0[:, 2], s * dist, atol=1e-11)


def test_simplified_model_ignores_the_length():
    rng = np.random.default_rng(2)
    s0 = np.column_stack([rng.normal(size=32), rng.normal(size=32), rng.normal(size=32), rng.uniform(0, 10, 32)])
    acts = np.stack([np.column_stack([rng.uniform(-4, 4, 32), rng.uniform(-0.3, 0.3, 32)]) for _ in range(12)])
    a = _roll(INV, s0, acts, 3.0)
    b = _roll(INV, s0, acts, 12.0)
    assert np.array_equal(a, b)
    assert not np.array_equal(_roll(BIC, s0, acts, 3.0), _roll(BIC, s0, acts, 12.0))


def test_simplified_model_is_invertible():
    rng = np.random.default_rng(3)
    n_ag, T = 200, 30
    s0 = np.column_stack([rng.uniform(-100, 100, n_ag), rng.uniform(-100, 100, n_ag), rng.uniform(-3, 3, n_ag),
                          rng.uniform(5, 15, n_ag)])
    acts = np.stack([np.column_stack([rng.uniform(-1.5, 1.5, n_ag), rng.uniform(-0.2, 0.2, n_ag)])
                     for _ in range(T)])
    traj = _roll(INV, s0, acts, 4.5)
    rec = invert(INV, traj, 4.5)
    np.testing.assert_allclose(rec, acts, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(_roll(INV, s0, rec, 4.5), traj, rtol=0, atol=1e-8)


def test_bicycle_inversion_recovers_app_b_actions_without_clipping():
    rng = np.random.default_rng(4)
    n_ag, T = 200, 30
    L = rng.uniform(3.5, 6.0, n_ag)
    s0 = np.column_stack([rng.uniform(-100, 100, n_ag), rng.uniform(-100, 100, n_ag), rng.uniform(-3, 3, n_ag),
                          rng.uniform(5, 15, n_ag)])
    acts = np.stack([np.column_stack([rng.uniform(-1.5, 1.5, n_ag), rng.uniform(-0.6, 0.6, n_ag)])
                     for _ in range(T)])
    traj = _roll(BIC, s0, acts, L)
    assert np.abs(traj[:, :, 3]).max() < BIC.v_max
    rec = invert(BIC, traj, L)
    np.testing.assert_allclose(rec, acts, rtol=1e-9, atol=1e-9)


def test_rest_and_wrapped_headings():
    # at rest: no distance covered, curvature 0 by convention
    rest = np.array([[[1.0, 2.0, 0.5, 0.0]], [[1.0, 2.0, 0.5, 0.0]]])
    assert (invert(INV, rest, 4.5) == 0).all() and (invert(BIC, rest, 4.5) == 0).all()
    # a left turn through +pi: logged headings wrap to (-pi, pi]
    rng = np.random.default_rng(5)
    s0 = np.array([[0.0, 0.0, math.pi - 0.05, 10.0]])
    acts = np.stack([np.array([[rng.uniform(-1, 1), 0.1]]) for _ in range(10)])
    traj = _roll(INV, s0, acts, 4.5)
    wrapped = traj.copy()
    wrapped[:, :, 2] = (wrapped[:, :, 2] + math.pi) % (2 * math.pi) - math.pi
    assert (wrapped[:, 0, 2] < 0).any() and (wrapped[:, 0, 2] > 0).any()
    np.testing.assert_allclose(invert(INV, wrapped, 4.5), acts, atol=1e-9)
