"""Pins of the gradient oracle (oracle/gradient.py).

* its forward objective equals the C++ oracle's float64 objective;
* its directional derivatives equal central finite differences (h = 1e-4)
  of the C++ oracle's objective along seeded random directions, for actions
  and initial state, excluding directions whose +-h runs change a discrete
  decision (flags, selected indices); exclusions are counted;
* straight-line closed forms of App. B: with zero steering and weight only
  on the speed feature, d L / d a_m = (T - m) dt; with weight only on the
  goal offset along the heading, d L / d a_m = -sum_{t>=m} (t - m + 1/2) dt^2.
"""
import math

import numpy as np
import pytest

from oracle import OracleConfig
from oracle.gradient import objective_gradient, oracle_rollout
from paper_2408_01584_b300 import scenes
from tests._util import tiny_scene

CFG = OracleConfig(k_road=24, n_partners=5, episode_len=91, term_collision=True, term_offroad=True)
# the simplified invertible model (curvature actions), and the "all nontrivial" initialisation
INV = OracleConfig(k_road=24, n_partners=5, episode_len=91, term_collision=True, term_offroad=True, dynamics=1)
NTR = OracleConfig(k_road=24, n_partners=5, episode_len=91, term_collision=True, term_offroad=True,
                   nontrivial_init=True)


def _problem(seed=0, T=10, cfg=CFG):
    sc = scenes.make_scene(np.array([5, 8, 3]), np.array([600, 900, 400]), seed,
                           parked_frac=0.4 if cfg.nontrivial_init else 0.0)
    acts = scenes.make_actions(T, sc.num_agents, seed)
    if cfg.dynamics == 1:
        acts[:, :, 1] *= 0.2 / 0.7
    rng = np.random.default_rng(seed)
    w = rng.uniform(0, 1, CFG.feat)
    d_ell = rng.uniform(0.5, 1.5, (T, sc.num_agents))
    return sc, acts, w, 0.7, d_ell


def _objective(sc, acts, w, wr, d_ell, state0=None, cfg=CFG):
    dec = oracle_rollout(sc, cfg, acts, w, wr, state0)
    return float((dec.ell * d_ell).sum()), dec


def _same_decisions(a, b):
    return all((x == y).all() for x, y in ((a.flags_pre, b.flags_pre), (a.flags_post, b.flags_post),
                                           (a.road_idx, b.road_idx), (a.partner_idx, b.partner_idx)))


@pytest.mark.parametrize("cfg", [CFG, INV, NTR], ids=["bicycle", "invertible", "nontrivial"])
def test_forward_objective_matches_cpp_oracle(cfg):
    sc, acts, w, wr, d_ell = _problem(1, cfg=cfg)
    ell, _, _, dec = objective_gradient(sc, cfg, acts, w, wr, d_ell)
    np.testing.assert_allclose(ell, dec.ell, rtol=1e-10, atol=1e-8)
    if cfg.nontrivial_init:
        assert ((dec.flags_pre[0] & 16) != 0).any()


@pytest.mark.parametrize("seed,cfg", [(2, CFG), (3, CFG), (4, INV), (5, NTR)], ids=["b2", "b3", "inv", "ntr"])
def test_directional_derivatives_match_finite_differences(seed, cfg):
    sc, acts, w, wr, d_ell = _problem(seed, cfg=cfg)
    _, ga, gs, dec = objective_gradient(sc, cfg, acts, w, wr, d_ell)
    rng = np.random.default_rng(100 + seed)
    h = 1e-4
    s0 = sc.state().astype(np.float64)
    checked = excluded = 0
    worst = 0.0
    for k in range(16):
        # a direction on one agent's actions (all steps) and, every other
        # time, its initial state: other agents' decisions stay put
        i = rng.integers(sc.num_agents)
        da = np.zeros(acts.shape)
        ds = np.zeros(s0.shape)
        da[:, i] = rng.normal(size=(acts.shape[0], 2))
        if k % 2:
            ds[i] = rng.normal(size=4)
        # float32 inputs: perturb in float64 and let the oracle read float32 -> keep h large enough
        lp, dp = _objective(sc, (acts + h * da).astype(np.float32), w, wr, d_ell, (s0 + h * ds).astype(np.float32),
                            cfg)
        lm, dm = _objective(sc, (acts - h * da).astype(np.float32), w, wr, d_ell, (s0 - h * ds).astype(np.float32),
                            cfg)
        if not (_same_decisions(dp, dec) and _same_decisions(dm, dec)):
            excluded += 1
            continue
        # effective perturbation after float32 rounding of the inputs
        ea = ((acts + h * da).astype(np.float32).astype(np.float64) - (acts - h * da).astype(np.float32)) / 2
        es = ((s0 + h * ds).astype(np.float32).astype(np.float64) - (s0 - h * ds).astype(np.float32)) / 2
        fd = (lp - lm) / 2
        an = (ga * ea).sum() + (gs * es).sum()
        worst = max(worst, abs(fd - an) / (abs(an) + 1e-12))
        assert abs(fd - an) <= 1e-5 * abs(an) + 1e-8, (k, fd, an)
        checked += 1
    print(f"FD vs autograd: {checked} directions, {excluded} excluded, max rel err {worst:.2e}")
    assert checked >= 10, (checked, excluded)


def test_straight_line_closed_forms():
    T, dt = 12, 0.1
    # one agent heading along +x, goal far ahead, nothing else in range
    agent = (0.0, 0.0, 0.0, 5.0, 4.5, 2.0, 500.0, 0.0, 0)
    sc = tiny_scene([([agent], [(900.0, 900.0, 0, 0), (901.0, 900.0, 0, 0)])])
    cfg = OracleConfig(k_road=2, n_partners=1, episode_len=91)
    acts = np.zeros((T, 1, 2), np.float32)
    acts[:, 0, 0] = np.linspace(-1.0, 1.0, T)       # speed stays in range, no clipping
    m = np.arange(T)
    # speed feature only: ell_t = v_{t+1}
    w = np.zeros(cfg.feat)
    w[0] = 1.0
    _, ga, gs, _ = objective_gradient(sc, cfg, acts, w, 0.0)
    np.testing.assert_allclose(ga[:, 0, 0], (T - m) * dt, rtol=1e-12)
    np.testing.assert_allclose(gs[0, 3], T, rtol=1e-12)
    # goal offset along the heading: ell_t = gx - x_{t+1}
    w = np.zeros(cfg.feat)
    w[3] = 1.0
    _, ga, gs, _ = objective_gradient(sc, cfg, acts, w, 0.0)
    exp = np.array([-sum((t - mm + 0.5) * dt * dt for t in range(mm, T)) for mm in m])
    np.testing.assert_allclose(ga[:, 0, 0], exp, rtol=1e-12)
    np.testing.assert_allclose(gs[0, 0], -T, rtol=1e-12)
    # the smooth reward alone: d r_s / d x = -(x - gx) / sqrt(d^2 + c^2) at every step
    w = np.zeros(cfg.feat)
    _, ga, gs, dec = objective_gradient(sc, cfg, acts, w, 1.0)
    x = dec.states[1:, 0, 0]
    drdx = -(x - 500.0) / np.sqrt((x - 500.0) ** 2 + 1.0)
    np.testing.assert_allclose(gs[0, 0], drdx.sum(), rtol=1e-12)
    assert math.isfinite(ga.sum())
