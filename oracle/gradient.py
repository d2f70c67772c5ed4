"""Gradient oracle of the differentiable rollout (test infrastructure).

The objective of a rollout of T steps is
    L = sum_t sum_i d_ell[t,i] * ell[t,i],
    ell[t,i] = sum_f w_f * obs_t[i,f] + w_r * r_s(t,i),
where obs_t is the observation after step t (Sec. 3.2 "Sensor modalities",
ego frame), r_s = -(sqrt(d_goal^2 + c^2) - c) is a smooth goal reward (not in
the paper) counted for agents in the scene at the start of step t, and the
state follows the bicycle model of App. B, or the simplified invertible
model of Sec. 3.2 "Agent dynamics" (cfg.dynamics = 1).  Uncontrolled agents
of the "all nontrivial" initialisation (flag bit 16) do not move and have no
reward term (their reward is 0 too); like every agent still in the scene
they observe and are observed.  Collision, goal, done, selection
and clip decisions are the ones the brute-force oracle (oracle.cpp) takes
along its own float64 trajectory; with those fixed, L is a smooth function of
the actions and the initial state, and its gradient is taken here by PyTorch
autograd in float64 over a direct re-statement of the forward formulas.

Pins (tests/test_oracle_gradient.py): ell equals the C++ oracle's float64
objective; directional derivatives equal central finite differences of the
C++ oracle; straight-line closed forms.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from .oracle import Oracle, OracleConfig


@dataclasses.dataclass
class Decisions:
    flags_pre: np.ndarray    # uint8 [T, A]
    flags_post: np.ndarray   # uint8 [T, A]
    road_idx: np.ndarray     # int32 [T, A, K] (local, -1 = empty)
    partner_idx: np.ndarray  # int32 [T, A, P]
    ell: np.ndarray          # float64 [T, A] objective terms of the C++ oracle
    states: np.ndarray       # float64 [T+1, A, 4]


def oracle_rollout(scene, cfg: OracleConfig, actions, obs_weight, reward_weight, state0=None) -> Decisions:
    """Run the C++ oracle (float64) and record its decisions and ell."""
    o = Oracle(scene, cfg, 64)
    if state0 is not None:
        o.set_state(np.asarray(state0, np.float32))
    T, A = actions.shape[0], scene.num_agents
    w = np.asarray(obs_weight, np.float64)
    fpre = np.zeros((T, A), np.uint8)
    fpost = np.zeros((T, A), np.uint8)
    ridx = np.zeros((T, A, cfg.k_road), np.int32)
    pidx = np.zeros((T, A, cfg.n_partners), np.int32)
    ell = np.zeros((T, A))
    states = np.zeros((T + 1, A, 4))
    states[0] = o.get_state()[0]
    for t in range(T):
        fpre[t] = o.get_state()[1]
        out = o.step(actions[t])
        states[t + 1] = o.get_state()[0]
        fpost[t] = o.get_state()[1]
        obs, ridx[t], pidx[t] = o.observe64()
        act0 = (fpre[t] & 1) == 0
        ell[t] = obs @ w + reward_weight * np.where(act0, out["smooth_r"], 0.0)
    return Decisions(fpre, fpost, ridx, pidx, ell, states)


def _bicycle(state, act, L, dt, vmax):
    x, y, th, v = state.unbind(-1)
    a, d = act.unbind(-1)
    vbar = torch.clamp(v + 0.5 * a * dt, -vmax, vmax)
    beta = torch.atan(0.5 * torch.tan(d))
    x = x + vbar * torch.cos(th + beta) * dt
    y = y + vbar * torch.sin(th + beta) * dt
    th2 = th + vbar * torch.cos(beta) * torch.tan(d) / L * dt
    v = torch.clamp(v + a * dt, -vmax, vmax)
    return torch.stack([x, y, th2, v], -1)


def _invertible(state, act, dt):
    x, y, th, v = state.unbind(-1)
    a, k = act.unbind(-1)
    ds = v * dt + 0.5 * a * dt * dt
    return torch.stack([x + torch.cos(th) * ds, y + torch.sin(th) * ds, th + k * ds, v + a * dt], -1)


def objective_gradient(scene, cfg: OracleConfig, actions, obs_weight, reward_weight, d_ell=None, state0=None,
                       dec: Decisions | None = None):
    """Returns (ell [T,A] from the autograd forward, d_actions [T,A,2],
    d_state0 [A,4], decisions)."""
    f64 = torch.float64
    T, A = actions.shape[0], scene.num_agents
    K, P = cfg.k_road, cfg.n_partners
    if dec is None:
        dec = oracle_rollout(scene, cfg, actions, obs_weight, reward_weight, state0)
    s0 = torch.tensor(scene.state() if state0 is None else np.asarray(state0, np.float32), dtype=f64,
                      requires_grad=True)
    a = torch.tensor(np.asarray(actions, np.float32), dtype=f64, requires_grad=True)
    w = torch.tensor(np.asarray(obs_weight, np.float64))
    dl = torch.ones(T, A, dtype=f64) if d_ell is None else torch.tensor(np.asarray(d_ell, np.float64))
    L = torch.tensor(scene.length, dtype=f64)
    Wd = torch.tensor(scene.width, dtype=f64)
    gx = torch.tensor(scene.goal_x, dtype=f64)
    gy = torch.tensor(scene.goal_y, dtype=f64)
    rx = torch.tensor(scene.road_x, dtype=f64)
    ry = torch.tensor(scene.road_y, dtype=f64)
    rtype = torch.tensor(scene.road_type.astype(np.float64))
    world = np.repeat(np.arange(scene.num_worlds), np.diff(scene.agent_off))
    a0 = torch.tensor(scene.agent_off[world].astype(np.int64))
    r0 = torch.tensor(scene.road_off[world].astype(np.int64))
    wP = w[8:8 + 8 * P].reshape(P, 8)
    wR = w[8 + 8 * P:].reshape(K, 4)
    c_s = cfg.smooth_c
    state = s0
    total = torch.zeros((), dtype=f64)
    ells = []
    for t in range(T):
        moving = torch.tensor((dec.flags_pre[t] & (1 | 16)) == 0)       # in the scene and controlled
        nxt = _invertible(state, a[t], cfg.dt) if cfg.dynamics == 1 else _bicycle(state, a[t], L, cfg.dt, cfg.v_max)
        state = torch.where(moving[:, None], nxt, state)
        fpost = dec.flags_post[t]
        live = torch.tensor((fpost & 1) == 0, dtype=f64)
        x, y, th, v = state.unbind(-1)
        c, s = torch.cos(th), torch.sin(th)
        # ego row: (v, L, W, goal x', goal y', collided, offroad, goal)
        gdx, gdy = gx - x, gy - y
        ego = torch.stack([v, L, Wd, c * gdx + s * gdy, -s * gdx + c * gdy], -1)
        flags = torch.tensor(np.stack([(fpost >> 2) & 1, (fpost >> 3) & 1, (fpost >> 1) & 1], -1).astype(np.float64))
        ell = live * (ego @ w[:5]) + flags @ w[5:8]
        # partners
        pi = torch.tensor(dec.partner_idx[t].astype(np.int64))
        if P:
            pv = (pi >= 0).to(f64) * live[:, None]
            jg = a0[:, None] + pi.clamp(min=0)
            dx, dy = x[jg] - x[:, None], y[jg] - y[:, None]
            dth = th[jg] - th[:, None]
            feats = torch.stack([c[:, None] * dx + s[:, None] * dy, -s[:, None] * dx + c[:, None] * dy,
                                 torch.cos(dth), torch.sin(dth), v[jg], L[jg], Wd[jg], torch.ones_like(dx)], -1)
            ell = ell + ((feats * wP).sum(-1) * pv).sum(-1)
        # road points
        ri = torch.tensor(dec.road_idx[t].astype(np.int64))
        if K:
            rv = (ri >= 0).to(f64) * live[:, None]
            rg = r0[:, None] + ri.clamp(min=0)
            dx, dy = rx[rg] - x[:, None], ry[rg] - y[:, None]
            feats = torch.stack([c[:, None] * dx + s[:, None] * dy, -s[:, None] * dx + c[:, None] * dy, rtype[rg],
                                 torch.ones_like(dx)], -1)
            ell = ell + ((feats * wR).sum(-1) * rv).sum(-1)
        # smooth goal reward of controlled agents in the scene before the step
        rs = -(torch.sqrt((x - gx) ** 2 + (y - gy) ** 2 + c_s * c_s) - c_s)
        ell = ell + reward_weight * torch.where(moving, rs, torch.zeros_like(rs))
        ells.append(ell.detach())
        total = total + (dl[t] * ell).sum()
    total.backward()
    return torch.stack(ells).numpy(), a.grad.numpy(), s0.grad.numpy(), dec
