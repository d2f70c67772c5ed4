"""GPU parity of the simplified invertible model and of the expert-action
inversion (Sec. 3.2 "Agent dynamics") against the float64 oracle, through the
C ABI.

* the model's step, teacher-forced per step, per-stage and fused, with the
  decisions checked on the GPU's post-step state;
* fused and per-stage forms bit-identical;
* gd_invert_actions against the oracle's inversion on the same float32
  trajectories, for both models, including headings wrapped to (-pi, pi];
* the round trip on the GPU: a trajectory stepped by the library, inverted,
  gives back its actions, and replaying them gives back the trajectory;
* the 1,024 x 64 workload at full size: inversion of a 91-step trajectory of
  every agent, sampled against the oracle.
"""
import math

import numpy as np
import pytest

from oracle import Oracle, OracleConfig
from oracle.oracle import bicycle, invert
from paper_2408_01584_b300 import scenes
from tests import parity
from tests._util import small_scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _curv_actions(T, A, seed):
    """Acceleration U[-4, 4] m/s^2, curvature U[-0.2, 0.2] 1/m."""
    a = scenes.make_actions(T, A, seed)
    a[:, :, 1] *= 0.2 / 0.7
    return a


@pytest.mark.parametrize("form", ["plain", "fused"])
def test_invertible_step_matches_oracle(form):
    from paper_2408_01584_b300 import gd
    sc = small_scene(seed=21)
    fl = gd.GD_TERM_COLLISION | gd.GD_TERM_OFFROAD | gd.GD_AUTO_RESET | (gd.GD_BATCHED if form == "fused" else 0)
    env = gd.Env(sc, k_road=32, n_partners=8, episode_len=12, dynamics=gd.GD_DYN_INVERTIBLE, flags=fl)
    orc = Oracle(sc, OracleConfig(k_road=32, n_partners=8, episode_len=12, term_collision=True, term_offroad=True,
                                  auto_reset=True, dynamics=1))
    T = 16                                    # crosses one episode end (auto-reset)
    acts = _curv_actions(T, sc.num_agents, 21)
    ex = parity.Exceptions()
    cpu = lambda t: t.detach().cpu().numpy()
    for t in range(T):
        s_pre, f_pre, t_pre = [cpu(x) for x in env.get_state()]
        env.step(torch.from_numpy(acts[t]).cuda())
        env.sync()
        s_post, f_post, t_post = [cpu(x) for x in env.get_state()]
        orc.set_state(s_pre, f_pre, t_pre)
        orc.step(acts[t])
        active = (f_pre & gd.GD_FLAG_DONE) == 0
        parity.check_state(s_post, orc.get_state()[0], active, ex, t)
        orc.set_state(s_pre, f_pre, t_pre)
        o = orc.step_post(s_post)
        o["flags"] = orc.get_state()[1]
        parity.check_decisions(dict(flags=f_post, reward=cpu(env.reward), done=cpu(env.done),
                                    world_done=cpu(env.world_done)), o, ex, t)
    env.close()


def test_invertible_fused_equals_per_stage():
    from paper_2408_01584_b300 import gd
    sc = small_scene(seed=22)
    T = 10
    acts = torch.from_numpy(_curv_actions(T, sc.num_agents, 22)).cuda().contiguous()
    outs = []
    for batched in (0, gd.GD_BATCHED):
        env = gd.Env(sc, k_road=32, n_partners=8, dynamics=gd.GD_DYN_INVERTIBLE,
                     flags=gd.GD_TERM_COLLISION | batched)
        obs = torch.empty(T, sc.num_agents, env.F, device="cuda")
        gd.gd_rollout(env.h, T, acts, obs, True)
        s, f, _ = env.get_state()
        env.sync()
        outs.append((s.cpu(), f.cpu(), obs.cpu()))
        env.close()
    for a, b in zip(*outs):
        assert torch.equal(a, b)


def _trajectories(model, n, T, seed, L):
    """float64 trajectories of the oracle's model from random states/actions."""
    rng = np.random.default_rng(seed)
    cfg = OracleConfig(dynamics=model)
    s = np.column_stack([rng.uniform(-150, 150, n), rng.uniform(-150, 150, n), rng.uniform(-3, 3, n),
                         rng.uniform(1, 15, n)])
    steer = (0.2 if model == 1 else 0.6)
    out = [s]
    for _ in range(T):
        a = np.column_stack([rng.uniform(-2, 2, n), rng.uniform(-steer, steer, n)])
        out.append(bicycle(cfg, out[-1], a, L))
    return np.stack(out)


@pytest.mark.parametrize("model", [0, 1])
def test_invert_matches_oracle(model):
    from paper_2408_01584_b300 import gd
    sc = small_scene(seed=23)
    A, T = sc.num_agents, 25
    L = sc.length.astype(np.float64)
    traj = _trajectories(model, A, T, 23, L).astype(np.float32)
    traj[T // 2:, : A // 2, 2] = (traj[T // 2:, : A // 2, 2] + np.float32(math.pi)) % np.float32(2 * math.pi) \
        - np.float32(math.pi)                              # half the agents with wrapped headings
    env = gd.Env(sc, dynamics=model)
    act = torch.empty(T, A, 2, device="cuda")
    gd.gd_invert_actions(env.h, T, torch.from_numpy(traj).cuda(), act)
    env.sync()
    got = act.cpu().numpy()
    ref = invert(OracleConfig(dynamics=model), traj.astype(np.float64), L)
    # float32 differences of float32 states: accel to ~ulp(v)/dt, steer to ~ulp(theta)/distance
    np.testing.assert_allclose(got[..., 0], ref[..., 0], rtol=1e-5, atol=2e-5)
    np.testing.assert_allclose(got[..., 1], ref[..., 1], rtol=1e-4, atol=1e-5)
    env.close()


def test_round_trip_on_the_gpu():
    """Library-stepped trajectory -> gd_invert_actions -> the same actions;
    replaying them reproduces the trajectory."""
    from paper_2408_01584_b300 import gd
    sc = small_scene(seed=24)
    A, T = sc.num_agents, 30
    env = gd.Env(sc, goal_radius=0.0, dynamics=gd.GD_DYN_INVERTIBLE)   # nothing ends: every agent moves
    acts = _curv_actions(T, A, 24)
    acts[:, :, 0] *= 0.25
    acts_d = torch.from_numpy(acts).cuda()
    states = torch.empty(T + 1, A, 4, device="cuda")
    states[0] = env.get_state()[0]
    for t in range(T):
        env.step(acts_d[t])
        states[t + 1] = env.get_state()[0]
    rec = torch.empty(T, A, 2, device="cuda")
    gd.gd_invert_actions(env.h, T, states, rec)
    env.sync()
    r = rec.cpu().numpy()
    ds = states[:-1, :, 3].cpu().numpy() * 0.1
    moving = np.abs(ds) > 0.05
    np.testing.assert_allclose(r[..., 0], acts[..., 0], rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(r[..., 1][moving], acts[..., 1][moving], rtol=1e-3, atol=1e-4)
    # replay the recovered actions
    gd.gd_reset(env.h)
    for t in range(T):
        env.step(rec[t])
    s_end = env.get_state()[0]
    env.sync()
    np.testing.assert_allclose(s_end.cpu().numpy(), states[-1].cpu().numpy(), rtol=1e-4, atol=2e-3)
    env.close()


def test_invert_full_size_workload_sampled():
    from paper_2408_01584_b300 import gd
    sc = scenes.workload_scene("plain_1024x64", 0)
    A, T = sc.num_agents, 91
    env = gd.Env(sc, goal_radius=0.0, dynamics=gd.GD_DYN_INVERTIBLE, flags=gd.GD_BATCHED)
    acts = _curv_actions(T, A, 3)
    acts_d = torch.from_numpy(acts).cuda()
    states = torch.empty(T + 1, A, 4, device="cuda")
    states[0] = env.get_state()[0]
    for t in range(T):
        env.step(acts_d[t])
        states[t + 1] = env.get_state()[0]
    rec = torch.empty(T, A, 2, device="cuda")
    gd.gd_invert_actions(env.h, T, states, rec)
    env.sync()
    sample = np.sort(np.random.default_rng(3).choice(A, 2000, replace=False))
    traj = states.cpu().numpy()[:, sample].astype(np.float64)
    ref = invert(OracleConfig(dynamics=1), traj, 4.5)
    got = rec.cpu().numpy()[:, sample]
    np.testing.assert_allclose(got[..., 0], ref[..., 0], rtol=1e-5, atol=2e-5)
    np.testing.assert_allclose(got[..., 1], ref[..., 1], rtol=1e-4, atol=1e-4)
    env.close()
