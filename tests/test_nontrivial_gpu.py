"""GPU parity of the "all nontrivial" initialisation (Sec. 3.2 "Simulator
sharp-edges") on mixed-type scenes with parked agents, through the C ABI.

* the uncontrolled set equals the oracle's (exceptions only within 1e-5 m of
  the 2 m threshold, where float32 and float64 distances may disagree);
* teacher-forced steps, per-stage and fused: states, decisions (reward,
  done = 1 for uncontrolled agents, end of episode from controlled agents
  only) and observation rows with parked cars among the partners;
* fused and per-stage rollouts bit-identical.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2408_01584_b300 import scenes
from tests._util import workload_config
from tests.test_parity_gpu import gd_kwargs, teacher_forced

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _flags(ocfg, batched):
    from paper_2408_01584_b300 import gd
    return (gd.GD_TERM_COLLISION if ocfg.term_collision else 0) | (gd.GD_TERM_OFFROAD if ocfg.term_offroad else 0) \
        | (gd.GD_AUTO_RESET if ocfg.auto_reset else 0) | gd.GD_NONTRIVIAL_INIT | (gd.GD_BATCHED if batched else 0)


def test_uncontrolled_set_matches_oracle():
    from paper_2408_01584_b300.gd import Env
    sc = scenes.workload_scene("nontrivial_1024x64", 0, worlds=64)
    ocfg = workload_config("nontrivial_1024x64", nontrivial_init=True)
    env = Env(sc, **gd_kwargs(ocfg, flags=_flags(ocfg, False)))
    g = env.get_state()[1].cpu().numpy()
    o = Oracle(sc, ocfg).get_state()[1]
    d = np.hypot(sc.x.astype(np.float64) - sc.goal_x, sc.y.astype(np.float64) - sc.goal_y)
    diff = g != o
    assert (np.abs(d[diff] - 2.0) <= 1e-5).all()
    assert 0.3 < ((g & 16) != 0).mean() < 0.7
    env.close()


@pytest.mark.parametrize("batched", [False, True])
def test_teacher_forced_nontrivial_mixed_types(batched):
    sc = scenes.workload_scene("nontrivial_1024x64", 1, worlds=12)
    ocfg = workload_config("nontrivial_1024x64", nontrivial_init=True, episode_len=9)
    acts = scenes.make_actions(20, sc.num_agents, 1)
    env, ex = teacher_forced(sc, ocfg, 20, acts, obs_every=4, gd_over=dict(flags=_flags(ocfg, batched)))
    f = env.get_state()[1].cpu().numpy()
    assert ((f & 16) != 0).any() and (sc.agent_type == 2).any() and (sc.agent_type == 1).any()
    print("exceptions:", ex.items)
    env.close()


def test_nontrivial_fused_equals_per_stage():
    from paper_2408_01584_b300 import gd
    sc = scenes.workload_scene("nontrivial_1024x64", 2, worlds=32)
    ocfg = workload_config("nontrivial_1024x64", nontrivial_init=True)
    T = 30
    acts = torch.from_numpy(scenes.make_actions(T, sc.num_agents, 2)).cuda().contiguous()
    outs = []
    for batched in (False, True):
        env = gd.Env(sc, **gd_kwargs(ocfg, flags=_flags(ocfg, batched)))
        obs = torch.empty(T, sc.num_agents, env.F, device="cuda")
        rew = torch.empty(T, sc.num_agents, device="cuda")
        done = torch.empty(T, sc.num_agents, dtype=torch.uint8, device="cuda")
        gd.gd_rollout(env.h, T, acts, obs, True, rew, done)
        s, f, t = env.get_state()
        env.sync()
        outs.append([x.cpu() for x in (s, f, t, obs, rew, done)])
        env.close()
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    done = outs[0][5].numpy()
    static = (outs[0][1].numpy() & 16) != 0
    assert (done[:, static] == 1).all()


def test_episode_stats_count_the_flags():
    from paper_2408_01584_b300 import gd
    sc = scenes.workload_scene("nontrivial_1024x64", 3, worlds=40)
    ocfg = workload_config("nontrivial_1024x64", nontrivial_init=True)
    env = gd.Env(sc, **gd_kwargs(ocfg, flags=_flags(ocfg, True)))
    acts = torch.from_numpy(scenes.make_actions(15, sc.num_agents, 3)).cuda()
    pw = torch.empty(sc.num_worlds, gd.GD_STATS, dtype=torch.int32, device="cuda")
    tot = torch.empty(gd.GD_STATS, dtype=torch.int64, device="cuda")
    world = np.repeat(np.arange(sc.num_worlds), np.diff(sc.agent_off))
    for t in range(15):
        env.step(acts[t])
        gd.gd_episode_stats(env.h, pw, tot)
        f = env.get_state()[1].cpu().numpy()
        env.sync()
        cols = [(f & 1) == 0, (f & (1 | 16)) == 0, (f & 2) != 0, (f & 4) != 0, (f & 8) != 0]
        exp = np.stack([np.bincount(world, weights=c, minlength=sc.num_worlds) for c in cols], 1).astype(np.int64)
        np.testing.assert_array_equal(pw.cpu().numpy(), exp)
        np.testing.assert_array_equal(tot.cpu().numpy(), exp.sum(0))
    assert exp[:, 0].sum() > exp[:, 1].sum()        # parked agents are in the scene but not controlled
    env.close()


def test_parked_selections_after_a_retune():
    # The split observation keeps each parked agent's road selection between
    # steps, tagged in its anchor with the road layout.  A retune rebuilds
    # the road blocks (another cell size than the 10 m the env starts with)
    # and restores the anchors it saved before: the kept selections name
    # positions of the old blocks and must not be read.  Rollouts before and
    # after the retune equal the per-stage form's, bit for bit.
    from paper_2408_01584_b300 import gd
    sc = scenes.workload_scene("nontrivial_1024x64", 4, worlds=64)
    ocfg = workload_config("nontrivial_1024x64", nontrivial_init=True)
    T = 12
    acts = torch.from_numpy(scenes.make_actions(T, sc.num_agents, 4)).cuda().contiguous()

    def rollout(env):
        gd.gd_reset(env.h)
        obs = torch.empty(T, sc.num_agents, env.F, device="cuda")
        gd.gd_rollout(env.h, T, acts, obs, True, None, None)
        env.sync()
        return obs.cpu()

    plain = gd.Env(sc, **gd_kwargs(ocfg, flags=_flags(ocfg, False)))
    ref = rollout(plain)
    plain.close()
    env = gd.Env(sc, **gd_kwargs(ocfg, flags=_flags(ocfg, True)), road_cell=10.0, obs_split=1)
    assert torch.equal(rollout(env), ref)
    gd.gd_autotune(env.h)
    info = gd.gd_get_info(env.h)
    assert abs(info.road_cell - 10.0) > 0.5 and info.obs_split == 1
    assert torch.equal(rollout(env), ref)
    env.close()
