"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Each step is teacher-forced (see tests/parity.py): state after the bicycle
step, decisions (collision, off-road, goal, reward, done, end of episode)
and the full observation row with its index lists are compared element by
element at sizes that span several grid tiles and a ragged tail, and at the
full 1,024 x 64 workload for sampled steps.
"""
import numpy as np
import pytest

from oracle import Oracle, OracleConfig
from paper_2408_01584_b300 import scenes
from tests import parity
from tests._util import small_scene, tiny_scene, workload_config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def gd_kwargs(c: OracleConfig, **over):
    from paper_2408_01584_b300 import gd
    fl = (gd.GD_TERM_COLLISION if c.term_collision else 0) | (gd.GD_TERM_OFFROAD if c.term_offroad else 0) | \
        (gd.GD_AUTO_RESET if c.auto_reset else 0)
    kw = dict(k_road=c.k_road, n_partners=c.n_partners, episode_len=c.episode_len, obs_radius=c.obs_radius,
              goal_radius=c.goal_radius, dt=c.dt, v_max=c.v_max, collision_penalty=c.collision_penalty,
              offroad_penalty=c.offroad_penalty, smooth_c=c.smooth_c, flags=fl)
    kw.update(over)
    return kw


def _np(t):
    return t.detach().cpu().numpy()


def teacher_forced(scene, ocfg, steps, actions, obs_every=1, obs_agents=None, gd_over=None, env=None):
    from paper_2408_01584_b300.gd import Env
    env = env or Env(scene, **gd_kwargs(ocfg, **(gd_over or {})))
    ora = Oracle(scene, ocfg)
    ex = parity.Exceptions()
    for t in range(steps):
        s_pre, f_pre, t_pre = [_np(x) for x in env.get_state()]
        env.step(torch.from_numpy(np.ascontiguousarray(actions[t])).cuda())
        env.sync()
        s_post, f_post, t_post = [_np(x) for x in env.get_state()]
        g = dict(flags=f_post, reward=_np(env.reward), done=_np(env.done), world_done=_np(env.world_done))
        # dynamics from the GPU's pre-step state
        ora.set_state(s_pre, f_pre, t_pre)
        ora.step(actions[t])
        o_post = ora.get_state()[0]
        parity.check_state(s_post, o_post, np.ones(len(s_post), bool), ex, t)
        np.testing.assert_array_equal(t_post, ora.get_state()[2])
        # decisions on the GPU's post-step state
        ora.set_state(s_pre, f_pre, t_pre)
        o = ora.step_post(s_post)
        o["flags"] = ora.get_state()[1]
        parity.check_decisions(g, o, ex, t)
        if obs_every and (t % obs_every == 0 or t == steps - 1):
            ora.set_state(s_post, f_post, t_post)
            gobs, gri, gpi = env.observe(with_idx=True)
            env.sync()
            oobs, ori, opi = ora.observe()
            parity.check_obs(_np(gobs), _np(gri), _np(gpi), ora, oobs, ori, opi, ocfg.k_road, ocfg.n_partners,
                             ocfg.obs_radius, ex, t, obs_agents)
    return env, ex


def test_initial_observation_plain_4x8():
    sc = scenes.workload_scene("plain_4x8", 0)
    ocfg = workload_config("plain_4x8")
    from paper_2408_01584_b300.gd import Env
    env = Env(sc, **gd_kwargs(ocfg))
    gobs, gri, gpi = env.observe(with_idx=True)
    env.sync()
    ora = Oracle(sc, ocfg)
    oobs, ori, opi = ora.observe()
    ex = parity.Exceptions()
    parity.check_obs(_np(gobs), _np(gri), _np(gpi), ora, oobs, ori, opi, ocfg.k_road, ocfg.n_partners,
                     ocfg.obs_radius, ex, 0)


@pytest.mark.parametrize("seed", [0, 1])
def test_teacher_forced_plain_4x8(seed):
    sc = scenes.workload_scene("plain_4x8", seed)
    ocfg = workload_config("plain_4x8")
    acts = scenes.make_actions(ocfg.episode_len, sc.num_agents, seed)
    _, ex = teacher_forced(sc, ocfg, ocfg.episode_len, acts)
    print("exceptions:", ex.items)


def test_teacher_forced_ragged_with_resets():
    # ragged worlds (1 .. 40 agents, 200 .. 3100 road points), termination on,
    # short episodes so that auto-reset happens several times
    sc = small_scene(seed=3)
    ocfg = OracleConfig(k_road=200, n_partners=63, episode_len=7, term_collision=True, term_offroad=True,
                        auto_reset=True)
    acts = scenes.make_actions(20, sc.num_agents, 3)
    _, ex = teacher_forced(sc, ocfg, 20, acts)
    print("exceptions:", ex.items)


def test_dense_collisions_and_offroad():
    sc = scenes.make_scene(np.array([60, 128, 45]), np.array([300, 400, 240]), 11, n_poly=2)
    ocfg = OracleConfig(k_road=64, n_partners=127, episode_len=30)
    acts = scenes.make_actions(12, sc.num_agents, 1)
    env, ex = teacher_forced(sc, ocfg, 12, acts)
    _, f, _ = env.get_state()
    f = _np(f)
    assert (f & 4).any() and (f & 8).any()      # the scene does exercise both tests


@pytest.mark.parametrize("form", ["per_stage", "batched_edge_grid", "batched_tile"])
def test_edge_worlds(form):
    # an empty world, a world without road, a lone agent far off the map,
    # pedestrians and cyclists, K and P larger than anything in range; the
    # batched forms run every step stage (pair lists included) on worlds of
    # 0 to 3 agents
    far = (5000.0, -3000.0, 0.3, 5.0, 4.5, 2.0, 5050.0, -3000.0, 0)
    ped = (0.0, 0.0, 0.0, 1.0, 0.8, 0.8, 3.0, 0.0, scenes.PEDESTRIAN)
    cyc = (0.0, 3.0, 0.0, 4.0, 1.8, 0.7, 40.0, 3.0, scenes.CYCLIST)
    car = (2.0, 0.0, 0.0, 2.0, 4.5, 2.0, 30.0, 0.0, 0)
    edge = [(-20.0 + k, 1.5, 1, 0) for k in range(41)] + [(-20.0 + k, -4.0, 0, 1) for k in range(41)]
    sc = tiny_scene([([], [(0.0, 0.0, 0, 0), (1.0, 0.0, 0, 0)]), ([car, ped], []), ([far], edge),
                     ([ped, cyc, car], edge)])
    ocfg = OracleConfig(k_road=256, n_partners=127, episode_len=10, term_offroad=True, term_collision=True)
    acts = scenes.make_actions(6, sc.num_agents, 2)
    from paper_2408_01584_b300 import gd
    over = {} if form == "per_stage" else dict(flags=gd_kwargs(ocfg)["flags"] | gd.GD_BATCHED,
                                              road_no_tile=1 if form == "batched_edge_grid" else 0)
    teacher_forced(sc, ocfg, 6, acts, gd_over=over)


def test_zero_slots():
    sc = small_scene(seed=6, worlds=3)
    for k, p in ((0, 5), (7, 0), (0, 0)):
        ocfg = OracleConfig(k_road=k, n_partners=p, episode_len=91)
        acts = scenes.make_actions(2, sc.num_agents, 0)
        teacher_forced(sc, ocfg, 2, acts)


def test_full_size_plain_1024x64_sampled_steps():
    sc = scenes.workload_scene("plain_1024x64", 0)
    ocfg = workload_config("plain_1024x64")
    acts = scenes.make_actions(3, sc.num_agents, 0)
    rng = np.random.default_rng(0)
    agents = np.sort(rng.choice(sc.num_agents, 4096, replace=False))
    _, ex = teacher_forced(sc, ocfg, 3, acts, obs_every=1, obs_agents=agents)
    print("exceptions:", len(ex))


def test_full_size_uneven_4096_sampled_steps():
    # the uneven batch at full size (4,096 worlds, 1 to 128 agents and 500 to
    # 20,000 road points each) in the tuned batched form the bench times:
    # every agent of the worlds with the most agents and with the most road
    # points, and 4,096 agents at random, over three teacher-forced steps
    from paper_2408_01584_b300 import gd
    from paper_2408_01584_b300.gd import Env
    sc = scenes.workload_scene("uneven_4096", 0)
    ocfg = workload_config("uneven_4096")
    acts = scenes.make_actions(3, sc.num_agents, 0)
    env = Env(sc, **gd_kwargs(ocfg, flags=gd_kwargs(ocfg)["flags"] | gd.GD_BATCHED))
    gd.gd_autotune(env.h)
    apw, rpw = np.diff(sc.agent_off), np.diff(sc.road_off)
    worlds = np.unique(np.concatenate([np.argsort(apw)[-8:], np.argsort(rpw)[-8:]]))
    assert apw[worlds].max() == 128 and rpw[worlds].max() > 19000
    big = np.concatenate([np.arange(sc.agent_off[w], sc.agent_off[w + 1]) for w in worlds])
    rng = np.random.default_rng(0)
    agents = np.unique(np.concatenate([big, rng.choice(sc.num_agents, 4096, replace=False)]))
    _, ex = teacher_forced(sc, ocfg, 3, acts, obs_every=1, obs_agents=agents, env=env)
    env.close()
    print("exceptions:", len(ex))


@pytest.mark.parametrize("batched", [False, True])
def test_largest_world(batched):
    # one world at both per-world limits, 128 agents and 32,767 road points:
    # block positions up to 32,766 in the keys' 16-bit position field, a road
    # block (393 KB) too large for a shared-memory tile
    from paper_2408_01584_b300 import gd
    sc = scenes.make_scene(np.array([128]), np.array([32767]), 41)
    ocfg = OracleConfig(k_road=200, n_partners=63, episode_len=91, term_collision=True, term_offroad=True)
    acts = scenes.make_actions(3, sc.num_agents, 41)
    over = dict(flags=gd_kwargs(ocfg)["flags"] | (gd.GD_BATCHED if batched else 0))
    env, ex = teacher_forced(sc, ocfg, 3, acts, obs_every=1, gd_over=over)
    if batched:
        gd.gd_autotune(env.h)
        env, ex2 = teacher_forced(sc, ocfg, 2, acts, obs_every=1, env=env)
    env.close()
    print("exceptions:", len(ex))


def _long_box_scene(seed):
    # one world: horizontal road edges 9 m apart and two vertical ones, each
    # its own polyline, 3 m between points; boxes 5 to 45 m long at headings
    # that put them over 1 to 6 rows of the 8 m edge grid
    rng = np.random.default_rng(seed)
    pts, poly = [], 0
    for k in range(-4, 5):
        pts += [(float(x), 9.0 * k + 0.3, 1, poly) for x in np.arange(-60.0, 61.0, 3.0)]
        poly += 1
    for x0 in (-50.0, 50.0):
        pts += [(x0, float(y), 1, poly) for y in np.arange(-45.0, 46.0, 3.0)]
        poly += 1
    pts += [(float(x), float(y), 0, poly + 1) for x, y in rng.uniform(-55, 55, (200, 2))]
    agents = []
    for q in range(40):
        length = float((5.0, 12.0, 20.0, 30.0, 45.0)[q % 5])
        theta = float((0.0, np.pi / 2, np.pi / 3, 1.2, -np.pi / 2, 2.9)[q % 6])
        x, y = rng.uniform(-40, 40), rng.uniform(-32, 32)
        agents.append((x, y, theta, 1.0, length, 2.5, x + 30.0, y, 0))
    return tiny_scene([(agents, pts)])


@pytest.mark.parametrize("form", ["per_stage", "batched_edge_grid", "batched_tile"])
def test_road_edges_under_long_boxes(form):
    # the road-edge test of boxes that span more cell rows than the step reads
    # up front, against the oracle's test over every edge segment
    from paper_2408_01584_b300 import gd
    sc = _long_box_scene(3)
    ocfg = OracleConfig(k_road=16, n_partners=7, episode_len=91)
    over = {} if form == "per_stage" else dict(flags=gd_kwargs(ocfg)["flags"] | gd.GD_BATCHED,
                                              road_no_tile=1 if form == "batched_edge_grid" else 0)
    acts = scenes.make_actions(6, sc.num_agents, 3)
    env, ex = teacher_forced(sc, ocfg, 6, acts, obs_every=3, gd_over=over)
    flags = _np(env.get_state()[1])
    n_off = int(np.sum((flags & 8) != 0))
    assert 0 < n_off < sc.num_agents, n_off    # both outcomes occur
    print("offroad:", n_off, "exceptions:", ex.items)
    env.close()


def test_free_running_drift_91_steps():
    # the per-step comparisons above are teacher-forced; this one lets the
    # float32 GPU rollout and the float64 oracle each run on their own for a
    # whole 91-step episode of 16 worlds of the 1,024 x 64 workload (same
    # actions) and reports how far the states drift apart, per step, over
    # the agents whose flags have agreed so far (a decision that flips near
    # its cutoff sends an agent on another path, and its world's partners
    # with it, so the world is dropped from that step on)
    from paper_2408_01584_b300.gd import Env
    sc = scenes.workload_scene("plain_1024x64", 0).subset(0, 16)
    ocfg = workload_config("plain_1024x64", auto_reset=False)
    T = 91
    acts = scenes.make_actions(T, sc.num_agents, 0)
    env = Env(sc, **gd_kwargs(ocfg))
    ora = Oracle(sc, ocfg)
    world = np.repeat(np.arange(sc.num_worlds), np.diff(sc.agent_off))
    agree = np.ones(sc.num_worlds, bool)
    pos_err, head_err, kept = [], [], []
    for t in range(T):
        env.step(torch.from_numpy(acts[t]).cuda())
        env.sync()
        ora.step(acts[t])
        gs, gf, _ = [_np(x) for x in env.get_state()]
        os_, of = ora.get_state()[:2]
        bad = np.zeros(sc.num_worlds, bool)
        np.logical_or.at(bad, world, gf != of)
        agree &= ~bad
        m = agree[world] & ((gf & 1) == 0)
        d = np.abs(gs.astype(np.float64) - os_.astype(np.float64))
        pos_err.append(float(np.hypot(d[m, 0], d[m, 1]).max()) if m.any() else 0.0)
        head_err.append(float(d[m, 2].max()) if m.any() else 0.0)
        kept.append(int(agree.sum()))
    print("free-running drift, max position error (m) at steps 1, 10, 30, 60, 91:",
          [f"{pos_err[k]:.2e}" for k in (0, 9, 29, 59, 90)],
          "heading (rad):", [f"{head_err[k]:.2e}" for k in (0, 9, 29, 59, 90)],
          "worlds still agreeing:", [kept[k] for k in (0, 9, 29, 59, 90)])
    assert kept[9] >= 8
    # rounding, not a modelling difference: far below a metre after a whole episode
    assert max(pos_err) < 1e-2 and max(head_err) < 1e-3
    env.close()
