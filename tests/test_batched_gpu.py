"""GPU parity of the batched form (GD_BATCHED: persistent per-world kernel
with the road tile in shared memory, whole rollouts as one CUDA graph)
against the oracle, and bitwise equality with the per-stage form, for both
the split observation (step launch, then a persistent kernel over agents;
the default) and the fused one (obs_split = 0).
"""
import numpy as np
import pytest

from oracle import OracleConfig
from paper_2408_01584_b300 import scenes
from tests._util import small_scene, workload_config
from tests.test_parity_gpu import _np, gd_kwargs, teacher_forced

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _batched(ocfg, **over):
    from paper_2408_01584_b300 import gd
    kw = gd_kwargs(ocfg, **over)
    kw["flags"] |= gd.GD_BATCHED
    return kw


@pytest.mark.parametrize("split", [1, 0])
def test_batched_teacher_forced_ragged_with_resets(split):
    sc = small_scene(seed=3)
    ocfg = OracleConfig(k_road=200, n_partners=63, episode_len=7, term_collision=True, term_offroad=True,
                        auto_reset=True)
    acts = scenes.make_actions(20, sc.num_agents, 3)
    from paper_2408_01584_b300.gd import Env
    env = Env(sc, **_batched(ocfg, obs_split=split))
    from paper_2408_01584_b300 import gd
    assert gd.gd_get_info(env.h).obs_split == split
    _, ex = teacher_forced(sc, ocfg, 20, acts, env=env)
    print("exceptions:", ex.items)


def test_batched_teacher_forced_uneven_subset():
    # 48 worlds of the uneven workload: 1..128 agents, 500..20,000 road points
    # (large worlds exceed the shared-memory tile and read road from global memory)
    sc = scenes.workload_scene("uneven_4096", 0).subset(0, 48)
    ocfg = workload_config("uneven_4096")
    acts = scenes.make_actions(4, sc.num_agents, 0)
    from paper_2408_01584_b300.gd import Env
    env = Env(sc, **_batched(ocfg))
    rng = np.random.default_rng(1)
    agents = np.sort(rng.choice(sc.num_agents, min(600, sc.num_agents), replace=False))
    _, ex = teacher_forced(sc, ocfg, 4, acts, env=env, obs_agents=agents)
    print("exceptions:", len(ex))


def _rollout(sc, kw, acts, mode):
    """Run a rollout; returns per-step (state, flags, reward, done, obs)."""
    from paper_2408_01584_b300 import gd
    env = gd.Env(sc, **kw)
    T = acts.shape[0]
    a = torch.from_numpy(acts).cuda().contiguous()
    out = []
    if mode == "graph":
        obs = torch.zeros(T, env.A, env.F, device="cuda")
        rew = torch.zeros(T, env.A, device="cuda")
        dn = torch.zeros(T, env.A, dtype=torch.uint8, device="cuda")
        gd.gd_rollout(env.h, T, a, obs, True, rew, dn)
        env.sync()
        s, f, _ = env.get_state()
        return dict(obs=_np(obs), reward=_np(rew), done=_np(dn), state=_np(s), flags=_np(f))
    obs_all, rew_all, dn_all = [], [], []
    for t in range(T):
        if mode == "fused":
            gd.gd_step_observe(env.h, a[t], env.reward, env.done, env.world_done, env.obs)
        else:
            env.step(a[t])
            env.observe()
        env.sync()
        obs_all.append(_np(env.obs).copy())
        rew_all.append(_np(env.reward).copy())
        dn_all.append(_np(env.done).copy())
    s, f, _ = env.get_state()
    return dict(obs=np.stack(obs_all), reward=np.stack(rew_all), done=np.stack(dn_all), state=_np(s), flags=_np(f))


@pytest.mark.parametrize("split", [1, 0])
@pytest.mark.parametrize("mode", ["stepwise", "fused", "graph"])
def test_batched_bitwise_equals_plain(mode, split):
    sc = small_scene(seed=9)
    ocfg = OracleConfig(k_road=200, n_partners=63, episode_len=9, term_collision=True, term_offroad=True,
                        auto_reset=True)
    acts = scenes.make_actions(12, sc.num_agents, 9)
    plain = _rollout(sc, gd_kwargs(ocfg), acts, "stepwise")
    bat = _rollout(sc, _batched(ocfg, obs_split=split), acts, mode)
    for k in plain:
        np.testing.assert_array_equal(plain[k], bat[k], err_msg=k)


def test_graph_rollout_replay_and_full_size_agreement():
    # full 1,024 x 64 workload, 5 steps: graph replay (twice, after a reset)
    # equals the per-stage form bit for bit
    from paper_2408_01584_b300 import gd
    sc = scenes.workload_scene("plain_1024x64", 0)
    ocfg = workload_config("plain_1024x64")
    acts = scenes.make_actions(5, sc.num_agents, 0)
    plain = _rollout(sc, gd_kwargs(ocfg), acts, "stepwise")
    env = gd.Env(sc, **_batched(ocfg))
    a = torch.from_numpy(acts).cuda().contiguous()
    obs = torch.zeros(env.A, env.F, device="cuda")
    rew = torch.zeros(5, env.A, device="cuda")
    for rep in range(2):
        gd.gd_reset(env.h, None)
        gd.gd_rollout(env.h, 5, a, obs, False, rew, None)
        env.sync()
        np.testing.assert_array_equal(_np(obs), plain["obs"][-1])
        np.testing.assert_array_equal(_np(rew), plain["reward"])
        s, f, _ = env.get_state()
        np.testing.assert_array_equal(_np(s), plain["state"])


@pytest.mark.parametrize("cell,block,topk,notile,split", [(6.0, 128, 2, 0, 1), (8.0, 512, 1, 0, 0), (12.0, 256, 2, 0, 1),
                                                          (10.0, 512, 2, 0, 0), (8.0, 256, 1, 1, 1), (12.0, 128, 2, 1, 0),
                                                          (8.0, 128, 1, 1, 0), (6.0, 512, 2, 1, 1)])
def test_tuning_choices_do_not_change_results(cell, block, topk, notile, split):
    # road grid cell, CTA size, top-K strategy, the road tile and the split
    # observation are performance choices only
    sc = small_scene(seed=12)
    ocfg = OracleConfig(k_road=200, n_partners=63, episode_len=9, term_collision=True, term_offroad=True,
                        auto_reset=True)
    acts = scenes.make_actions(10, sc.num_agents, 12)
    plain = _rollout(sc, gd_kwargs(ocfg), acts, "stepwise")
    bat = _rollout(sc, _batched(ocfg, road_cell=cell, block_size=block, topk_strategy=topk, road_no_tile=notile,
                                obs_split=split), acts, "fused")
    for k in plain:
        np.testing.assert_array_equal(plain[k], bat[k], err_msg=k)


@pytest.mark.parametrize("split", [1, 0])
def test_index_outputs_split_and_fused(split):
    # gd_observe with road / partner index outputs, batched, equals the per-stage form
    from paper_2408_01584_b300 import gd
    sc = small_scene(seed=14)
    ocfg = OracleConfig(k_road=200, n_partners=63, episode_len=9, term_collision=True, term_offroad=True,
                        auto_reset=True)
    acts = torch.from_numpy(scenes.make_actions(5, sc.num_agents, 14)).cuda().contiguous()
    outs = []
    for kw in (gd_kwargs(ocfg), _batched(ocfg, obs_split=split)):
        env = gd.Env(sc, **kw)
        res = []
        for t in range(5):
            env.step(acts[t])
            res.append([_np(x).copy() for x in env.observe(with_idx=True)])
        env.sync()
        outs.append(res)
        env.close()
    for a, b in zip(*outs):
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)


def test_autotune_then_rollout_matches_plain():
    from paper_2408_01584_b300 import gd
    sc = scenes.workload_scene("plain_4x8", 1)
    ocfg = workload_config("plain_4x8")
    acts = scenes.make_actions(ocfg.episode_len, sc.num_agents, 1)
    plain = _rollout(sc, gd_kwargs(ocfg), acts, "stepwise")
    env = gd.Env(sc, **_batched(ocfg))
    before = [_np(x).copy() for x in env.get_state()]
    gd.gd_autotune(env.h)
    after = [_np(x) for x in env.get_state()]
    for b, a in zip(before, after):
        np.testing.assert_array_equal(b, a)           # the tuner leaves the state as it was
    info = gd.gd_get_info(env.h)
    assert info.block_size in (128, 256, 512) and info.topk_strategy in (1, 2) and info.road_cell >= 3.3
    assert info.obs_split in (0, 1)
    a = torch.from_numpy(acts).cuda().contiguous()
    obs = torch.zeros(ocfg.episode_len, env.A, env.F, device="cuda")
    rew = torch.zeros(ocfg.episode_len, env.A, device="cuda")
    dn = torch.zeros(ocfg.episode_len, env.A, dtype=torch.uint8, device="cuda")
    gd.gd_rollout(env.h, ocfg.episode_len, a, obs, True, rew, dn)
    env.sync()
    np.testing.assert_array_equal(_np(obs), plain["obs"])
    np.testing.assert_array_equal(_np(rew), plain["reward"])
    print("autotuned:", info.block_size, info.road_cell, info.topk_strategy)


@pytest.mark.parametrize("split", [1, 0])
def test_rollout_host_equals_device_rollout(split):
    """gd_rollout_host (pinned host actions / rewards / done, copies overlapped
    with the steps) gives the same results as gd_rollout on device buffers
    (split form), with the split or the fused observation."""
    from paper_2408_01584_b300 import gd
    sc = small_scene(seed=31)
    ocfg = OracleConfig(k_road=64, n_partners=16, episode_len=9, term_collision=True, term_offroad=True,
                        auto_reset=True)
    T, A = 21, sc.num_agents                     # three copy chunks of 8, the last one partial
    acts = scenes.make_actions(T, A, 31)
    outs = []
    for host in (False, True):
        env = gd.Env(sc, **_batched(ocfg, obs_split=split if host else 1))
        if host:
            a_h = torch.from_numpy(acts).pin_memory()
            r_h = torch.empty(T, A).pin_memory()
            d_h = torch.empty(T, A, dtype=torch.uint8).pin_memory()
            for _ in range(2):                   # the second call replays the captured graph
                gd.gd_reset(env.h)
                gd.gd_rollout_host(env.h, T, a_h, env.obs, r_h, d_h)
            env.sync()
            r, d = r_h.clone(), d_h.clone()
            with pytest.raises(ValueError):                                    # the binding refuses pageable memory
                gd.gd_rollout_host(env.h, T, torch.from_numpy(acts), env.obs)
            import ctypes
            st = gd.load_library().gd_rollout_host(env.h, T, ctypes.c_void_p(acts.ctypes.data),
                                                   ctypes.c_void_p(env.obs.data_ptr()), None, None)
            assert st == 1 and "page-locked" in gd.gd_last_error(env.h)     # and so does the C ABI
        else:
            r = torch.empty(T, A, device="cuda")
            d = torch.empty(T, A, dtype=torch.uint8, device="cuda")
            gd.gd_rollout(env.h, T, torch.from_numpy(acts).cuda(), env.obs, False, r, d)
            env.sync()
            r, d = r.cpu(), d.cpu()
        s, f, t = env.get_state()
        outs.append((r, d, env.obs.cpu(), s.cpu(), f.cpu(), t.cpu()))
        env.close()
    for a, b in zip(*outs):
        assert torch.equal(a, b)


def test_envs_with_different_shared_memory_coexist():
    # a kernel's shared-memory limit belongs to the kernel, not to an env: an
    # env created later with fewer rays, a coarser grid and no road tile must
    # not break the launches of an earlier env that needs more
    from paper_2408_01584_b300 import gd
    sc = small_scene(seed=21)
    ocfg = OracleConfig(k_road=200, n_partners=63, episode_len=9)
    acts = torch.from_numpy(scenes.make_actions(2, sc.num_agents, 21)).cuda().contiguous()

    def run(env):
        env.step(acts[0])
        depth, cls = env.lidar()
        obs = env.observe()[0]
        env.sync()
        return _np(depth).copy(), _np(cls).copy(), _np(obs).copy()

    ref_env = gd.Env(sc, **_batched(ocfg, lidar_rays=3000, road_cell=6.0))
    ref = run(ref_env)
    ref_env.close()
    big = gd.Env(sc, **_batched(ocfg, lidar_rays=3000, road_cell=6.0))
    small = gd.Env(sc, **_batched(ocfg, lidar_rays=64, road_cell=12.0, road_no_tile=1, lidar_no_tile=1))
    run(small)
    for x, y in zip(run(big), ref):
        np.testing.assert_array_equal(x, y)
    big.close()
    small.close()


def test_batched_teacher_forced_fwdbwd_subset_tuned():
    # the forward step at the 8,192-world forward+backward workload's largest
    # shapes (128 agents and 10,000 road points down to 32 and 5,000; K = 200,
    # P = 63), autotuned, teacher-forced against the oracle for 5 steps on a
    # sample of agents
    from paper_2408_01584_b300 import gd
    from paper_2408_01584_b300.gd import Env
    wl = scenes.WORKLOADS["fwdbwd_8192"]
    sc = scenes.make_scene(np.array([128, 96, 64, 32]), np.array([10000, 8300, 6700, 5000]), 2, n_poly=wl["n_poly"])
    ocfg = workload_config("fwdbwd_8192")
    acts = scenes.make_actions(5, sc.num_agents, 2)
    env = Env(sc, **_batched(ocfg))
    gd.gd_autotune(env.h)
    info = gd.gd_get_info(env.h)
    rng = np.random.default_rng(2)
    agents = np.sort(rng.choice(sc.num_agents, 160, replace=False))
    _, ex = teacher_forced(sc, ocfg, 5, acts, env=env, obs_agents=agents)
    print(f"fwdbwd subset forward: split {info.obs_split}, block {info.block_size}, cell {info.road_cell}, "
          f"exceptions {len(ex)}")


@pytest.mark.parametrize("T", [1, 2, 3])
def test_overlapped_graph_short_rollouts(T):
    # the captured split rollout alternates two state buffers (the last step
    # writes the env's own): one, two and three steps, against the
    # per-stage form, and a step taken after the rollout starts from its
    # final state
    sc = small_scene(seed=17)
    ocfg = OracleConfig(k_road=64, n_partners=16, episode_len=9, term_collision=True, term_offroad=True,
                        auto_reset=True)
    acts = scenes.make_actions(T + 1, sc.num_agents, 17)
    plain = _rollout(sc, gd_kwargs(ocfg), acts, "stepwise")
    from paper_2408_01584_b300 import gd
    env = gd.Env(sc, **_batched(ocfg))
    a = torch.from_numpy(acts).cuda().contiguous()
    obs = torch.zeros(T, env.A, env.F, device="cuda")
    rew = torch.zeros(T, env.A, device="cuda")
    gd.gd_rollout(env.h, T, a[:T], obs, True, rew, None)
    env.step(a[T])
    env.observe()
    env.sync()
    np.testing.assert_array_equal(_np(obs), plain["obs"][:T])
    np.testing.assert_array_equal(_np(rew), plain["reward"][:T])
    np.testing.assert_array_equal(_np(env.obs), plain["obs"][T])
    s, f, _ = env.get_state()
    np.testing.assert_array_equal(_np(s), plain["state"])
    env.close()
