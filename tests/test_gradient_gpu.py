"""GPU parity of the differentiable rollout (adjoint kernels behind
torch.autograd) against the float64 gradient oracle.

The oracle gradient is taken along the oracle's own float64 trajectory with
its own decisions.  Free-running float32 and float64 trajectories drift
apart by rounding, and sooner or later two nearly equidistant road points
swap ranks: from that step on the two objectives are different piecewise-
smooth functions.  So each world's objective is truncated (d_ell = 0) at the
first step where the GPU's decision trace (flags, selected road points and
partners) differs from the oracle's; the gradients of the truncated
objectives must agree to GRAD_RTOL.  The first-divergence steps are
reported.
"""
import numpy as np
import pytest

from oracle import OracleConfig
from oracle.gradient import objective_gradient
from paper_2408_01584_b300 import scenes
from tests._util import workload_config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-4     # max |g_gpu - g_oracle| / max |g_oracle| per world (float32 adjoint vs float64)


def _kw(ocfg):
    from paper_2408_01584_b300 import gd
    fl = gd.GD_DIFFERENTIABLE | (gd.GD_TERM_COLLISION if ocfg.term_collision else 0) | \
        (gd.GD_TERM_OFFROAD if ocfg.term_offroad else 0) | (gd.GD_NONTRIVIAL_INIT if ocfg.nontrivial_init else 0)
    return dict(k_road=ocfg.k_road, n_partners=ocfg.n_partners, episode_len=ocfg.episode_len, flags=fl,
                smooth_c=ocfg.smooth_c, dynamics=ocfg.dynamics)


def _gpu_decisions(sc, ocfg, acts):
    """Flags and index lists of the GPU along its own trajectory."""
    from paper_2408_01584_b300 import gd
    env = gd.Env(sc, **_kw(ocfg))
    T = acts.shape[0]
    fpre, fpost, ridx, pidx = [], [], [], []
    a = torch.from_numpy(acts).cuda()
    for t in range(T):
        fpre.append(env.get_state()[1].cpu().numpy())
        env.step(a[t])
        fpost.append(env.get_state()[1].cpu().numpy())
        _, ri, pi = env.observe(with_idx=True)
        ridx.append(ri.cpu().numpy())
        pidx.append(pi.cpu().numpy())
    env.close()
    return np.stack(fpre), np.stack(fpost), np.stack(ridx), np.stack(pidx)


def _first_divergence(sc, dec, gpu):
    """Per world: the first step at which the GPU's decision trace differs
    from the oracle's (T if never)."""
    fpre, fpost, ridx, pidx = gpu
    T = fpre.shape[0]
    diff = ((fpre != dec.flags_pre) | (fpost != dec.flags_post) | (ridx != dec.road_idx).any(-1)
            | (pidx != dec.partner_idx).any(-1))            # [T, A]
    out = []
    for wd in range(sc.num_worlds):
        d = diff[:, sc.agent_off[wd]:sc.agent_off[wd + 1]].any(-1)
        out.append(int(np.argmax(d)) if d.any() else T)
    return np.array(out)


def _compare(sc, ocfg, acts, w, wr, d_ell, min_clean, min_steps):
    """Gradient of the objective truncated, per world, at the first step
    where the GPU and oracle decisions differ (d_ell = 0 from there on):
    below that step both follow the same decisions, so both gradients are
    gradients of the same smooth function."""
    from paper_2408_01584_b300 import gd
    from paper_2408_01584_b300.autograd import rollout_objective
    T = acts.shape[0]
    dec = objective_gradient(sc, ocfg, acts, w, wr, d_ell)[3]
    tw = _first_divergence(sc, dec, _gpu_decisions(sc, ocfg, acts))
    world = np.repeat(np.arange(sc.num_worlds), np.diff(sc.agent_off))
    keep = (np.arange(T)[:, None] < tw[world][None, :]).astype(np.float64)
    d_cut = d_ell * keep
    ell_o, ga_o, gs_o, _ = objective_gradient(sc, ocfg, acts, w, wr, d_cut, dec=dec)
    env = gd.Env(sc, **_kw(ocfg))
    a = torch.from_numpy(acts).cuda().requires_grad_(True)
    s0 = torch.from_numpy(sc.state()).cuda().requires_grad_(True)
    wt = torch.from_numpy(w.astype(np.float32)).cuda()
    ell = rollout_objective(env, a, wt, wr, s0)
    (ell * torch.from_numpy(d_cut.astype(np.float32)).cuda()).sum().backward()
    g_a, g_s, ell_g = a.grad.cpu().numpy(), s0.grad.cpu().numpy(), ell.detach().cpu().numpy()
    clean, worst = [], 0.0
    for wd in range(sc.num_worlds):
        a0, a1 = sc.agent_off[wd], sc.agent_off[wd + 1]
        if a1 == a0 or tw[wd] < min_steps:
            continue
        sl, n = slice(a0, a1), tw[wd]
        clean.append(wd)
        np.testing.assert_allclose(ell_g[:n, sl], ell_o[:n, sl], rtol=2e-4,
                                   atol=2e-4 * np.abs(ell_o[:n, sl]).max() + 1e-3)
        ref = max(np.abs(ga_o[:, sl]).max(), np.abs(gs_o[sl]).max())
        err = max(np.abs(g_a[:, sl] - ga_o[:, sl]).max(), np.abs(g_s[sl] - gs_o[sl]).max()) / ref
        worst = max(worst, err)
        assert err <= GRAD_RTOL, (wd, err)
    print(f"gradient parity: {len(clean)} worlds compared over their first {min_steps}+ identical-decision steps "
          f"(median {int(np.median(tw))} of {T}), max rel err {worst:.2e}; first-divergence steps: {tw.tolist()}")
    assert len(clean) >= min_clean
    env.close()
    return worst


def test_gradient_small_ragged():
    sc = scenes.make_scene(np.array([5, 8, 3, 12]), np.array([600, 900, 400, 1500]), 4)
    ocfg = OracleConfig(k_road=24, n_partners=5, episode_len=91, term_collision=True, term_offroad=True)
    T = 12
    acts = scenes.make_actions(T, sc.num_agents, 4)
    rng = np.random.default_rng(4)
    w = rng.uniform(0, 1, ocfg.feat)
    d_ell = rng.uniform(0.5, 1.5, (T, sc.num_agents))
    _compare(sc, ocfg, acts, w, 0.7, d_ell, min_clean=2, min_steps=4)


@pytest.mark.parametrize("variant", ["invertible", "nontrivial"])
def test_gradient_model_variants(variant):
    # the simplified invertible model (curvature actions), or the "all
    # nontrivial" initialisation with parked agents (frozen, no reward term)
    inv = variant == "invertible"
    sc = scenes.make_scene(np.array([5, 8, 3, 12]), np.array([600, 900, 400, 1500]), 6,
                           parked_frac=0.0 if inv else 0.4)
    ocfg = OracleConfig(k_road=24, n_partners=5, episode_len=91, term_collision=True, term_offroad=True,
                        dynamics=1 if inv else 0, nontrivial_init=not inv)
    T = 12
    acts = scenes.make_actions(T, sc.num_agents, 6)
    if inv:
        acts[:, :, 1] *= 0.2 / 0.7
    rng = np.random.default_rng(6)
    w = rng.uniform(0, 1, ocfg.feat)
    d_ell = rng.uniform(0.5, 1.5, (T, sc.num_agents))
    _compare(sc, ocfg, acts, w, 0.7, d_ell, min_clean=2, min_steps=4)


def test_gradient_differentiable_workload_91_steps():
    # 64 worlds of the 512 x 32 differentiable workload, 91 steps, checkpoint every 10
    sc = scenes.workload_scene("diff_512x32", 0).subset(0, 64)
    ocfg = workload_config("diff_512x32")
    T = 91
    acts = scenes.make_actions(T, sc.num_agents, 0)
    rng = np.random.default_rng(0)
    w = rng.uniform(0, 1, ocfg.feat)
    _compare(sc, ocfg, acts, w, 1.0, np.ones((T, sc.num_agents)), min_clean=8, min_steps=10)


def test_backward_is_deterministic_and_step_backward_matches():
    from paper_2408_01584_b300 import gd
    sc = scenes.make_scene(np.array([6, 9]), np.array([700, 800]), 5)
    ocfg = OracleConfig(k_road=24, n_partners=5, episode_len=91)
    env = gd.Env(sc, **_kw(ocfg))
    T = 6
    acts = torch.from_numpy(scenes.make_actions(T, sc.num_agents, 5)).cuda().contiguous()
    rng = np.random.default_rng(5)
    w = torch.from_numpy(rng.uniform(0, 1, ocfg.feat).astype(np.float32)).cuda()
    ell = torch.empty(T, sc.num_agents, device="cuda")
    gd.gd_reset(env.h)
    gd.gd_rollout_objective(env.h, T, acts, w, 0.5, ell, env.obs)
    outs = []
    for _ in range(2):
        da = torch.empty(T, sc.num_agents, 2, device="cuda")
        ds = torch.empty(sc.num_agents, 4, device="cuda")
        gd.gd_rollout_backward(env.h, w, 0.5, None, da, ds)
        env.sync()
        outs.append((da.cpu().numpy(), ds.cpu().numpy()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    # one-step adjoint from the initial state equals the T = 1 rollout gradient
    gd.gd_reset(env.h)
    d_state = torch.empty(sc.num_agents, 4, device="cuda")
    d_act = torch.empty(sc.num_agents, 2, device="cuda")
    rew = torch.full((sc.num_agents,), 0.5, device="cuda")
    gd.gd_step_backward(env.h, acts[0], None, None, w, rew, d_state, d_act)
    env.sync()
    _, ga_o, gs_o, _ = objective_gradient(sc, ocfg, acts[:1].cpu().numpy(), w.cpu().numpy().astype(np.float64), 0.5)
    ref = max(np.abs(ga_o).max(), np.abs(gs_o).max())
    assert np.abs(d_act.cpu().numpy() - ga_o[0]).max() / ref < GRAD_RTOL
    assert np.abs(d_state.cpu().numpy() - gs_o).max() / ref < GRAD_RTOL


def _objective_and_gradient(sc, ocfg, acts, w, **over):
    from paper_2408_01584_b300 import gd
    env = gd.Env(sc, **dict(_kw(ocfg), **over))
    T = acts.shape[0]
    ell = torch.empty(T, sc.num_agents, device="cuda")
    obs = torch.empty(sc.num_agents, env.F, device="cuda")
    gd.gd_rollout_objective(env.h, T, acts, w, 0.5, ell, obs)
    da = torch.empty(T, sc.num_agents, 2, device="cuda")
    ds = torch.empty(sc.num_agents, 4, device="cuda")
    gd.gd_rollout_backward(env.h, w, 0.5, None, da, ds)
    env.sync()
    out = [x.cpu().numpy() for x in (ell, obs, da, ds)]
    env.close()
    return out


@pytest.mark.parametrize("T", [1, 7])
def test_split_and_fused_objective_and_gradients_are_identical(T):
    # the split observation completes the objective term the step launch
    # started (r_s), with the fused kernel's rounding: same terms, same rows,
    # same gradients
    sc = scenes.make_scene(np.array([6, 9, 17]), np.array([700, 800, 1500]), 8)
    ocfg = OracleConfig(k_road=48, n_partners=7, episode_len=91)
    acts = torch.from_numpy(scenes.make_actions(T, sc.num_agents, 8)).cuda().contiguous()
    w = torch.from_numpy(np.random.default_rng(8).uniform(0, 1, ocfg.feat).astype(np.float32)).cuda()
    fused = _objective_and_gradient(sc, ocfg, acts, w, obs_split=0)
    split = _objective_and_gradient(sc, ocfg, acts, w, obs_split=1)
    for a, b in zip(fused, split):
        np.testing.assert_array_equal(a, b)


def test_bounded_reselection_equals_full_radius():
    # gd_rollout_backward re-selects each agent's road points inside the disk
    # of the forward step's K-th distance; gd_step_backward re-selects over
    # the full radius: from the same state the gradients are bit-identical
    from paper_2408_01584_b300 import gd
    sc = scenes.make_scene(np.array([12, 20]), np.array([900, 2500]), 9)
    ocfg = OracleConfig(k_road=200, n_partners=15, episode_len=91)
    acts = torch.from_numpy(scenes.make_actions(1, sc.num_agents, 9)).cuda().contiguous()
    w = torch.from_numpy(np.random.default_rng(9).uniform(0, 1, ocfg.feat).astype(np.float32)).cuda()
    env = gd.Env(sc, **_kw(ocfg))
    ell = torch.empty(1, sc.num_agents, device="cuda")
    gd.gd_rollout_objective(env.h, 1, acts, w, 0.5, ell, env.obs)
    da = torch.empty(1, sc.num_agents, 2, device="cuda")
    ds = torch.empty(sc.num_agents, 4, device="cuda")
    gd.gd_rollout_backward(env.h, w, 0.5, None, da, ds)
    gd.gd_reset(env.h)
    d_state = torch.empty(sc.num_agents, 4, device="cuda")
    d_act = torch.empty(sc.num_agents, 2, device="cuda")
    rew = torch.full((sc.num_agents,), 0.5, device="cuda")
    gd.gd_step_backward(env.h, acts[0], None, None, w, rew, d_state, d_act)
    env.sync()
    np.testing.assert_array_equal(da[0].cpu().numpy(), d_act.cpu().numpy())
    np.testing.assert_array_equal(ds.cpu().numpy(), d_state.cpu().numpy())
    env.close()
