"""GPU parity of the differentiable rollout (adjoint kernels behind
torch.autograd) against the float64 gradient oracle.

The oracle gradient is taken along the oracle's own float64 trajectory with
its own decisions.  Free-running float32 and float64 trajectories drift
apart by rounding, and sooner or later two nearly equidistant road points
swap ranks: from that step on the two objectives are different piecewise-
smooth functions.  So the objective is truncated (d_ell = 0) where the
GPU's decision trace differs from the oracle's:
  * a flag (collision, off-road, goal, done) changes the trajectory of its
    agent and what the world's other agents see: the whole world's terms are
    dropped from the first step where any of its flags differ;
  * a selection (road points, partners, and their order) only enters the
    observer's own row: that agent's terms are dropped from the first step
    where its own index lists differ.
The gradients of the truncated objectives must agree to GRAD_RTOL.  The
first-divergence steps are reported.
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
    """Per agent: the first step whose objective term may differ between
    the GPU and the oracle (T if none): the first step where a flag of its
    world differs, or where its own selection (road or partner index list)
    differs, whichever comes first."""
    fpre, fpost, ridx, pidx = gpu
    T, A = fpre.shape
    first = lambda d: np.where(d.any(0), np.argmax(d, 0), T)       # [T, n] -> [n]
    flag = (fpre != dec.flags_pre) | (fpost != dec.flags_post)     # [T, A]
    sel = (ridx != dec.road_idx).any(-1) | (pidx != dec.partner_idx).any(-1)
    world = np.repeat(np.arange(sc.num_worlds), np.diff(sc.agent_off))
    wflag = np.zeros((T, sc.num_worlds), bool)
    for t in range(T):
        np.logical_or.at(wflag[t], world, flag[t])
    return np.minimum(first(wflag)[world], first(sel))


def _compare(sc, ocfg, acts, w, wr, d_ell, min_clean, min_steps):
    """Gradient of the objective truncated, per world, at the first step
    where the GPU and oracle decisions differ (d_ell = 0 from there on):
    below that step both follow the same decisions, so both gradients are
    gradients of the same smooth function."""
    from paper_2408_01584_b300 import gd
    from paper_2408_01584_b300.autograd import rollout_objective
    T = acts.shape[0]
    dec = objective_gradient(sc, ocfg, acts, w, wr, d_ell)[3]
    ta = _first_divergence(sc, dec, _gpu_decisions(sc, ocfg, acts))
    keep = (np.arange(T)[:, None] < ta[None, :]).astype(np.float64)
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
        if a1 == a0 or ta[a0:a1].max() < min_steps:
            continue
        sl = slice(a0, a1)
        clean.append(wd)
        m = keep[:, sl] > 0
        np.testing.assert_allclose(ell_g[:, sl][m], ell_o[:, sl][m], rtol=2e-4,
                                   atol=2e-4 * np.abs(ell_o[:, sl][m]).max() + 1e-3)
        ref = max(np.abs(ga_o[:, sl]).max(), np.abs(gs_o[sl]).max())
        err = max(np.abs(g_a[:, sl] - ga_o[:, sl]).max(), np.abs(g_s[sl] - gs_o[sl]).max()) / ref
        worst = max(worst, err)
        assert err <= GRAD_RTOL, (wd, err)
    print(f"gradient parity: {len(clean)} worlds compared; agent-steps compared {int(keep.sum())} of {keep.size} "
          f"(per-agent cut-off median {int(np.median(ta))} of {T}, {int((ta == T).sum())} of {len(ta)} agents to "
          f"the end), max rel err {worst:.2e}")
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


def _fwd_bwd(sc, ocfg, acts, w, wr, d_ell=None, reps=1, tune=False, **over):
    """Objective and gradients through the C ABI: ell [T, A], d_actions
    [T, A, 2], d_state0 [A, 4] of each of `reps` backward calls (the first
    call captures the backward graph in the batched form, later calls
    replay it)."""
    from paper_2408_01584_b300 import gd
    env = gd.Env(sc, **dict(_kw(ocfg), **over))
    if tune:
        gd.gd_autotune(env.h)
    T, A = acts.shape[0], sc.num_agents
    a = torch.from_numpy(acts).cuda().contiguous()
    wt = torch.from_numpy(np.asarray(w, np.float32)).cuda()
    dl = None if d_ell is None else torch.from_numpy(np.asarray(d_ell, np.float32)).cuda()
    ell = torch.empty(T, A, device="cuda")
    outs = []
    for _ in range(reps):
        gd.gd_reset(env.h)
        gd.gd_rollout_objective(env.h, T, a, wt, wr, ell, env.obs)
        da = torch.full((T, A, 2), float("nan"), device="cuda")
        ds = torch.full((A, 4), float("nan"), device="cuda")
        gd.gd_rollout_backward(env.h, wt, wr, dl, da, ds)
        env.sync()
        outs.append((ell.cpu().numpy().copy(), da.cpu().numpy(), ds.cpu().numpy()))
    info = gd.gd_get_info(env.h)
    env.close()
    return outs, info


def test_graph_pair_equals_host_issued_launches():
    # GD_BATCHED replays the objective and the backward pass as two captured
    # CUDA graphs; without it every launch is issued from the host.  Same
    # kernels, same order: bit-identical terms and gradients, and a replay
    # equals the capturing call.
    from paper_2408_01584_b300 import gd
    sc = scenes.make_scene(np.array([6, 9, 17, 1]), np.array([700, 800, 1500, 300]), 12)
    ocfg = OracleConfig(k_road=48, n_partners=7, episode_len=23, term_collision=True, term_offroad=True)
    T = 23        # three segments, the last one partial
    acts = scenes.make_actions(T, sc.num_agents, 12)
    rng = np.random.default_rng(12)
    w = rng.uniform(0, 1, ocfg.feat)
    d_ell = rng.uniform(0.5, 1.5, (T, sc.num_agents))
    host, info_h = _fwd_bwd(sc, ocfg, acts, w, 0.7, d_ell)
    graph, info = _fwd_bwd(sc, ocfg, acts, w, 0.7, d_ell, reps=3, flags=_kw(ocfg)["flags"] | gd.GD_BATCHED)
    for rep in graph:
        for a, b in zip(host[0], rep):
            np.testing.assert_array_equal(a, b)
    assert np.isfinite(host[0][1]).all() and np.isfinite(host[0][2]).all()
    # the graphs hold kernel launches only, no copy or memset node: the
    # objective one launch pair per step (split form) plus a checkpoint copy
    # kernel per segment, the backward per segment a checkpoint copy, the
    # recomputed steps and the adjoint launch pair (split form)
    segs = (T + 9) // 10
    assert info_h.objective_graph_kernels == 0 and info_h.backward_graph_kernels == 0     # nothing captured
    assert info.objective_graph_other == 0 and info.backward_graph_other == 0
    per_step = 2 if info.obs_split else 1
    assert info.objective_graph_kernels == per_step * T + segs
    # (the recomputed steps: one launch per segment from the recorded
    # decisions, else a step launch per step)
    recomputed = segs if info.adjoint_recompute else T
    assert info.backward_graph_kernels == segs + recomputed + (2 * segs if info.adjoint_split else T)


def test_parked_agents_graph_pair_equals_host_issued_launches():
    # With parked agents (the "all nontrivial" initialisation) the batched
    # objective keeps their road selections between steps (and records them
    # for the backward pass); the host-issued plain form selects every step.
    # Terms and gradients are bit-identical.
    from paper_2408_01584_b300 import gd
    sc = scenes.make_scene(np.array([6, 9, 17, 12]), np.array([700, 800, 1500, 900]), 21, parked_frac=0.4)
    ocfg = OracleConfig(k_road=48, n_partners=7, episode_len=23, term_collision=True, term_offroad=True,
                        nontrivial_init=True)
    T = 23
    acts = scenes.make_actions(T, sc.num_agents, 21)
    rng = np.random.default_rng(21)
    w = rng.uniform(0, 1, ocfg.feat)
    host, _ = _fwd_bwd(sc, ocfg, acts, w, 0.7)
    graph, info = _fwd_bwd(sc, ocfg, acts, w, 0.7, reps=2, flags=_kw(ocfg)["flags"] | gd.GD_BATCHED, obs_split=1)
    assert info.obs_split == 1
    for rep in graph:
        for a, b in zip(host[0], rep):
            np.testing.assert_array_equal(a, b)
    assert np.isfinite(host[0][1]).all()


def test_road_rebuild_between_objective_and_backward():
    # The objective rollout records its road selections as positions in the
    # world's road blocks, which the backward pass reads.  A retune between
    # the two rebuilds the blocks (other cell sizes), so the backward pass
    # must select again; it gives the same gradients, and so does the record
    # of an objective rollout taken after the retune.
    from paper_2408_01584_b300 import gd
    sc = scenes.make_scene(np.full(64, 24), np.full(64, 1500), 14)
    ocfg = OracleConfig(k_road=48, n_partners=7, episode_len=12, term_collision=True, term_offroad=True)
    T, A = 12, sc.num_agents
    rng = np.random.default_rng(13)
    a = torch.from_numpy(scenes.make_actions(T, A, 13)).cuda().contiguous()
    wt = torch.from_numpy(rng.uniform(0, 1, ocfg.feat).astype(np.float32)).cuda()
    ell = torch.empty(T, A, device="cuda")
    # a 10 m road cell, which the tuner does not try, so that its final
    # rebuild changes every block's layout
    env = gd.Env(sc, **dict(_kw(ocfg), flags=_kw(ocfg)["flags"] | gd.GD_BATCHED), road_cell=10.0)

    def objective():
        gd.gd_reset(env.h)
        gd.gd_rollout_objective(env.h, T, a, wt, 0.7, ell, env.obs)

    def backward():
        da = torch.full((T, A, 2), float("nan"), device="cuda")
        ds = torch.full((A, 4), float("nan"), device="cuda")
        gd.gd_rollout_backward(env.h, wt, 0.7, None, da, ds)
        env.sync()
        return da.cpu().numpy(), ds.cpu().numpy()

    objective()
    ref = backward()
    objective()
    # tuned from the initial state (the backward pass reads the objective's
    # checkpoints, not the env's state): the split adjoint, which reads the
    # records, and another cell size
    gd.gd_reset(env.h)
    gd.gd_autotune(env.h)
    info = gd.gd_get_info(env.h)
    assert abs(info.road_cell - 10.0) > 0.5 and info.adjoint_split == 1
    retuned = backward()
    objective()
    again = backward()
    env.close()
    assert np.isfinite(ref[0]).all() and np.isfinite(ref[1]).all()
    for got in (retuned, again):
        for x, y in zip(ref, got):
            np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("form", [dict(adjoint_split=0, road_no_tile=0), dict(adjoint_split=0, road_no_tile=1)])
def test_adjoint_forms_are_bit_identical(form):
    # the split adjoint (observer side over agents, then a thread per agent)
    # and the fused per-world kernel, with and without its road tile, sum the
    # same terms in the same order
    from paper_2408_01584_b300 import gd
    sc = scenes.make_scene(np.array([3, 40, 17, 128]), np.array([500, 2500, 1500, 9000]), 13)
    ocfg = OracleConfig(k_road=200, n_partners=63, episode_len=91, term_collision=True, term_offroad=True)
    T = 14
    acts = scenes.make_actions(T, sc.num_agents, 13)
    rng = np.random.default_rng(13)
    w = rng.uniform(0, 1, ocfg.feat)
    d_ell = rng.uniform(0.5, 1.5, (T, sc.num_agents))
    fl = _kw(ocfg)["flags"] | gd.GD_BATCHED
    split, info_s = _fwd_bwd(sc, ocfg, acts, w, 0.7, d_ell, flags=fl, adjoint_split=1)
    fused, info_f = _fwd_bwd(sc, ocfg, acts, w, 0.7, d_ell, flags=fl, **form)
    assert info_s.adjoint_split == 1 and info_f.adjoint_split == 0
    assert info_f.adjoint_road_tile == 1 - form["road_no_tile"]
    for a, b in zip(split[0], fused[0]):
        np.testing.assert_array_equal(a, b)


def _c5_subset(worlds=4, seed=0):
    """Worlds shaped like the 8,192-world forward+backward workload at its
    largest: agents 128 down to 32, road points 10,000 down to 5,000 (the
    workload's generator settings)."""
    wl = scenes.WORKLOADS["fwdbwd_8192"]
    A_w = np.linspace(128, 32, worlds).round().astype(np.int64)
    N_w = np.linspace(10000, 5000, worlds).round().astype(np.int64)
    return scenes.make_scene(A_w, N_w, seed, n_poly=wl["n_poly"])


def test_gradient_fwdbwd_subset_tuned():
    # 4 worlds at the 8,192-world workload's largest shapes (128 agents and
    # 10,000 road points down to 32 and 5,000), K = 200, P = 63, 12 steps,
    # with the autotuned forward and adjoint forms; per world up to its first
    # decision divergence, as above
    from paper_2408_01584_b300 import gd
    from paper_2408_01584_b300.autograd import rollout_objective
    sc = _c5_subset(4, 5)
    ocfg = workload_config("fwdbwd_8192")
    T = 12
    acts = scenes.make_actions(T, sc.num_agents, 5)
    rng = np.random.default_rng(5)
    w = rng.uniform(0, 1, ocfg.feat)
    d_ell = np.ones((T, sc.num_agents))
    dec = objective_gradient(sc, ocfg, acts, w, 1.0, d_ell)[3]
    ta = _first_divergence(sc, dec, _gpu_decisions(sc, ocfg, acts))
    d_cut = d_ell * (np.arange(T)[:, None] < ta[None, :])
    _, ga_o, gs_o, _ = objective_gradient(sc, ocfg, acts, w, 1.0, d_cut, dec=dec)
    env = gd.Env(sc, **dict(_kw(ocfg), flags=_kw(ocfg)["flags"] | gd.GD_BATCHED))
    gd.gd_autotune(env.h)
    info = gd.gd_get_info(env.h)
    a = torch.from_numpy(acts).cuda().requires_grad_(True)
    s0 = torch.from_numpy(sc.state()).cuda().requires_grad_(True)
    ell = rollout_objective(env, a, torch.from_numpy(w.astype(np.float32)).cuda(), 1.0, s0)
    (ell * torch.from_numpy(d_cut.astype(np.float32)).cuda()).sum().backward()
    g_a, g_s = a.grad.cpu().numpy(), s0.grad.cpu().numpy()
    worst, compared = 0.0, 0
    for wd in range(sc.num_worlds):
        sl = slice(sc.agent_off[wd], sc.agent_off[wd + 1])
        if ta[sl].max() < 2:
            continue
        compared += 1
        ref = max(np.abs(ga_o[:, sl]).max(), np.abs(gs_o[sl]).max())
        err = max(np.abs(g_a[:, sl] - ga_o[:, sl]).max(), np.abs(g_s[sl] - gs_o[sl]).max()) / ref
        worst = max(worst, err)
        assert err <= GRAD_RTOL, (wd, err)
    print(f"fwdbwd subset: agents {np.diff(sc.agent_off).tolist()}, agent-steps compared {int(d_cut.sum())} of "
          f"{d_cut.size}, adjoint split {info.adjoint_split} tile {info.adjoint_road_tile}, max rel err {worst:.2e}")
    assert compared >= sc.num_worlds - 1
    env.close()


def _smooth_scene(seed):
    """Worlds where no decision can change along a 91-step rollout of either
    precision, so the objective is one smooth function over the whole
    episode: every road point and every other agent is always inside the
    (2 km) observation radius and every slot list holds all of them (K = 256
    >= road points, P >= agents - 1); goals are 5 km away (never reached);
    no termination, and actions small enough that no speed is clipped."""
    sc = scenes.make_scene(np.array([6, 9, 12, 5]), np.array([200, 180, 240, 150]), seed, n_poly=2)
    sc.goal_x[:] += 5000.0
    return sc


def test_gradient_91_steps_every_segment():
    # 91 steps, ten checkpoint segments, compared in full: the objective's
    # weights are the same for every slot of a kind, so the order of the
    # slots (where float32 and float64 may break near-ties differently) does
    # not change it, and the flag features get weight 0 (collisions are
    # flagged but end nothing)
    sc = _smooth_scene(21)
    ocfg = OracleConfig(k_road=256, n_partners=15, episode_len=91, obs_radius=2000.0)
    T = 91
    acts = scenes.make_actions(T, sc.num_agents, 21)
    acts[..., 0] *= 0.25
    acts[..., 1] *= 0.4
    rng = np.random.default_rng(21)
    w_ego, w_p, w_r = rng.uniform(0, 1, 8), rng.uniform(0, 1, 8), rng.uniform(0, 1, 4)
    w_ego[5:8] = 0.0
    w = np.concatenate([w_ego, np.tile(w_p, ocfg.n_partners), np.tile(w_r, ocfg.k_road)])
    d_ell = rng.uniform(0.5, 1.5, (T, sc.num_agents))
    ell_o, ga_o, gs_o, dec = objective_gradient(sc, ocfg, acts, w, 0.7, d_ell)
    # the decision sets along the oracle's trajectory: every agent sees every
    # road point and every other agent at every step
    nr = np.diff(sc.road_off)[np.repeat(np.arange(sc.num_worlds), np.diff(sc.agent_off))]
    assert ((dec.road_idx >= 0).sum(-1) == nr[None, :]).all()
    assert ((dec.flags_post & 1) == 0).all() and (np.abs(dec.states[..., 3]) < 29.0).all()
    outs, _ = _fwd_bwd(sc, ocfg, acts, w, 0.7, d_ell, obs_radius=2000.0)
    ell_g, g_a, g_s = outs[0]
    np.testing.assert_allclose(ell_g, ell_o, rtol=2e-4, atol=2e-4 * np.abs(ell_o).max())
    ref = max(np.abs(ga_o).max(), np.abs(gs_o).max())
    err_a = np.abs(g_a - ga_o).max(axis=(1, 2)) / ref          # per step
    err_s = np.abs(g_s - gs_o).max() / ref
    seg = [float(err_a[s:s + 10].max()) for s in range(0, T, 10)]
    print(f"91-step gradient, every segment: max rel err per segment {['%.1e' % e for e in seg]}, "
          f"initial state {err_s:.1e}")
    assert max(seg) <= GRAD_RTOL and err_s <= GRAD_RTOL
    # the gradient of the last segment is not trivially zero
    assert np.abs(ga_o[81:]).max() > 1e-3 * ref


def test_timed_passes_equal_the_rollout_calls():
    # gd_time_objective / gd_time_backward (launch by launch under events)
    # compute what gd_rollout_objective / gd_rollout_backward compute, and
    # count their launches per kind
    from paper_2408_01584_b300 import gd
    sc = scenes.make_scene(np.array([6, 9, 17]), np.array([700, 800, 1500]), 14)
    ocfg = OracleConfig(k_road=48, n_partners=7, episode_len=91, term_collision=True, term_offroad=True)
    T = 23
    acts = scenes.make_actions(T, sc.num_agents, 14)
    rng = np.random.default_rng(14)
    w = torch.from_numpy(rng.uniform(0, 1, ocfg.feat).astype(np.float32)).cuda()
    env = gd.Env(sc, **dict(_kw(ocfg), flags=_kw(ocfg)["flags"] | gd.GD_BATCHED))
    a = torch.from_numpy(acts).cuda().contiguous()
    A = sc.num_agents
    outs = []
    for timed in (False, True):
        ell = torch.empty(T, A, device="cuda")
        da = torch.empty(T, A, 2, device="cuda")
        ds = torch.empty(A, 4, device="cuda")
        gd.gd_reset(env.h)
        if timed:
            ms_o, n_o = gd.gd_time_objective(env.h, T, a, w, 0.7, ell, env.obs)
            ms_b, n_b = gd.gd_time_backward(env.h, w, 0.7, None, da, ds)
        else:
            gd.gd_rollout_objective(env.h, T, a, w, 0.7, ell, env.obs)
            gd.gd_rollout_backward(env.h, w, 0.7, None, da, ds)
        env.sync()
        outs.append([x.cpu().numpy() for x in (ell, da, ds)])
    for x, y in zip(*outs):
        np.testing.assert_array_equal(x, y)
    info = gd.gd_get_info(env.h)
    segs = (T + 9) // 10
    assert n_o[0] == segs and n_o[2] == T and n_o[1] == (T if info.obs_split else 0)
    assert n_b[0] == segs and n_b[1] == (segs if info.adjoint_recompute else T)
    assert n_b[2] == (segs if info.adjoint_split else T) and n_b[3] == (segs if info.adjoint_split else 0)
    assert all(m >= 0 for m in ms_o + ms_b) and sum(ms_b) > 0
    env.close()


@pytest.mark.parametrize("batched", [False, True])
@pytest.mark.parametrize("parked", [False, True])
def test_recompute_from_recorded_decisions_is_bit_identical(batched, parked):
    # The backward pass recomputes a checkpoint segment's states in one
    # thread-per-agent launch from the objective rollout's recorded
    # decisions (each step's post-step flags) instead of a step launch per
    # step.  Same states, so bit-identical terms and gradients, with agents
    # that collide, leave the road or reach their goal inside the rollout,
    # and with parked (static) agents.
    from paper_2408_01584_b300 import gd
    sc = scenes.make_scene(np.array([6, 9, 17, 12]), np.array([700, 800, 1500, 900]), 31,
                           parked_frac=0.4 if parked else 0.0)
    ocfg = OracleConfig(k_road=48, n_partners=7, episode_len=23, term_collision=True, term_offroad=True,
                        nontrivial_init=parked)
    T = 23
    acts = scenes.make_actions(T, sc.num_agents, 31)
    rng = np.random.default_rng(31)
    w = rng.uniform(0, 1, ocfg.feat)
    d_ell = rng.uniform(0.5, 1.5, (T, sc.num_agents))
    fl = _kw(ocfg)["flags"] | (gd.GD_BATCHED if batched else 0)
    rec, info_r = _fwd_bwd(sc, ocfg, acts, w, 0.7, d_ell, reps=2, flags=fl)
    ref, info_s = _fwd_bwd(sc, ocfg, acts, w, 0.7, d_ell, flags=fl, adjoint_recompute=0)
    assert info_r.adjoint_recompute == 1 and info_s.adjoint_recompute == 0
    for rep in rec:
        for a, b in zip(ref[0], rep):
            np.testing.assert_array_equal(a, b)
    assert np.isfinite(ref[0][1]).all() and np.isfinite(ref[0][2]).all()
    # the decisions did change inside the rollout: some agents ended early
    env = gd.Env(sc, **dict(_kw(ocfg), flags=fl))
    a = torch.from_numpy(acts).cuda().contiguous()
    done0 = None
    for t in range(T):
        env.step(a[t])
        d = env.done.cpu().numpy().astype(bool)
        if done0 is None:
            done0 = d
    env.close()
    assert (d & ~done0).any()


def test_objective_steps_are_bounded_by_the_episode():
    # the per-step records hold episode_len steps: a longer objective rollout
    # is refused before anything launches (episode_len 23 is not a multiple
    # of the 10-step checkpoint interval)
    from paper_2408_01584_b300 import gd
    sc = scenes.make_scene(np.array([6, 9]), np.array([700, 800]), 3)
    ocfg = OracleConfig(k_road=16, n_partners=7, episode_len=23)
    env = gd.Env(sc, **_kw(ocfg))
    T = 24
    a = torch.zeros(T, sc.num_agents, 2, device="cuda")
    wt = torch.ones(ocfg.feat, device="cuda")
    ell = torch.empty(T, sc.num_agents, device="cuda")
    with pytest.raises(gd.GdError) as err:
        gd.gd_rollout_objective(env.h, T, a, wt, 1.0, ell, env.obs)
    assert err.value.status == 1 and "episode_len" in str(err.value)      # GD_ERR_INVALID_ARG
    gd.gd_rollout_objective(env.h, T - 1, a[: T - 1], wt, 1.0, ell[: T - 1], env.obs)
    env.sync()
    assert np.isfinite(ell[: T - 1].cpu().numpy()).all()
    env.close()


def test_recompute_forms_identical_at_full_fwdbwd_8192():
    # The whole 8,192-world forward+backward workload (658,227 agents,
    # K = 200, P = 63, 91 steps) in the bench's batched form: the backward's
    # one-launch recompute from the recorded flags and the step-kernel
    # recompute give bit-identical objective terms and gradients.
    import hashlib
    from paper_2408_01584_b300 import gd
    name = "fwdbwd_8192"
    sc = scenes.workload_scene(name, 0)
    ocfg = workload_config(name)
    T = ocfg.episode_len
    acts = scenes.make_actions(T, sc.num_agents, 0)
    w = np.random.default_rng(0).uniform(0, 1, ocfg.feat)
    fl = _kw(ocfg)["flags"] | gd.GD_BATCHED
    digests = []
    for rec in (1, 0):
        outs, info = _fwd_bwd(sc, ocfg, acts, w, 1.0, flags=fl, adjoint_recompute=rec)
        assert info.adjoint_recompute == rec
        ell, da, ds = outs[0]
        assert np.isfinite(da).all() and np.isfinite(ds).all() and np.abs(da).max() > 0
        digests.append([hashlib.sha1(np.ascontiguousarray(x).tobytes()).hexdigest() for x in (ell, da, ds)])
        del outs, ell, da, ds
    assert digests[0] == digests[1]
