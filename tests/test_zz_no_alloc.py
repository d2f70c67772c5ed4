"""gd_collide_noalloc: the collision query for callers that cannot allocate
device memory (their GPU memory belongs to another pool allocator, or their
loop cannot take the synchronisation of cudaMalloc / cudaFree).

It must give the same per-agent collision flags as gd_step records in
GD_FLAG_COLLIDED for the same state, on consecutive calls (its working array
is shared by every call and keeps the previous call's contents), and must
refuse inputs larger than its fixed working array.  Kept in its own file,
collected last.
"""
import numpy as np
import pytest

from paper_2408_01584_b300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup():
    from paper_2408_01584_b300 import gd
    from paper_2408_01584_b300.build import build
    build()
    # crowded worlds so that many boxes overlap; no termination, so collided
    # agents stay in the scene
    sc = scenes.make_scene(np.array([60, 128, 45, 1, 0, 90]), np.array([300, 400, 240, 100, 50, 500]), 13, n_poly=2)
    env = gd.Env(sc, k_road=16, n_partners=8, episode_len=50)
    extent = torch.from_numpy(np.stack([sc.length, sc.width], 1).astype(np.float32)).cuda().contiguous()
    return gd, sc, env, extent


def test_matches_gd_step_on_consecutive_calls():
    gd, sc, env, extent = _setup()
    acts = scenes.make_actions(4, sc.num_agents, 5)
    cell = 5.0            # >= the 4.92 m box diagonal
    out = torch.full((sc.num_agents,), 7, dtype=torch.uint8, device="cuda")
    calls = 0
    for t in range(4):
        _, f_pre, _ = env.get_state()
        active = ((f_pre & gd.GD_FLAG_DONE) == 0).to(torch.uint8).contiguous()
        env.step(torch.from_numpy(acts[t]).cuda())
        state, f_post, _ = env.get_state()
        torch.cuda.synchronize()
        gd.gd_collide_noalloc(sc.agent_off, state, extent, active, cell, out,
                              torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        calls += 1
        got = out.cpu().numpy()
        exp = ((f_post.cpu().numpy() & gd.GD_FLAG_COLLIDED) != 0).astype(np.uint8)
        act = active.cpu().numpy().astype(bool)
        np.testing.assert_array_equal(got[act], exp[act], err_msg=f"step {t}")
        assert (got[~act] == 0).all()
        assert exp[act].sum() > 5            # the scene does collide
    assert calls == 4
    env.close()


def test_null_active_means_all_agents():
    gd, sc, env, extent = _setup()
    env.step(torch.zeros(sc.num_agents, 2, device="cuda"))
    state, f_post, _ = env.get_state()
    out = torch.empty(sc.num_agents, dtype=torch.uint8, device="cuda")
    for _ in range(2):
        gd.gd_collide_noalloc(sc.agent_off, state, extent, None, 5.0, out, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        exp = ((f_post.cpu().numpy() & gd.GD_FLAG_COLLIDED) != 0).astype(np.uint8)
        np.testing.assert_array_equal(out.cpu().numpy(), exp)
    env.close()


def test_rejects_sizes_beyond_the_working_array():
    from paper_2408_01584_b300 import gd
    state = torch.zeros(4, 4, device="cuda")
    extent = torch.ones(4, 2, device="cuda")
    out = torch.zeros(4, dtype=torch.uint8, device="cuda")
    too_many_agents = np.concatenate([[0], np.full(2049, 128)]).cumsum().astype(np.int32)
    with pytest.raises(gd.GdError) as e:
        gd.gd_collide_noalloc(too_many_agents, state, extent, None, 5.0, out)
    assert e.value.status == 4 and "GD_NOALLOC_MAX_AGENTS" in gd.gd_last_error(None)
    with pytest.raises(gd.GdError) as e:
        gd.gd_collide_noalloc(np.zeros(16386, np.int32), state, extent, None, 5.0, out)
    assert e.value.status == 4 and "GD_NOALLOC_MAX_WORLDS" in gd.gd_last_error(None)
    with pytest.raises(gd.GdError) as e:
        gd.gd_collide_noalloc(np.array([0, 129], np.int32), state, extent, None, 5.0, out)
    assert e.value.status == 4
    with pytest.raises(gd.GdError) as e:
        gd.gd_collide_noalloc(np.array([0, 4], np.int32), state, extent, None, 0.0, out)
    assert e.value.status == 1
