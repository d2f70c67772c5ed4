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
    # the capacity checks of the C entry point itself (called through ctypes
    # directly: the binding would refuse these small tensors first)
    import ctypes
    from paper_2408_01584_b300 import gd
    lib = gd.load_library()
    state = torch.zeros(4, 4, device="cuda")
    extent = torch.ones(4, 2, device="cuda")
    out = torch.zeros(4, dtype=torch.uint8, device="cuda")

    def call(off, cell=5.0):
        off = np.ascontiguousarray(off, np.int32)
        return lib.gd_collide_noalloc(len(off) - 1, off.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.c_void_p(state.data_ptr()), ctypes.c_void_p(extent.data_ptr()), None,
                                      ctypes.c_float(cell), ctypes.c_void_p(out.data_ptr()), None)

    too_many_agents = np.concatenate([[0], np.full(2049, 128)]).cumsum()
    assert call(too_many_agents) == 4 and "GD_NOALLOC_MAX_AGENTS" in gd.gd_last_error(None)
    assert call(np.zeros(16386)) == 4 and "GD_NOALLOC_MAX_WORLDS" in gd.gd_last_error(None)
    assert call([0, 129]) == 4
    assert call([0, 4], cell=0.0) == 1
    torch.cuda.synchronize()
    assert (out.cpu().numpy() == 0).all()          # nothing was launched


def test_later_calls_allocate_nothing():
    # after a first call (which loads the module and its array), further
    # calls change neither the device's free memory nor the caching
    # allocator's counts
    gd, sc, env, extent = _setup()
    env.step(torch.zeros(sc.num_agents, 2, device="cuda"))
    state, _, _ = env.get_state()
    out = torch.empty(sc.num_agents, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    gd.gd_collide_noalloc(sc.agent_off, state, extent, None, 5.0, out, stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    stats0 = torch.cuda.memory_stats()
    for _ in range(5):
        gd.gd_collide_noalloc(sc.agent_off, state, extent, None, 5.0, out, stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    stats1 = torch.cuda.memory_stats()
    for k in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
        assert stats1.get(k, 0) == stats0.get(k, 0), k
    env.close()


def test_binding_refuses_wrong_sized_buffers():
    # the C entry point cannot see device buffer sizes; the binding checks
    # dtype and length against agent_off[-1] before anything launches
    from paper_2408_01584_b300 import gd
    off = np.array([0, 3, 4], np.int32)
    state = torch.zeros(4, 4, device="cuda")
    extent = torch.ones(4, 2, device="cuda")
    out = torch.zeros(4, dtype=torch.uint8, device="cuda")
    gd.gd_collide_noalloc(off, state, extent, None, 5.0, out)      # the right sizes pass
    torch.cuda.synchronize()
    bad = [dict(collided=torch.zeros(3, dtype=torch.uint8, device="cuda")),
           dict(state=torch.zeros(4, 4, dtype=torch.float64, device="cuda")),
           dict(state=torch.zeros(3, 4, device="cuda")),
           dict(extent=torch.ones(4, 3, device="cuda")),
           dict(active=torch.ones(5, dtype=torch.uint8, device="cuda")),
           dict(collided=torch.zeros(4, dtype=torch.int32, device="cuda"))]
    for b in bad:
        args = dict(state=state, extent=extent, active=None, collided=out)
        args.update(b)
        with pytest.raises(ValueError):
            gd.gd_collide_noalloc(off, args["state"], args["extent"], args["active"], 5.0, args["collided"])


def test_refuses_a_capturing_stream():
    # a captured call would keep agent_off's host address and read it again
    # at every replay: the entry point refuses and enqueues nothing, and the
    # capture itself stays valid
    from paper_2408_01584_b300 import gd
    off = np.array([0, 3, 4], np.int32)
    state = torch.zeros(4, 4, device="cuda")
    extent = torch.ones(4, 2, device="cuda")
    out = torch.full((4,), 7, dtype=torch.uint8, device="cuda")
    x = torch.zeros(1, device="cuda")
    gd.gd_collide_noalloc(off, state, extent, None, 5.0, out)      # first call before any capture
    torch.cuda.synchronize()
    out.fill_(7)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        graph.capture_begin()
        x.add_(1.0)
        with pytest.raises(gd.GdError) as err:
            gd.gd_collide_noalloc(off, state, extent, None, 5.0, out, side.cuda_stream)
        graph.capture_end()
    assert err.value.status == 1 and "captured" in str(err.value)      # GD_ERR_INVALID_ARG
    graph.replay()
    torch.cuda.synchronize()
    assert x.item() == 1.0
    assert (out.cpu().numpy() == 7).all()
