"""Failure detection without any GPU fault.

* a non-finite action or |steer| >= pi/2 sets the sticky device error word;
  gd_sync reports GD_ERR_INVALID_ARG and clears it, and the env keeps working;
* a bounded device-side wait that runs out (a barrier phase nothing
  completes, a limit of a few milliseconds) reports GD_ERR_TIMEOUT through
  gd_sync and leaves the context usable;
* a misaligned observation pointer is refused before anything is launched.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2408_01584_b300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _env(**kw):
    from paper_2408_01584_b300 import gd
    sc = scenes.workload_scene("plain_4x8", 0)
    return gd, sc, gd.Env(sc, k_road=64, n_partners=7, episode_len=20, **kw)


@pytest.mark.parametrize("batched", [False, True])
def test_bad_actions_reported_at_sync(batched):
    gd, sc, env = _env(flags=gd_flags(batched))
    for bad in (float("nan"), float("inf"), 1.6):
        a = torch.zeros(sc.num_agents, 2, device="cuda")
        a[3, 1 if bad == 1.6 else 0] = bad
        env.step(a)
        with pytest.raises(gd.GdError) as e:
            env.sync()
        assert e.value.status == 1 and "action" in str(e.value)
        env.step(torch.zeros(sc.num_agents, 2, device="cuda"))
        env.sync()                      # cleared; the env still steps
    env.close()


def gd_flags(batched):
    from paper_2408_01584_b300 import gd
    return gd.GD_BATCHED if batched else 0


def test_bounded_wait_times_out_without_fault():
    gd, sc, env = _env()
    gd.gd_selftest_timeout(env.h, 3000)
    with pytest.raises(gd.GdError) as e:
        env.sync()
    assert e.value.status == 5
    # the context is still healthy: step, observe and compare with a fresh env
    a = torch.from_numpy(scenes.make_actions(1, sc.num_agents, 0)[0]).cuda()
    env.step(a)
    obs, _, _ = env.observe()
    env.sync()
    _, _, ref = _env()
    ref.step(a)
    ref_obs, _, _ = ref.observe()
    ref.sync()
    np.testing.assert_array_equal(obs.cpu().numpy(), ref_obs.cpu().numpy())
    env.close()
    ref.close()


def test_misaligned_observation_pointer_is_refused():
    gd, sc, env = _env()
    lib = gd.load_library()
    buf = torch.zeros(sc.num_agents * env.F + 4, device="cuda")
    st = lib.gd_observe(env.h, C.c_void_p(buf.data_ptr() + 4), None, None)
    assert st == 1 and "16-byte" in gd.gd_last_error(env.h)
    st = lib.gd_step(env.h, None, None, None, None)
    assert st == 1
    env.sync()
    env.close()
