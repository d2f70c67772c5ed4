"""Python binding of the C ABI in include/gd.h (argument marshalling only).

Every function has the name of the C entry point it calls.  Device buffers
are torch CUDA tensors (PyTorch provides memory and streams; every step of
the simulation runs in libgd.so's kernels).  A missing library or a call
on a machine without CUDA raises; there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgd.so")

GD_OK = 0
STATUS = {0: "GD_OK", 1: "GD_ERR_INVALID_ARG", 2: "GD_ERR_CUDA", 3: "GD_ERR_OOM", 4: "GD_ERR_CAPACITY",
          5: "GD_ERR_TIMEOUT", 6: "GD_ERR_STATE"}

GD_TERM_COLLISION = 0x1
GD_TERM_OFFROAD = 0x2
GD_AUTO_RESET = 0x4
GD_BATCHED = 0x8
GD_DIFFERENTIABLE = 0x10
GD_NONTRIVIAL_INIT = 0x20

GD_FLAG_DONE, GD_FLAG_GOAL, GD_FLAG_COLLIDED, GD_FLAG_OFFROAD, GD_FLAG_STATIC = 1, 2, 4, 8, 16

# symbols declared in include/gd.h
SYMBOLS = ("gd_default_config", "gd_create", "gd_destroy", "gd_get_info", "gd_reset", "gd_step", "gd_observe",
           "gd_step_observe", "gd_rollout", "gd_rollout_backward", "gd_step_backward", "gd_get_state",
           "gd_set_state", "gd_autotune", "gd_sync", "gd_last_error", "gd_collide_noalloc",
           "gd_rollout_objective", "gd_selftest_timeout", "gd_observe_lidar", "gd_step_observe_lidar",
           "gd_rollout_lidar", "gd_invert_actions", "gd_decimate", "gd_episode_stats", "gd_rollout_host",
           "gd_time_backward", "gd_time_objective", "gd_decimate_scene")

GD_STATS = 5   # in the scene, controlled in the scene, goal, collided, off-road

DECIMATE_AREA = 1e-3     # m^2, default tolerance of decimate_scene (10-15x on 0.1 m-sampled roads)

GD_DYN_BICYCLE, GD_DYN_INVERTIBLE = 0, 1

GD_MAX_LIDAR_RAYS = 8192
LIDAR_NONE, LIDAR_AGENT, LIDAR_ROAD_EDGE = 0, 1, 2


class GdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class gd_config(C.Structure):
    _fields_ = [("k_road", C.c_int32), ("n_partners", C.c_int32), ("episode_len", C.c_int32),
                ("ckpt_every", C.c_int32), ("obs_radius", C.c_float), ("goal_radius", C.c_float),
                ("dt", C.c_float), ("v_max", C.c_float), ("collision_penalty", C.c_float),
                ("offroad_penalty", C.c_float), ("smooth_c", C.c_float), ("flags", C.c_uint32),
                ("block_size", C.c_int32), ("road_cell", C.c_float), ("topk_strategy", C.c_int32),
                ("lidar_rays", C.c_int32), ("lidar_fov", C.c_float), ("lidar_block_size", C.c_int32),
                ("lidar_no_tile", C.c_int32), ("lidar_split", C.c_int32), ("dynamics", C.c_int32),
                ("nontrivial_dist", C.c_float), ("road_no_tile", C.c_int32), ("obs_split", C.c_int32),
                ("adjoint_split", C.c_int32), ("adjoint_recompute", C.c_int32)]


class gd_scene_batch(C.Structure):
    _fields_ = [("num_worlds", C.c_int32), ("agent_off", C.c_void_p), ("road_off", C.c_void_p),
                ("x", C.c_void_p), ("y", C.c_void_p), ("theta", C.c_void_p), ("v", C.c_void_p),
                ("length", C.c_void_p), ("width", C.c_void_p), ("goal_x", C.c_void_p),
                ("goal_y", C.c_void_p), ("agent_type", C.c_void_p), ("road_x", C.c_void_p),
                ("road_y", C.c_void_p), ("road_type", C.c_void_p), ("road_poly", C.c_void_p)]


class gd_info(C.Structure):
    _fields_ = [("num_worlds", C.c_int32), ("num_agents", C.c_int32), ("num_road", C.c_int32),
                ("feat", C.c_int32), ("max_agents_per_world", C.c_int32), ("k_road", C.c_int32),
                ("n_partners", C.c_int32), ("episode_len", C.c_int32), ("device_bytes", C.c_int64),
                ("block_size", C.c_int32), ("road_cell", C.c_float), ("topk_strategy", C.c_int32),
                ("lidar_rays", C.c_int32), ("lidar_fov", C.c_float), ("lidar_block_size", C.c_int32),
                ("lidar_road_tile", C.c_int32), ("lidar_split", C.c_int32),
                ("road_tile", C.c_int32), ("obs_split", C.c_int32), ("adjoint_split", C.c_int32),
                ("adjoint_road_tile", C.c_int32), ("objective_graph_kernels", C.c_int32),
                ("objective_graph_other", C.c_int32), ("backward_graph_kernels", C.c_int32),
                ("backward_graph_other", C.c_int32), ("adjoint_recompute", C.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libgd.so (built by paper_2408_01584_b300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run paper_2408_01584_b300.build.build() (nvcc, sm_103a)")
    lib = C.CDLL(path)
    vp, i32, f32 = C.c_void_p, C.c_int32, C.c_float
    lib.gd_default_config.argtypes = [C.POINTER(gd_config)]
    lib.gd_default_config.restype = None
    lib.gd_create.argtypes = [C.POINTER(gd_config), C.POINTER(gd_scene_batch), vp, C.POINTER(vp)]
    lib.gd_destroy.argtypes = [vp]
    lib.gd_get_info.argtypes = [vp, C.POINTER(gd_info)]
    lib.gd_reset.argtypes = [vp, vp]
    lib.gd_step.argtypes = [vp, vp, vp, vp, vp]
    lib.gd_observe.argtypes = [vp, vp, vp, vp]
    lib.gd_step_observe.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.gd_rollout.argtypes = [vp, i32, vp, vp, i32, vp, vp]
    lib.gd_rollout_backward.argtypes = [vp, vp, f32, vp, vp, vp]
    lib.gd_rollout_objective.argtypes = [vp, i32, vp, vp, f32, vp, vp]
    lib.gd_selftest_timeout.argtypes = [vp, i32]
    lib.gd_step_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.gd_get_state.argtypes = [vp, vp, vp, vp]
    lib.gd_set_state.argtypes = [vp, vp, vp, vp]
    lib.gd_autotune.argtypes = [vp]
    lib.gd_sync.argtypes = [vp]
    lib.gd_last_error.argtypes = [vp]
    lib.gd_last_error.restype = C.c_char_p
    lib.gd_collide_noalloc.argtypes = [i32, vp, vp, vp, vp, f32, vp, vp]
    lib.gd_observe_lidar.argtypes = [vp, vp, vp, vp]
    lib.gd_step_observe_lidar.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.gd_rollout_lidar.argtypes = [vp, i32, vp, vp, vp, vp, i32, vp, vp]
    lib.gd_invert_actions.argtypes = [vp, i32, vp, vp]
    lib.gd_decimate.argtypes = [i32, i32, vp, vp, vp, f32, vp, vp]
    lib.gd_decimate_scene.argtypes = [C.POINTER(gd_scene_batch), f32, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.gd_episode_stats.argtypes = [vp, vp, vp]
    lib.gd_rollout_host.argtypes = [vp, i32, vp, vp, vp, vp]
    lib.gd_time_backward.argtypes = [vp, vp, f32, vp, vp, vp, vp, vp]
    lib.gd_time_objective.argtypes = [vp, i32, vp, vp, f32, vp, vp, vp, vp]
    for name in SYMBOLS:
        fn = getattr(lib, name)
        if name not in ("gd_default_config", "gd_last_error"):
            fn.restype = C.c_int
    _lib = lib
    return lib


def _check(lib, env, st):
    if st != GD_OK:
        msg = lib.gd_last_error(env)
        raise GdError(st, msg.decode() if msg else "")


def _ptr(t, dtype=None, numel=None, align=None):
    """Device pointer of a torch CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    p = t.data_ptr()
    if align and p % align:
        raise ValueError(f"tensor must be {align}-byte aligned")
    return C.c_void_p(p)


def gd_default_config(**over) -> gd_config:
    lib = load_library()
    c = gd_config()
    lib.gd_default_config(C.byref(c))
    for k, v in over.items():
        setattr(c, k, v)
    return c


def gd_create(cfg: gd_config, scene, stream=None):
    """Upload a ``scenes.Scene`` (host numpy arrays); returns the env handle."""
    lib = load_library()
    arrs = _scene_arrays(scene)
    sb = gd_scene_batch(num_worlds=scene.num_worlds, **{k: a.ctypes.data for k, a in arrs.items()})
    env = C.c_void_p()
    st = lib.gd_create(C.byref(cfg), C.byref(sb), C.c_void_p(stream or 0), C.byref(env))
    _check(lib, None, st)
    return env


def gd_destroy(env):
    load_library().gd_destroy(env)


def gd_get_info(env) -> gd_info:
    lib = load_library()
    info = gd_info()
    _check(lib, env, lib.gd_get_info(env, C.byref(info)))
    return info


def gd_reset(env, world_mask=None):
    lib = load_library()
    _check(lib, env, lib.gd_reset(env, _ptr(world_mask)))


def gd_step(env, actions, reward=None, done=None, world_done=None):
    lib = load_library()
    _check(lib, env, lib.gd_step(env, _ptr(actions), _ptr(reward), _ptr(done), _ptr(world_done)))


def gd_observe(env, obs, road_idx=None, partner_idx=None):
    lib = load_library()
    _check(lib, env, lib.gd_observe(env, _ptr(obs, align=16), _ptr(road_idx), _ptr(partner_idx)))


def gd_step_observe(env, actions, reward, done, world_done, obs):
    lib = load_library()
    _check(lib, env, lib.gd_step_observe(env, _ptr(actions), _ptr(reward), _ptr(done), _ptr(world_done),
                                         _ptr(obs, align=16)))


def gd_rollout(env, steps, actions, obs, obs_per_step=False, reward=None, done=None):
    lib = load_library()
    _check(lib, env, lib.gd_rollout(env, int(steps), _ptr(actions), _ptr(obs, align=16), int(bool(obs_per_step)),
                                    _ptr(reward), _ptr(done)))


def gd_observe_lidar(env, head, depth, cls=None):
    lib = load_library()
    _check(lib, env, lib.gd_observe_lidar(env, _ptr(head, align=4), _ptr(depth, align=4), _ptr(cls)))


def gd_step_observe_lidar(env, actions, head, reward, done, world_done, depth, cls=None):
    lib = load_library()
    _check(lib, env, lib.gd_step_observe_lidar(env, _ptr(actions, align=8), _ptr(head, align=4), _ptr(reward),
                                               _ptr(done), _ptr(world_done), _ptr(depth, align=4), _ptr(cls)))


def gd_rollout_lidar(env, steps, actions, head, depth, cls=None, obs_per_step=False, reward=None, done=None):
    lib = load_library()
    _check(lib, env, lib.gd_rollout_lidar(env, int(steps), _ptr(actions, align=8), _ptr(head, align=4),
                                          _ptr(depth, align=4), _ptr(cls), int(bool(obs_per_step)), _ptr(reward),
                                          _ptr(done)))


def gd_invert_actions(env, steps, states, actions):
    """Expert actions [steps, A, 2] of trajectories states [steps+1, A, 4]."""
    lib = load_library()
    _check(lib, env, lib.gd_invert_actions(env, int(steps), _ptr(states, align=16), _ptr(actions, align=8)))


def _hptr(t):
    """Host pointer of a page-locked CPU tensor (or None)."""
    if t is None:
        return None
    if t.is_cuda or not t.is_pinned() or not t.is_contiguous():
        raise ValueError("expected a contiguous page-locked (pinned) CPU tensor")
    return C.c_void_p(t.data_ptr())


def gd_rollout_host(env, steps, actions_host, obs, reward_host=None, done_host=None):
    """gd_rollout on pinned host tensors (actions [T,A,2], reward [T,A],
    done [T,A]); obs is a CUDA tensor [A,F].  Call gd_sync before reading
    the outputs."""
    lib = load_library()
    _check(lib, env, lib.gd_rollout_host(env, int(steps), _hptr(actions_host), _ptr(obs, align=16),
                                         _hptr(reward_host), _hptr(done_host)))


def gd_episode_stats(env, per_world=None, totals=None):
    """Counts (GD_STATS columns) per world (int32 [W, 5]) and in total (int64 [5])."""
    lib = load_library()
    _check(lib, env, lib.gd_episode_stats(env, _ptr(per_world, align=4), _ptr(totals, align=8)))


def gd_decimate(poly_off, x, y, area_tol, keep, stream=None):
    """Visvalingam-Whyatt keep mask of polylines: poly_off int32 [P+1], x, y
    float [N] and keep uint8 [N] are CUDA tensors."""
    lib = load_library()
    st = lib.gd_decimate(int(poly_off.numel()) - 1, int(x.numel()), _ptr(poly_off, align=4), _ptr(x, align=4),
                         _ptr(y, align=4), float(area_tol), _ptr(keep), C.c_void_p(stream or 0))
    _check(lib, None, st)


def polylines(scene):
    """CSR offsets [P+1] of the scene's polylines: maximal runs of
    consecutive road points of one world with the same polyline id."""
    N = scene.num_road
    brk = np.zeros(N, bool)
    if N:
        brk[0] = True
        brk[1:] = scene.road_poly[1:] != scene.road_poly[:-1]
        brk[scene.road_off[:-1][scene.road_off[:-1] < N]] = True
    return np.append(np.nonzero(brk)[0], N).astype(np.int32)


def _scene_arrays(scene):
    """Contiguous host arrays of a ``scenes.Scene`` in the C ABI's types."""
    arrs = dict(agent_off=np.ascontiguousarray(scene.agent_off, np.int32),
                road_off=np.ascontiguousarray(scene.road_off, np.int32))
    for k in ("x", "y", "theta", "v", "length", "width", "goal_x", "goal_y", "road_x", "road_y"):
        arrs[k] = np.ascontiguousarray(getattr(scene, k), np.float32)
    arrs["agent_type"] = np.ascontiguousarray(scene.agent_type, np.uint8)
    arrs["road_type"] = np.ascontiguousarray(scene.road_type, np.uint8)
    arrs["road_poly"] = np.ascontiguousarray(scene.road_poly, np.int32)
    return arrs


def decimate_scene(scene, area_tol=DECIMATE_AREA, stream=None):
    """The scene with its road polylines decimated (gd_decimate_scene);
    returns (decimated scene, keep mask uint8 [N] over the original points).
    Road indices of the decimated scene count the kept points in order."""
    import dataclasses
    lib = load_library()
    arrs = _scene_arrays(scene)
    sb = gd_scene_batch(num_worlds=scene.num_worlds, **{k: a.ctypes.data for k, a in arrs.items()})
    N = scene.num_road
    keep = np.zeros(N, np.uint8)
    off = np.zeros(scene.num_worlds + 1, np.int32)
    rx, ry = np.zeros(N, np.float32), np.zeros(N, np.float32)
    rt, rp = np.zeros(N, np.uint8), np.zeros(N, np.int32)
    kept = C.c_int32(0)
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    st = lib.gd_decimate_scene(C.byref(sb), float(area_tol), C.c_void_p(stream or 0), p(keep), p(off), p(rx), p(ry),
                               p(rt), p(rp), C.byref(kept))
    _check(lib, None, st)
    m = kept.value
    out = dataclasses.replace(scene, road_x=rx[:m].copy(), road_y=ry[:m].copy(), road_type=rt[:m].copy(),
                              road_poly=rp[:m].copy(), road_off=off)
    return out, keep


def gd_rollout_objective(env, steps, actions, obs_weight, reward_weight, ell, obs=None):
    lib = load_library()
    _check(lib, env, lib.gd_rollout_objective(env, int(steps), _ptr(actions), _ptr(obs_weight, align=16),
                                              float(reward_weight), _ptr(ell), _ptr(obs, align=16)))


def gd_rollout_backward(env, obs_weight, reward_weight, d_ell, d_actions, d_state0=None):
    lib = load_library()
    _check(lib, env, lib.gd_rollout_backward(env, _ptr(obs_weight, align=16), float(reward_weight), _ptr(d_ell),
                                             _ptr(d_actions), _ptr(d_state0)))


GD_BWD_KINDS = 4
BWD_KINDS = ("checkpoint copy", "recomputed step", "adjoint observer side (or fused adjoint)",
             "adjoint per-agent part")


def gd_time_backward(env, obs_weight, reward_weight, d_ell, d_actions, d_state0=None):
    """gd_rollout_backward launch by launch under CUDA events: returns
    (ms [4], launches [4]) per kind (see BWD_KINDS); blocks."""
    lib = load_library()
    ms = (C.c_float * GD_BWD_KINDS)()
    n = (C.c_int32 * GD_BWD_KINDS)()
    _check(lib, env, lib.gd_time_backward(env, _ptr(obs_weight, align=16), float(reward_weight), _ptr(d_ell),
                                          _ptr(d_actions), _ptr(d_state0), ms, n))
    return list(ms), list(n)


GD_OBJ_KINDS = 3
OBJ_KINDS = ("checkpoint copy", "step launch (split form)", "observation launch (or fused step + observation)")


def gd_time_objective(env, steps, actions, obs_weight, reward_weight, ell, obs):
    """gd_rollout_objective launch by launch under CUDA events: returns
    (ms [3], launches [3]) per kind (see OBJ_KINDS); blocks."""
    lib = load_library()
    ms = (C.c_float * GD_OBJ_KINDS)()
    n = (C.c_int32 * GD_OBJ_KINDS)()
    _check(lib, env, lib.gd_time_objective(env, int(steps), _ptr(actions), _ptr(obs_weight, align=16),
                                           float(reward_weight), _ptr(ell), _ptr(obs, align=16), ms, n))
    return list(ms), list(n)


def gd_step_backward(env, actions, d_state_next, d_obs, obs_weight, d_reward_s, d_state, d_actions):
    lib = load_library()
    _check(lib, env, lib.gd_step_backward(env, _ptr(actions), _ptr(d_state_next), _ptr(d_obs), _ptr(obs_weight),
                                          _ptr(d_reward_s), _ptr(d_state), _ptr(d_actions)))


def gd_get_state(env, state=None, flags=None, t=None):
    lib = load_library()
    _check(lib, env, lib.gd_get_state(env, _ptr(state), _ptr(flags), _ptr(t)))


def gd_set_state(env, state=None, flags=None, t=None):
    lib = load_library()
    _check(lib, env, lib.gd_set_state(env, _ptr(state), _ptr(flags), _ptr(t)))


def gd_autotune(env):
    lib = load_library()
    _check(lib, env, lib.gd_autotune(env))


def gd_selftest_timeout(env, wait_us):
    lib = load_library()
    _check(lib, env, lib.gd_selftest_timeout(env, int(wait_us)))


def gd_sync(env):
    lib = load_library()
    _check(lib, env, lib.gd_sync(env))


def gd_last_error(env=None) -> str:
    m = load_library().gd_last_error(env)
    return m.decode() if m else ""


def gd_collide_noalloc(agent_off, state, extent, active, cell, collided, stream=None):
    """Allocation-free collision query: agent_off is a HOST int32 array
    [W+1]; state [A,4], extent [A,2], active [A] (or None) and collided [A]
    are CUDA tensors.  See include/gd.h for who needs it."""
    import torch
    lib = load_library()
    off = np.ascontiguousarray(agent_off, np.int32)
    # the C entry point cannot see the size of a device buffer: a tensor of
    # the wrong dtype or length is refused here, before anything launches
    A = int(off[-1]) if len(off) else 0
    st = lib.gd_collide_noalloc(len(off) - 1, off.ctypes.data_as(C.c_void_p),
                                _ptr(state, dtype=torch.float32, numel=4 * A, align=16),
                                _ptr(extent, dtype=torch.float32, numel=2 * A, align=8),
                                _ptr(active, dtype=torch.uint8, numel=A), float(cell),
                                _ptr(collided, dtype=torch.uint8, numel=A), C.c_void_p(stream or 0))
    _check(lib, None, st)


class Env:
    """Convenience owner of one env handle plus its per-step output tensors."""

    def __init__(self, scene, stream=None, **cfg):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the CUDA library needs a CUDA device")
        self.torch = torch
        self.cfg = gd_default_config(**cfg)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = gd_create(self.cfg, scene, self.stream.cuda_stream)
        info = gd_get_info(self.h)
        self.W, self.A, self.F = info.num_worlds, info.num_agents, info.feat
        self.K, self.P = info.k_road, info.n_partners
        dev = torch.device("cuda", torch.cuda.current_device())
        self.reward = torch.zeros(self.A, dtype=torch.float32, device=dev)
        self.done = torch.zeros(self.A, dtype=torch.uint8, device=dev)
        self.world_done = torch.zeros(self.W, dtype=torch.uint8, device=dev)
        self.obs = torch.zeros(self.A, self.F, dtype=torch.float32, device=dev)
        self.n_rays = info.lidar_rays
        if self.n_rays:
            self.depth = torch.zeros(self.A, self.n_rays, dtype=torch.float32, device=dev)
            self.cls = torch.zeros(self.A, self.n_rays, dtype=torch.uint8, device=dev)
        self.device = dev

    def close(self):
        if self.h:
            gd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, actions):
        gd_step(self.h, actions, self.reward, self.done, self.world_done)

    def observe(self, with_idx=False):
        ri = pi = None
        if with_idx:
            t = self.torch
            ri = t.empty(self.A, self.K, dtype=t.int32, device=self.device)
            pi = t.empty(self.A, self.P, dtype=t.int32, device=self.device)
        gd_observe(self.h, self.obs, ri, pi)
        return self.obs, ri, pi

    def lidar(self, head=None):
        """LiDAR / view-cone scan after the last step: (depth [A, n], cls [A, n])."""
        gd_observe_lidar(self.h, head, self.depth, self.cls)
        return self.depth, self.cls

    def get_state(self):
        t = self.torch
        s = t.empty(self.A, 4, dtype=t.float32, device=self.device)
        f = t.empty(self.A, dtype=t.uint8, device=self.device)
        tt = t.empty(self.W, dtype=t.int32, device=self.device)
        gd_get_state(self.h, s, f, tt)
        return s, f, tt

    def set_state(self, state=None, flags=None, t=None):
        gd_set_state(self.h, state, flags, t)

    def sync(self):
        gd_sync(self.h)
