"""ctypes front end of the brute-force C++ oracle (test infrastructure).

The arithmetic lives in ``oracle.cpp``; this file builds it with g++, loads
it and marshals numpy arrays.  Nothing here imports the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

TERM_COLLISION = 1
TERM_OFFROAD = 2
AUTO_RESET = 4
NONTRIVIAL_INIT = 32

DONE, GOAL, COLLIDED, OFFROAD, STATIC = 1, 2, 4, 8, 16


def build_oracle(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so next to it (g++, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O3", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-Wall", _SRC,
               "-o", _LIB + ".tmp"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Cfg(C.Structure):
    _fields_ = [("k_road", C.c_int32), ("n_partners", C.c_int32), ("episode_len", C.c_int32),
                ("obs_radius", C.c_double), ("goal_radius", C.c_double), ("dt", C.c_double),
                ("v_max", C.c_double), ("collision_penalty", C.c_double),
                ("offroad_penalty", C.c_double), ("smooth_c", C.c_double), ("flags", C.c_uint32),
                ("dynamics", C.c_int32), ("nontrivial_dist", C.c_double)]


def load_oracle():
    global _lib
    if _lib is None:
        build_oracle()
        lib = C.CDLL(_LIB)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        lib.or_create.restype = vp
        lib.or_create.argtypes = [C.POINTER(_Cfg), C.c_int, i32] + [vp] * 15
        lib.or_destroy.argtypes = [vp]
        lib.or_reset.argtypes = [vp, vp]
        lib.or_step.argtypes = [vp] * 9
        lib.or_step_post.argtypes = [vp] * 9
        lib.or_observe.argtypes = [vp] * 4
        lib.or_observe64.argtypes = [vp] * 4
        lib.or_road_point.argtypes = [vp, i32, i32, vp, vp]
        lib.or_partner.argtypes = [vp, i32, i32, vp, vp]
        lib.or_get_state.argtypes = [vp] * 5
        lib.or_set_state.argtypes = [vp] * 4
        lib.or_bicycle.argtypes = [C.POINTER(_Cfg), i64, vp, vp, vp]
        lib.or_invert.argtypes = [C.POINTER(_Cfg), i32, i64, vp, vp, vp]
        lib.or_decimate.argtypes = [i32, vp, vp, vp, C.c_float, vp]
        lib.or_box_box.restype = C.c_double
        lib.or_box_box.argtypes = [vp, vp]
        lib.or_box_seg.restype = C.c_double
        lib.or_box_seg.argtypes = [vp, vp]
        lib.or_lidar.argtypes = [vp, i32, C.c_double, vp, vp, i32, C.c_double, vp, vp, vp, vp]
        lib.or_num_threads.restype = C.c_int
        _lib = lib
    return _lib


@dataclasses.dataclass
class OracleConfig:
    """Simulator settings (SI units).  Defaults: 50 m observation radius
    (Fig. 1), goal radius 2 m, dt 0.1 s (10 Hz), 91-step episodes."""
    k_road: int = 200
    n_partners: int = 63
    episode_len: int = 91
    obs_radius: float = 50.0
    goal_radius: float = 2.0
    dt: float = 0.1
    v_max: float = 30.0
    collision_penalty: float = 0.0
    offroad_penalty: float = 0.0
    smooth_c: float = 1.0
    term_collision: bool = False
    term_offroad: bool = False
    auto_reset: bool = False
    dynamics: int = 0          # 0: kinematic bicycle (App. B); 1: simplified invertible model (Sec. 3.2)
    nontrivial_init: bool = False   # Sec. 3.2 "Initialization modes": agents near their goal are not controlled
    nontrivial_dist: float = 2.0

    @property
    def feat(self) -> int:
        return 8 + 8 * self.n_partners + 4 * self.k_road

    def c(self) -> _Cfg:
        fl = (TERM_COLLISION if self.term_collision else 0) | (TERM_OFFROAD if self.term_offroad else 0) \
            | (AUTO_RESET if self.auto_reset else 0) | (NONTRIVIAL_INIT if self.nontrivial_init else 0)
        return _Cfg(self.k_road, self.n_partners, self.episode_len, self.obs_radius, self.goal_radius,
                    self.dt, self.v_max, self.collision_penalty, self.offroad_penalty, self.smooth_c, fl,
                    self.dynamics, self.nontrivial_dist)


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class Oracle:
    """Brute-force simulator over a ``scenes.Scene`` (host memory)."""

    def __init__(self, scene, cfg: OracleConfig, precision: int = 64):
        self.lib = load_oracle()
        self.cfg = cfg
        self.A = scene.num_agents
        self.W = scene.num_worlds
        self.agent_off = scene.agent_off.copy()
        self._keep = [_c(scene.agent_off, np.int32), _c(scene.road_off, np.int32)] + \
            [_c(getattr(scene, k), np.float32) for k in
             ("x", "y", "theta", "v", "length", "width", "goal_x", "goal_y")] + \
            [_c(scene.agent_type, np.uint8), _c(scene.road_x, np.float32), _c(scene.road_y, np.float32),
             _c(scene.road_type, np.uint8), _c(scene.road_poly, np.int32)]
        self._cfg = cfg.c()
        self.h = self.lib.or_create(C.byref(self._cfg), precision, self.W, *[_p(a) for a in self._keep])

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.or_destroy(self.h)
            self.h = None

    def reset(self, mask=None):
        m = None if mask is None else _c(mask, np.uint8)
        self.lib.or_reset(self.h, _p(m))

    def _outs(self):
        A, W = self.A, self.W
        return dict(reward=np.zeros(A, np.float32), done=np.zeros(A, np.uint8), world_done=np.zeros(W, np.uint8),
                    coll_margin=np.zeros(A), off_margin=np.zeros(A), goal_margin=np.zeros(A),
                    smooth_r=np.zeros(A))

    def step(self, actions):
        a = _c(actions, np.float32).reshape(self.A, 2)
        o = self._outs()
        self.lib.or_step(self.h, _p(a), *[_p(o[k]) for k in o])
        return o

    def step_post(self, post_state):
        s = _c(post_state, np.float32).reshape(self.A, 4)
        o = self._outs()
        self.lib.or_step_post(self.h, _p(s), *[_p(o[k]) for k in o])
        return o

    def observe(self):
        cfg = self.cfg
        obs = np.zeros((self.A, cfg.feat), np.float32)
        ridx = np.zeros((self.A, cfg.k_road), np.int32)
        pidx = np.zeros((self.A, cfg.n_partners), np.int32)
        self.lib.or_observe(self.h, _p(obs), _p(ridx), _p(pidx))
        return obs, ridx, pidx

    def observe64(self):
        """Observation rows in float64 (same layout) with the index lists."""
        cfg = self.cfg
        obs = np.zeros((self.A, cfg.feat), np.float64)
        ridx = np.zeros((self.A, cfg.k_road), np.int32)
        pidx = np.zeros((self.A, cfg.n_partners), np.int32)
        self.lib.or_observe64(self.h, _p(obs), _p(ridx), _p(pidx))
        return obs, ridx, pidx

    def lidar(self, n_rays: int, fov: float = 2 * np.pi, head=None, agents=None, band: float = 2e-4):
        """LiDAR / view-cone scan (readings in oracle.cpp, above lidar()):
        for the agents `agents` (global indices; None = all) returns
        depth float64 [n, n_rays], cls uint8 (0 none, 1 agent, 2 road edge),
        fragile uint8 (1 = a decision within `band` m of flipping) and
        sens = |d depth / d ray angle|."""
        sel = None if agents is None else _c(agents, np.int32)
        n = self.A if sel is None else len(sel)
        hd = None if head is None else _c(head, np.float32).reshape(self.A)
        out = dict(depth=np.zeros((n, n_rays)), cls=np.zeros((n, n_rays), np.uint8),
                   fragile=np.zeros((n, n_rays), np.uint8), sens=np.zeros((n, n_rays)))
        self.lib.or_lidar(self.h, int(n_rays), float(fov), _p(hd), _p(sel), n, float(band),
                          _p(out["depth"]), _p(out["cls"]), _p(out["fragile"]), _p(out["sens"]))
        return out

    def road_point(self, i: int, j: int):
        f = np.zeros(4, np.float32)
        d = np.zeros(1)
        self.lib.or_road_point(self.h, int(i), int(j), _p(f), _p(d))
        return f, float(d[0])

    def partner(self, i: int, j: int):
        f = np.zeros(8, np.float32)
        d = np.zeros(1)
        self.lib.or_partner(self.h, int(i), int(j), _p(f), _p(d))
        return f, float(d[0])

    def get_state(self):
        s = np.zeros((self.A, 4))
        f = np.zeros(self.A, np.uint8)
        t = np.zeros(self.W, np.int32)
        wd = np.zeros(self.W, np.uint8)
        self.lib.or_get_state(self.h, _p(s), _p(f), _p(t), _p(wd))
        return s, f, t, wd

    def set_state(self, state=None, flags=None, t=None):
        s = None if state is None else _c(state, np.float32).reshape(self.A, 4)
        f = None if flags is None else _c(flags, np.uint8)
        tt = None if t is None else _c(t, np.int32)
        self.lib.or_set_state(self.h, _p(s), _p(f), _p(tt))


def bicycle(cfg: OracleConfig, state, actions, length):
    """One dynamics step (cfg.dynamics: App. B, or the simplified invertible
    model of Sec. 3.2) of independent agents in float64: state [n,4] (x, y,
    theta, v), actions [n,2] (accel, steer), length [n]; returns new state."""
    lib = load_oracle()
    s = np.array(state, dtype=np.float64, copy=True).reshape(-1, 4)
    a = _c(actions, np.float64).reshape(-1, 2)
    L = _c(np.broadcast_to(length, (s.shape[0],)), np.float64)
    c = cfg.c()
    lib.or_bicycle(C.byref(c), s.shape[0], _p(s), _p(a), _p(L))
    return s


def invert(cfg: OracleConfig, states, length):
    """Expert actions [T, n, 2] of trajectories states [T+1, n, 4] under
    cfg.dynamics (readings in oracle.cpp, above invert_step), float64."""
    lib = load_oracle()
    s = _c(states, np.float64)
    T, n = s.shape[0] - 1, s.shape[1]
    L = _c(np.broadcast_to(length, (n,)), np.float64)
    out = np.zeros((T, n, 2))
    c = cfg.c()
    lib.or_invert(C.byref(c), T, n, _p(s), _p(L), _p(out))
    return out


def decimate(poly_off, x, y, tol):
    """Visvalingam-Whyatt keep mask (uint8 [N]) of the polylines
    poly_off [P+1] over float32 points x, y with area tolerance tol (m^2)."""
    lib = load_oracle()
    off = _c(poly_off, np.int32)
    xx, yy = _c(x, np.float32), _c(y, np.float32)
    keep = np.zeros(xx.shape[0], np.uint8)
    lib.or_decimate(len(off) - 1, _p(off), _p(xx), _p(yy), float(tol), _p(keep))
    return keep


def box_box(p, q) -> float:
    """Penetration depth of boxes (cx, cy, theta, length, width); > 0 iff overlap."""
    lib = load_oracle()
    return lib.or_box_box(_p(_c(p, np.float64)), _p(_c(q, np.float64)))


def box_seg(p, s) -> float:
    """Penetration depth of a box and a segment (x0, y0, x1, y1); > 0 iff they cross."""
    lib = load_oracle()
    return lib.or_box_seg(_p(_c(p, np.float64)), _p(_c(s, np.float64)))


def num_threads() -> int:
    return load_oracle().or_num_threads()
