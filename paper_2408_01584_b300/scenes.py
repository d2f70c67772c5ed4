"""Seeded synthetic driving scenes and action streams (inputs only).

This module draws the INPUTS of the simulator step: road polylines, agent
start states, goals and per-step actions.  It holds none of the simulator's
arithmetic (no dynamics, collision, observation or reward code), so both the
CUDA library and the CPU oracle can consume what it produces.

The Waymo Open Motion Dataset used by the paper (Sec. 3.2, "Dataset") is not
available here; these scenes stand in for it with the structure the paper
describes: maps made of polylines sampled along lanes without lane
connectivity (Sec. 3.1, Sec. 3.2 "Dataset"), road-edge polylines that agents
must not cross (Sec. 3.2 "Termination conditions"), ragged agent counts per
world (Sec. 3.1, Fig. 3 centre) and goals along the agent's lane
(Sec. 3.2 "Rewards").

Recipe (all draws from ``numpy.random.Generator(PCG64(seed))``):
  * map side S = 300 * sqrt(N_w / 4000) m, centred at the origin;
  * n_poly polylines per world (default 2 * max(1, round(N_w / 200))), half
    lane centrelines (type LANE = 0), half road edges (type ROAD_EDGE = 1);
  * a lane starts uniformly in [-S/2, S/2]^2 with a uniform heading and is a
    chain of pieces, each straight (length U[10, 50] m) or a circular arc
    (radius U[15, 80] m, turn U[-pi/2, pi/2]) with probability 1/2, sampled
    every 1 m of arc length;
  * each road edge is its lane shifted 3 m along the lane's left normal;
  * agents are 4.5 x 2.0 m boxes placed at a lane point with the lane's
    tangent heading, re-drawn (up to 100 tries) when closer than 8 m to an
    agent already placed; initial speed U[0, 15] m/s; goal = the lane point
    U{20..60} m further along the same lane;
  * actions are i.i.d. per (step, agent): acceleration U[-4, 4] m/s^2,
    steering U[-0.7, 0.7] rad.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

LANE = 0
ROAD_EDGE = 1

VEHICLE = 0
CYCLIST = 1
PEDESTRIAN = 2

_PIECES = 64          # pieces drawn per lane (far more than a 100 m lane needs)
_EDGE_OFFSET = 3.0    # m, lateral offset of a road edge from its lane
_MIN_SEP = 8.0        # m, rejection distance between placed agents
_TRIES = 100


@dataclasses.dataclass
class Scene:
    """Ragged batch of worlds in CSR layout (world w owns agents
    ``agent_off[w]:agent_off[w+1]`` and road points ``road_off[w]:road_off[w+1]``).
    All coordinates are metres in the world's own frame, headings radians."""

    agent_off: np.ndarray   # int32 [W+1]
    road_off: np.ndarray    # int32 [W+1]
    x: np.ndarray           # float32 [A]
    y: np.ndarray
    theta: np.ndarray
    v: np.ndarray
    length: np.ndarray
    width: np.ndarray
    goal_x: np.ndarray
    goal_y: np.ndarray
    agent_type: np.ndarray  # uint8 [A]
    road_x: np.ndarray      # float32 [N]
    road_y: np.ndarray
    road_type: np.ndarray   # uint8 [N]
    road_poly: np.ndarray   # int32 [N], polyline id local to the world

    @property
    def num_worlds(self) -> int:
        return int(self.agent_off.shape[0] - 1)

    @property
    def num_agents(self) -> int:
        return int(self.agent_off[-1])

    @property
    def num_road(self) -> int:
        return int(self.road_off[-1])

    def agents_per_world(self) -> np.ndarray:
        return np.diff(self.agent_off)

    def road_per_world(self) -> np.ndarray:
        return np.diff(self.road_off)

    def state(self) -> np.ndarray:
        """Initial state as float32 [A, 4] = (x, y, theta, v)."""
        return np.stack([self.x, self.y, self.theta, self.v], axis=1).astype(np.float32)

    def subset(self, w0: int, w1: int) -> "Scene":
        """Worlds [w0, w1) as a scene of their own (same arrays, re-based)."""
        a0, a1 = int(self.agent_off[w0]), int(self.agent_off[w1])
        r0, r1 = int(self.road_off[w0]), int(self.road_off[w1])
        sl = slice(a0, a1)
        rl = slice(r0, r1)
        return Scene(
            agent_off=(self.agent_off[w0:w1 + 1] - a0).astype(np.int32),
            road_off=(self.road_off[w0:w1 + 1] - r0).astype(np.int32),
            x=self.x[sl].copy(), y=self.y[sl].copy(), theta=self.theta[sl].copy(),
            v=self.v[sl].copy(), length=self.length[sl].copy(), width=self.width[sl].copy(),
            goal_x=self.goal_x[sl].copy(), goal_y=self.goal_y[sl].copy(),
            agent_type=self.agent_type[sl].copy(),
            road_x=self.road_x[rl].copy(), road_y=self.road_y[rl].copy(),
            road_type=self.road_type[rl].copy(), road_poly=self.road_poly[rl].copy())

    def transformed(self, angle: float, tx: float, ty: float) -> "Scene":
        """The same scene moved by a rigid motion (rotation by ``angle`` about
        the origin, then translation).  Used by invariance tests."""
        c, s = math.cos(angle), math.sin(angle)

        def mv(px, py):
            px = px.astype(np.float64)
            py = py.astype(np.float64)
            return ((c * px - s * py + tx).astype(np.float32),
                    (s * px + c * py + ty).astype(np.float32))

        out = dataclasses.replace(self)
        out.x, out.y = mv(self.x, self.y)
        out.goal_x, out.goal_y = mv(self.goal_x, self.goal_y)
        out.road_x, out.road_y = mv(self.road_x, self.road_y)
        out.theta = (self.theta.astype(np.float64) + angle).astype(np.float32)
        return out


def _lanes(rng, n_pts, starts, headings, spacing=1.0):
    """Sample lane centrelines every ``spacing`` m of arc length.  ``n_pts[l]``
    points for lane l, starting at ``starts[l]`` with heading ``headings[l]``.
    Returns (px, py, th) padded arrays [L, nmax] (heading at each point)."""
    L = n_pts.shape[0]
    nmax = int(n_pts.max()) if L else 0
    straight = rng.random((L, _PIECES)) < 0.5
    slen = rng.uniform(10.0, 50.0, (L, _PIECES))
    radius = rng.uniform(15.0, 80.0, (L, _PIECES))
    turn = rng.uniform(-math.pi / 2, math.pi / 2, (L, _PIECES))
    alen = radius * np.abs(turn)
    plen = np.where(straight, slen, alen)
    plen = np.maximum(plen, 1e-3)
    kappa = np.where(straight, 0.0, turn / plen)
    cum = np.cumsum(plen, axis=1)                      # end arc position of each piece
    # piece index of each step (midpoint s = (k + 0.5) spacing), vectorised across lanes
    big = float(np.ceil(cum[:, -1].max() + 2.0)) if L else 1.0
    flat = (cum + big * np.arange(L)[:, None]).ravel()
    s = (np.arange(max(nmax - 1, 0), dtype=np.float64) + 0.5) * spacing
    q = (s[None, :] + big * np.arange(L)[:, None]).ravel()
    piece = np.searchsorted(flat, q, side="right").reshape(L, -1) - _PIECES * np.arange(L)[:, None]
    piece = np.clip(piece, 0, _PIECES - 1)
    k_step = np.take_along_axis(kappa, piece, axis=1) * spacing   # [L, nmax-1] heading change per step
    th = np.empty((L, nmax))
    th[:, 0] = headings
    if nmax > 1:
        th[:, 1:] = headings[:, None] + np.cumsum(k_step, axis=1)
    mid = th[:, :-1] + 0.5 * k_step
    px = np.empty((L, nmax))
    py = np.empty((L, nmax))
    px[:, 0] = starts[:, 0]
    py[:, 0] = starts[:, 1]
    if nmax > 1:
        px[:, 1:] = starts[:, 0:1] + np.cumsum(spacing * np.cos(mid), axis=1)
        py[:, 1:] = starts[:, 1:2] + np.cumsum(spacing * np.sin(mid), axis=1)
    return px, py, th


def make_scene(agents_per_world, road_per_world, seed: int, n_poly=None,
               type_mix=(1.0, 0.0, 0.0), agent_length=4.5, agent_width=2.0, parked_frac=0.0,
               spacing=1.0) -> Scene:
    """Build a seeded scene.

    agents_per_world / road_per_world: int arrays [W] (A_w >= 0, N_w >= 2).
    n_poly: polylines per world (int, array [W] or None for the default
    2 * max(1, round(N_w / 200))); must be even (lane + edge pairs).
    type_mix: probabilities of (vehicle, cyclist, pedestrian).
    spacing: metres between consecutive polyline points (1 m by default;
    0.1 m is the source sampling the paper decimates, Sec. 3.1).  The map
    side and the agent / goal placement scale with the road length.
    parked_frac: each agent is, with this probability, parked: speed 0 and
    its goal within 1.5 m of where it stands (the scenes of Sec. 3.2
    "Initialization modes", where 25-75% of agents start at or near their
    goal).  Drawn after everything else, so other draws do not change.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    A_w = np.asarray(agents_per_world, dtype=np.int64)
    N_w = np.asarray(road_per_world, dtype=np.int64)
    W = A_w.shape[0]
    assert N_w.shape[0] == W and (N_w >= 2).all() and (A_w >= 0).all()
    if n_poly is None:
        P_w = 2 * np.maximum(1, np.round(N_w / 200.0).astype(np.int64))
    else:
        P_w = np.broadcast_to(np.asarray(n_poly, dtype=np.int64), (W,)).copy()
    assert (P_w % 2 == 0).all() and (P_w >= 2).all()
    nl_w = P_w // 2
    side = 300.0 * np.sqrt(N_w * spacing / 4000.0)

    # points per lane: the lanes of world w share ceil(N_w/2) points, edges floor(N_w/2)
    lane_world = np.repeat(np.arange(W), nl_w)
    lane_rank = np.arange(lane_world.shape[0]) - np.repeat(np.cumsum(nl_w) - nl_w, nl_w)
    lane_total = (N_w + 1) // 2
    base = lane_total // nl_w
    rem = lane_total - base * nl_w
    lane_pts = base[lane_world] + (lane_rank < rem[lane_world])
    edge_pts = lane_pts.copy()
    odd_last = ((N_w % 2) == 1)[lane_world] & (lane_rank == nl_w[lane_world] - 1)
    edge_pts[odd_last] -= 1
    assert (edge_pts >= 1).all(), "too many polylines for the road-point budget"

    L = lane_world.shape[0]
    half = 0.5 * side[lane_world]
    starts = np.stack([rng.uniform(-1.0, 1.0, L) * half, rng.uniform(-1.0, 1.0, L) * half], axis=1)
    heads = rng.uniform(0.0, 2 * math.pi, L)
    px, py, th = _lanes(rng, lane_pts, starts, heads, spacing)
    ex = px - _EDGE_OFFSET * np.sin(th)
    ey = py + _EDGE_OFFSET * np.cos(th)

    # road arrays: per world, lane0, edge0, lane1, edge1, ...
    counts = np.stack([lane_pts, edge_pts], axis=1).ravel()
    road_x = np.empty(int(counts.sum()), np.float32)
    road_y = np.empty_like(road_x)
    road_type = np.empty(road_x.shape, np.uint8)
    road_poly = np.empty(road_x.shape, np.int32)
    col = np.arange(px.shape[1])[None, :]
    lane_mask = col < lane_pts[:, None]
    edge_mask = col < edge_pts[:, None]
    # interleave lanes and edges by filling a [L, 2, nmax] array in order
    nmax = px.shape[1]
    allx = np.stack([px, ex], axis=1)
    ally = np.stack([py, ey], axis=1)
    allm = np.stack([lane_mask, edge_mask], axis=1)
    typ = np.broadcast_to(np.array([LANE, ROAD_EDGE], np.uint8)[None, :, None], allm.shape)
    pid = (2 * lane_rank)[:, None, None] + np.array([0, 1])[None, :, None]
    pid = np.broadcast_to(pid, allm.shape)
    road_x[:] = allx[allm]
    road_y[:] = ally[allm]
    road_type[:] = typ[allm]
    road_poly[:] = pid[allm]
    road_off = np.zeros(W + 1, np.int32)
    road_off[1:] = np.cumsum(N_w)
    assert road_off[-1] == road_x.shape[0]

    # agents
    A = int(A_w.sum())
    agent_off = np.zeros(W + 1, np.int32)
    agent_off[1:] = np.cumsum(A_w)
    lane_off = np.zeros(W + 1, np.int64)
    lane_off[1:] = np.cumsum(nl_w)
    amax = int(A_w.max()) if W else 0
    pos = np.full((W, max(amax, 1), 2), np.nan)
    lane_of = np.zeros((W, max(amax, 1)), np.int64)
    k_of = np.zeros((W, max(amax, 1)), np.int64)
    for slot in range(amax):
        need = np.nonzero(A_w > slot)[0]
        chosen_lane = np.zeros(W, np.int64)
        chosen_k = np.zeros(W, np.int64)
        pending = need.copy()
        for _ in range(_TRIES):
            if pending.size == 0:
                break
            ln = lane_off[pending] + rng.integers(0, nl_w[pending])
            hi = np.maximum(lane_pts[ln] - int(round(21 / spacing)), 1)
            kk = rng.integers(0, hi)
            cx, cy = px[ln, kk], py[ln, kk]
            chosen_lane[pending] = ln
            chosen_k[pending] = kk
            if slot == 0:
                pending = pending[:0]
                break
            d2 = (pos[pending, :slot, 0] - cx[:, None]) ** 2 + (pos[pending, :slot, 1] - cy[:, None]) ** 2
            ok = (d2 >= _MIN_SEP ** 2).all(axis=1)
            pending = pending[~ok]
        # after the last try the latest draw is accepted as is
        lane_of[need, slot] = chosen_lane[need]
        k_of[need, slot] = chosen_k[need]
        pos[need, slot, 0] = px[chosen_lane[need], chosen_k[need]]
        pos[need, slot, 1] = py[chosen_lane[need], chosen_k[need]]

    wa = np.repeat(np.arange(W), A_w)
    sa = np.arange(A) - agent_off[wa]
    ln = lane_of[wa, sa]
    kk = k_of[wa, sa]
    n_l = lane_pts[ln]
    k1 = np.minimum(kk + 1, n_l - 1)
    k0 = np.where(k1 == kk, kk - 1, kk)
    heading = np.arctan2(py[ln, k1] - py[ln, k0], px[ln, k1] - px[ln, k0])
    gk = np.minimum(kk + np.round(rng.integers(20, 61, A) / spacing).astype(np.int64), n_l - 1)
    v0 = rng.uniform(0.0, 15.0, A)
    mix = np.asarray(type_mix, dtype=np.float64)
    mix = mix / mix.sum()
    atype = rng.choice(3, size=A, p=mix).astype(np.uint8) if mix[0] < 1.0 else np.zeros(A, np.uint8)

    x0, y0 = px[ln, kk], py[ln, kk]
    gx, gy = px[ln, gk], py[ln, gk]
    if parked_frac > 0.0:
        parked = rng.random(A) < parked_frac
        r = rng.uniform(0.0, 1.5, A)
        ang = rng.uniform(0.0, 2 * math.pi, A)
        gx = np.where(parked, x0 + r * np.cos(ang), gx)
        gy = np.where(parked, y0 + r * np.sin(ang), gy)
        v0 = np.where(parked, 0.0, v0)

    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Scene(
        agent_off=agent_off, road_off=road_off,
        x=f32(x0), y=f32(y0), theta=f32(heading), v=f32(v0),
        length=np.full(A, agent_length, np.float32), width=np.full(A, agent_width, np.float32),
        goal_x=f32(gx), goal_y=f32(gy), agent_type=atype,
        road_x=road_x, road_y=road_y, road_type=road_type, road_poly=road_poly)


def make_actions(steps: int, num_agents: int, seed: int) -> np.ndarray:
    """i.i.d. actions float32 [steps, A, 2] = (accel m/s^2, steer rad)."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x5EED))
    a = np.empty((steps, num_agents, 2), np.float32)
    a[..., 0] = rng.uniform(-4.0, 4.0, (steps, num_agents))
    a[..., 1] = rng.uniform(-0.7, 0.7, (steps, num_agents))
    return a


# ---------------------------------------------------------------------------
# Workloads.  Each names the batch shape, the observation sizes and the
# episode settings; ``workload_scene`` draws the matching seeded scene.
# ---------------------------------------------------------------------------
WORKLOADS = {
    # 4 worlds x 8 agents, 1,000 road points on 6 polylines, 20 steps, K=64, P=7
    "plain_4x8": dict(worlds=4, agents=("fixed", 8), road=("fixed", 1000), n_poly=6,
                      k_road=64, n_partners=7, steps=20,
                      term_collision=False, term_offroad=False, auto_reset=False),
    # 1,024 worlds x 64 agents, 4,000 road points on 40 polylines, 91 steps, K=200, P=63
    "plain_1024x64": dict(worlds=1024, agents=("fixed", 64), road=("fixed", 4000), n_poly=40,
                          k_road=200, n_partners=63, steps=91,
                          term_collision=True, term_offroad=True, auto_reset=True),
    # 4,096 worlds, agents log-uniform [1,128], road points U[500, 20,000]
    "uneven_4096": dict(worlds=4096, agents=("loguniform", 1, 128), road=("uniform", 500, 20000),
                        n_poly=None, k_road=200, n_partners=63, steps=91,
                        term_collision=True, term_offroad=True, auto_reset=True),
    # 512 worlds x 32 agents, 2,000 road points, differentiable, 91 steps
    "diff_512x32": dict(worlds=512, agents=("fixed", 32), road=("fixed", 2000), n_poly=None,
                        k_road=200, n_partners=31, steps=91,
                        term_collision=True, term_offroad=True, auto_reset=False),
    # 8,192 worlds, agents U[32,128], road points U[5,000, 10,000], fwd+bwd
    "fwdbwd_8192": dict(worlds=8192, agents=("uniform", 32, 128), road=("uniform", 5000, 10000),
                        n_poly=None, k_road=200, n_partners=63, steps=91,
                        term_collision=True, term_offroad=True, auto_reset=False),
    # 1,024 x 64 as plain_1024x64 with mixed agent types (70% vehicles, 15%
    # cyclists, 15% pedestrians), half the agents parked at their goal, and
    # the "all nontrivial" initialisation (only agents > 2 m from their goal
    # are controlled)
    "nontrivial_1024x64": dict(worlds=1024, agents=("fixed", 64), road=("fixed", 4000), n_poly=40,
                               k_road=200, n_partners=63, steps=91,
                               term_collision=True, term_offroad=True, auto_reset=True,
                               type_mix=(0.7, 0.15, 0.15), parked_frac=0.5, nontrivial_init=True),
    # 256 worlds x 64 agents on roads sampled every 0.1 m (24 polylines of
    # 1,000 points per world, the source sampling the paper decimates 10-15x)
    "dense_roads_256x64": dict(worlds=256, agents=("fixed", 64), road=("fixed", 24000), n_poly=24, spacing=0.1,
                               k_road=200, n_partners=63, steps=91,
                               term_collision=True, term_offroad=True, auto_reset=True),
}


def _counts(spec, W, rng):
    kind = spec[0]
    if kind == "fixed":
        return np.full(W, spec[1], np.int64)
    if kind == "uniform":
        return rng.integers(spec[1], spec[2] + 1, W)
    if kind == "loguniform":
        lo, hi = spec[1], spec[2]
        c = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi + 1), W))).astype(np.int64)
        return np.clip(c, lo, hi)
    raise ValueError(kind)


def workload_scene(name: str, seed: int = 0, worlds: int | None = None) -> Scene:
    """Seeded scene of a named workload (optionally its first ``worlds`` worlds)."""
    wl = WORKLOADS[name]
    W = wl["worlds"]
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    A_w = _counts(wl["agents"], W, rng)
    N_w = _counts(wl["road"], W, rng)
    if worlds is not None:
        A_w, N_w = A_w[:worlds], N_w[:worlds]
    return make_scene(A_w, N_w, seed, n_poly=wl["n_poly"], type_mix=wl.get("type_mix", (1.0, 0.0, 0.0)),
                      parked_frac=wl.get("parked_frac", 0.0), spacing=wl.get("spacing", 1.0))
