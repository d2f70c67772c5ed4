"""Helpers shared by the tests: hand-built tiny scenes and workload settings."""
import numpy as np

from paper_2408_01584_b300 import scenes
from oracle import OracleConfig


def tiny_scene(worlds):
    """worlds: list of (agents, road) where agents is a list of
    (x, y, theta, v, length, width, goal_x, goal_y, type) and road a list of
    (x, y, type, poly)."""
    a_off, r_off = [0], [0]
    cols = {k: [] for k in ("x", "y", "theta", "v", "length", "width", "goal_x", "goal_y", "agent_type")}
    rcols = {k: [] for k in ("road_x", "road_y", "road_type", "road_poly")}
    for agents, road in worlds:
        for a in agents:
            for k, val in zip(cols, a):
                cols[k].append(val)
        for r in road:
            for k, val in zip(rcols, r):
                rcols[k].append(val)
        a_off.append(a_off[-1] + len(agents))
        r_off.append(r_off[-1] + len(road))
    f = lambda k, d: np.array(cols[k] if k in cols else rcols[k], dtype=d)
    return scenes.Scene(
        agent_off=np.array(a_off, np.int32), road_off=np.array(r_off, np.int32),
        x=f("x", np.float32), y=f("y", np.float32), theta=f("theta", np.float32), v=f("v", np.float32),
        length=f("length", np.float32), width=f("width", np.float32), goal_x=f("goal_x", np.float32),
        goal_y=f("goal_y", np.float32), agent_type=f("agent_type", np.uint8),
        road_x=f("road_x", np.float32), road_y=f("road_y", np.float32),
        road_type=f("road_type", np.uint8), road_poly=f("road_poly", np.int32))


def workload_config(name, **over) -> OracleConfig:
    wl = scenes.WORKLOADS[name]
    kw = dict(k_road=wl["k_road"], n_partners=wl["n_partners"], episode_len=wl["steps"],
              term_collision=wl["term_collision"], term_offroad=wl["term_offroad"],
              auto_reset=wl["auto_reset"])
    kw.update(over)
    return OracleConfig(**kw)


def small_scene(seed=0, worlds=6, agents=(3, 9, 16, 1, 24, 40), road=(300, 900, 1500, 200, 2500, 3100)):
    """Ragged scene with a few worlds of different sizes (parity-sized)."""
    return scenes.make_scene(np.array(agents[:worlds]), np.array(road[:worlds]), seed)
