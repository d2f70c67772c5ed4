"""Pins of the oracle's reward, termination, collision flags and reset.

Rewards: 1 on reaching the goal within delta, else 0 (Sec. 3.2 "Rewards").
Termination: on the goal, optionally on collision; the agent leaves the
scene afterwards; cars and cyclists crossing a road edge are in collision,
pedestrians may cross (Sec. 3.2 "Termination conditions").  The collision
decisions are re-derived here by polygon clipping, independently of the
oracle's separating-axis code.
"""
import math

import numpy as np

from oracle import Oracle, OracleConfig
from paper_2408_01584_b300 import scenes
from tests._util import tiny_scene, small_scene
from tests.test_oracle_geometry import _area, _clip, _corners, _seg_inside_length


def test_reward_once_done_monotone_goal_iff_distance():
    sc = small_scene(seed=7)
    cfg = OracleConfig(k_road=8, n_partners=2, episode_len=91, goal_radius=2.0,
                       term_collision=True, term_offroad=True)
    o = Oracle(sc, cfg)
    acts = scenes.make_actions(91, sc.num_agents, 3)
    # drive half the agents straight at their goal so that goals are reached
    total = np.zeros(sc.num_agents)
    prev_done = np.zeros(sc.num_agents, bool)
    prev_goal = np.zeros(sc.num_agents, bool)
    n_goal = 0
    for t in range(91):
        st, fl, _, _ = o.get_state()
        a = acts[t].copy()
        hd = np.arctan2(sc.goal_y - st[:, 1], sc.goal_x - st[:, 0]) - st[:, 2]
        hd = (hd + np.pi) % (2 * np.pi) - np.pi
        steer = np.clip(hd, -0.6, 0.6)
        a[::2, 1] = steer[::2]
        a[::2, 0] = np.where(st[::2, 3] > 6.0, -1.0, 1.0)
        before, _, _, _ = o.get_state()
        out = o.step(a)
        st, fl, _, _ = o.get_state()
        done = out["done"].astype(bool)
        goal = (fl & 2) > 0
        total += out["reward"]
        assert (done >= prev_done).all()                               # done is monotone
        frozen = prev_done
        np.testing.assert_array_equal(st[frozen], before[frozen])      # done agents do not move
        assert (out["reward"][frozen] == 0).all()
        dist = np.hypot(st[:, 0] - sc.goal_x, st[:, 1] - sc.goal_y)
        newly = goal & ~prev_goal
        np.testing.assert_array_equal(newly, (~prev_done) & (dist <= 2.0))   # goal iff d <= delta
        np.testing.assert_array_equal(out["reward"], newly.astype(np.float32))
        n_goal += newly.sum()
        prev_done, prev_goal = done, goal
    assert (total <= 1).all()
    assert n_goal >= 3


def test_collision_flags_match_polygon_clipping():
    # dense worlds so that boxes do overlap
    sc = scenes.make_scene(np.array([30, 20]), np.array([300, 240]), 9, n_poly=2)
    cfg = OracleConfig(k_road=8, n_partners=2, episode_len=91)
    o = Oracle(sc, cfg)
    acts = scenes.make_actions(12, sc.num_agents, 2)
    seen_coll = seen_off = 0
    for t in range(12):
        out = o.step(acts[t])
        st, fl, _, _ = o.get_state()
        for w in range(sc.num_worlds):
            a0, a1 = sc.agent_off[w], sc.agent_off[w + 1]
            r0, r1 = sc.road_off[w], sc.road_off[w + 1]
            segs = [(j, j + 1) for j in range(r0, r1 - 1)
                    if sc.road_type[j] == 1 and sc.road_type[j + 1] == 1 and sc.road_poly[j] == sc.road_poly[j + 1]]
            for i in range(a0, a1):
                bi = [st[i, 0], st[i, 1], st[i, 2], sc.length[i], sc.width[i]]
                coll = any(_area(_clip(_corners(bi), _corners([st[j, 0], st[j, 1], st[j, 2], sc.length[j], sc.width[j]]))) > 1e-12
                           for j in range(a0, a1) if j != i)
                if abs(out["coll_margin"][i]) > 1e-6:
                    assert bool(fl[i] & 4) == coll, (t, i)
                off = any(_seg_inside_length(bi, [sc.road_x[a], sc.road_y[a], sc.road_x[b], sc.road_y[b]]) > 1e-9
                          for a, b in segs)
                if abs(out["off_margin"][i]) > 1e-6:
                    assert bool(fl[i] & 8) == off, (t, i)
                seen_coll += coll
                seen_off += off
    assert seen_coll > 5 and seen_off > 5


def test_pedestrians_may_cross_road_edges():
    edge = [(-10.0, 0.0, 1, 0), (10.0, 0.0, 1, 0)]
    car = (0, 0, 0.3, 0, 4.5, 2, 50, 50, scenes.VEHICLE)
    cyc = (0, 0, 0.3, 0, 1.8, 0.8, 50, 50, scenes.CYCLIST)
    ped = (0, 0, 0.3, 0, 0.6, 0.6, 50, 50, scenes.PEDESTRIAN)
    sc = tiny_scene([([car], edge), ([cyc], edge), ([ped], edge)])
    o = Oracle(sc, OracleConfig(k_road=2, n_partners=1, term_offroad=True))
    out = o.step(np.zeros((3, 2), np.float32))
    assert list(out["done"]) == [1, 1, 0]
    _, fl, _, _ = o.get_state()
    assert list(fl & 8) == [8, 8, 0]


def test_masked_reset_restores_snapshot_bitwise():
    sc = small_scene(seed=1, worlds=4)
    cfg = OracleConfig(k_road=8, n_partners=2, term_collision=True)
    o = Oracle(sc, cfg)
    acts = scenes.make_actions(6, sc.num_agents, 0)
    for t in range(6):
        o.step(acts[t])
    before, fb, tb, _ = o.get_state()
    o.reset(np.array([1, 0, 1, 0], np.uint8))
    after, fa, ta, _ = o.get_state()
    for w in range(4):
        sl = slice(sc.agent_off[w], sc.agent_off[w + 1])
        if w in (0, 2):
            np.testing.assert_array_equal(after[sl], sc.state()[sl].astype(np.float64))
            assert (fa[sl] == 0).all() and ta[w] == 0
        else:
            np.testing.assert_array_equal(after[sl], before[sl])
            np.testing.assert_array_equal(fa[sl], fb[sl])
            assert ta[w] == 6


def test_auto_reset_after_episode_end():
    sc = small_scene(seed=3, worlds=3)
    cfg = OracleConfig(k_road=8, n_partners=2, episode_len=4, auto_reset=True)
    o = Oracle(sc, cfg)
    fresh = Oracle(sc, cfg)
    acts = scenes.make_actions(5, sc.num_agents, 0)
    for t in range(4):
        out = o.step(acts[t])
    assert (out["world_done"] == 1).all()
    o.step(acts[4])          # worlds reset, then step once from the snapshot
    fresh.step(acts[4])
    s1, f1, t1, _ = o.get_state()
    s2, f2, t2, _ = fresh.get_state()
    np.testing.assert_array_equal(s1, s2)
    np.testing.assert_array_equal(f1, f2)
    assert (t1 == 1).all()


def test_float_and_double_oracles_agree_to_rounding():
    sc = small_scene(seed=8, worlds=3)
    cfg = OracleConfig(k_road=16, n_partners=4)
    o64, o32 = Oracle(sc, cfg, 64), Oracle(sc, cfg, 32)
    acts = scenes.make_actions(10, sc.num_agents, 5)
    for t in range(10):
        o64.step(acts[t])
        o32.step(acts[t])
    s64, _, _, _ = o64.get_state()
    s32, _, _, _ = o32.get_state()
    assert np.abs(s64 - s32).max() < 1e-3
    assert np.abs(s64 - s32).max() > 0      # the float build does round
