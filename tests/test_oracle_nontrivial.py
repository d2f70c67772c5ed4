"""Pins of the oracle's "all nontrivial" initialisation (Sec. 3.2 "Simulator
sharp-edges", "Initialization modes") and per-type rules on mixed scenes.

* exactly the agents within 2 m of their goal at the start are not
  controlled (brute-force distance check), and a reset restores that;
* an uncontrolled agent never moves, never scores and reports done, yet it
  stays in the scene: a controlled agent that drives into it collides, it
  is a partner in observations and a box for the LiDAR;
* a world's episode ends when its controlled agents are done; a world of
  uncontrolled agents only times out;
* on a mixed scene, pedestrians never get the off-road flag while vehicles
  and cyclists do.
"""
import numpy as np

from oracle import Oracle, OracleConfig
from oracle.oracle import DONE, OFFROAD, COLLIDED, STATIC
from paper_2408_01584_b300 import scenes
from tests._util import tiny_scene

CFG = OracleConfig(k_road=16, n_partners=8, episode_len=30, term_collision=True, term_offroad=True,
                   nontrivial_init=True)


def test_static_marking_is_the_distance_rule_and_survives_reset():
    sc = scenes.make_scene(np.array([20, 35, 9]), np.array([800, 1500, 600]), 6, type_mix=(0.6, 0.2, 0.2),
                           parked_frac=0.5)
    d = np.hypot(sc.x.astype(np.float64) - sc.goal_x, sc.y.astype(np.float64) - sc.goal_y)
    orc = Oracle(sc, CFG)
    f = orc.get_state()[1]
    np.testing.assert_array_equal((f & STATIC) != 0, d <= 2.0)
    assert 0.2 < (d <= 2.0).mean() < 0.8
    acts = scenes.make_actions(5, sc.num_agents, 6)
    for t in range(5):
        orc.step(acts[t])
    orc.reset()
    np.testing.assert_array_equal(orc.get_state()[1], f)
    # without the mode nobody is static
    assert (Oracle(sc, OracleConfig(k_road=16, n_partners=8)).get_state()[1] == 0).all()


def test_uncontrolled_agents_stay_put_score_nothing_and_report_done():
    sc = scenes.make_scene(np.array([24, 16]), np.array([1200, 900]), 7, parked_frac=0.5)
    orc = Oracle(sc, CFG)
    s0, f0 = orc.get_state()[:2]
    static = (f0 & STATIC) != 0
    assert static.any() and (~static).any()
    acts = scenes.make_actions(12, sc.num_agents, 7)
    for t in range(12):
        out = orc.step(acts[t])
        s, f = orc.get_state()[:2]
        assert (s[static] == s0[static]).all()
        assert (f[static] == STATIC).all()
        assert (out["reward"][static] == 0).all() and (out["done"][static] == 1).all()
    assert (s[~static] != s0[~static]).any()


def _agent(x, y, th, v, gx, gy, typ=0):
    return (x, y, th, v, 4.5, 2.0, gx, gy, typ)


def test_driving_into_a_parked_car_is_a_collision_and_parked_cars_are_seen():
    parked = _agent(10.0, 0.0, 0.0, 0.0, 10.5, 0.0)                  # 0.5 m from its goal: not controlled
    mover = _agent(0.0, 0.0, 0.0, 20.0, 200.0, 0.0)                  # heads straight into it
    sc = tiny_scene([([mover, parked], [])])
    orc = Oracle(sc, CFG)
    assert list(orc.get_state()[1]) == [0, STATIC]
    obs, ridx, pidx = orc.observe()
    assert pidx[0, 0] == 1                                          # the parked car is the mover's partner
    lid = orc.lidar(101, 0.5)
    assert lid["cls"][0, 50] == 1 and abs(lid["depth"][0, 50] - 7.75) < 1e-9
    hit = False
    for t in range(5):
        orc.step(np.zeros((2, 2), np.float32))
        f = orc.get_state()[1]
        hit = hit or bool(f[0] & COLLIDED)
        assert f[1] == STATIC
        if f[0] & DONE:
            break
    assert hit and (f[0] & DONE)                                    # collision ends the mover's episode


def test_episode_end_counts_controlled_agents_only():
    goal_reacher = _agent(0.0, 0.0, 0.0, 5.0, 3.0, 0.0)             # reaches its goal on the first steps
    parked = _agent(50.0, 50.0, 0.0, 0.0, 50.0, 51.0)
    sc = tiny_scene([([goal_reacher, parked], []), ([parked, parked], [])])
    orc = Oracle(sc, CFG)
    ends = []
    for t in range(30):
        out = orc.step(np.zeros((4, 2), np.float32))
        ends.append(out["world_done"].copy())
    ends = np.array(ends)
    first = np.argmax(ends[:, 0])
    assert ends[first, 0] == 1 and first < 5                        # ended by its one controlled agent
    assert ends[:-1, 1].sum() == 0 and ends[-1, 1] == 1             # no controlled agent: only the time limit


def test_pedestrians_cross_edges_vehicles_and_cyclists_do_not():
    # three agents driving across the same road edge, one of each type
    edge = [(-100.0, 5.0, 1, 0), (100.0, 5.0, 1, 0)]
    ag = [_agent(-20.0, 0.0, 1.5707963, 15.0, -20.0, 300.0, 0), _agent(0.0, 0.0, 1.5707963, 15.0, 0.0, 300.0, 1),
          _agent(20.0, 0.0, 1.5707963, 15.0, 20.0, 300.0, 2)]
    sc = tiny_scene([(ag, edge)])
    orc = Oracle(sc, OracleConfig(k_road=4, n_partners=2, episode_len=30))
    off = np.zeros(3, bool)
    for t in range(8):
        orc.step(np.zeros((3, 2), np.float32))
        off |= (orc.get_state()[1] & OFFROAD) != 0
    assert off[0] and off[1] and not off[2]
