"""Pins of the oracle's LiDAR / view-cone scan (Sec. 3.2 "Sensor modalities").

* closed forms: a straight road edge (depth = D / cos(angle), nothing past
  R, the R bound inclusive, lane centre lines transparent) and a box seen
  head-on and turned (front face 1 / cos, side faces 1 / sin);
* special cases: an agent inside another box sees it at depth 0 on every
  ray; a near box hides a far one until the near agent is done; a done
  agent sees nothing;
* the same geometry by two formulas: boxes replaced by road-edge polylines
  along their outlines give the same depths (slab test vs. segment test);
* invariances: a view cone with head rotation j * (ray spacing) equals the
  matching rays of the full scan; a rigid motion of the whole scene leaves
  every depth and class unchanged.
"""
import math

import numpy as np

from oracle import Oracle, OracleConfig
from paper_2408_01584_b300 import scenes
from tests._util import tiny_scene

CFG = OracleConfig(k_road=8, n_partners=4, episode_len=91)
R = CFG.obs_radius


def _angles(theta, n, fov, head=0.0):
    k = np.arange(n)
    return theta + head + (-fov / 2 + (k + 0.5) * fov / n)


def _ego(x=0.0, y=0.0, th=0.0):
    return (x, y, th, 0.0, 4.5, 2.0, 900.0, 900.0, 0)


def test_wall_closed_form_range_and_lane_transparency():
    th, D, n = 0.3, 20.0, 720
    road = [(D, -100.0, 1, 0), (D, 100.0, 1, 0),              # road edge x = D
            (D / 2, -100.0, 0, 1), (D / 2, 100.0, 0, 1),      # lane centre line: not an obstacle
            (80.0, -100.0, 1, 2), (80.0, 100.0, 1, 2)]        # road edge beyond R
    sc = tiny_scene([([_ego(th=th)], road)])
    out = Oracle(sc, CFG).lidar(n)
    phi = _angles(np.float64(np.float32(th)), n, 2 * math.pi)
    c = np.cos(phi)
    hit = (c > 0) & (D / np.where(c > 0, c, 1) <= R)
    exp = np.where(hit, D / np.where(hit, c, 1), R)
    np.testing.assert_allclose(out["depth"][0], exp, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(out["cls"][0], np.where(hit, 2, 0))
    assert hit.sum() > 100


def test_range_bound_is_inclusive():
    # odd ray count: the middle ray of the cone points straight along the heading
    n, fov = 201, 2 * math.pi / 3
    sc = tiny_scene([([_ego()], [(R, -10.0, 1, 0), (R, 10.0, 1, 0)])])
    out = Oracle(sc, CFG).lidar(n, fov)
    assert out["cls"][0, 100] == 2 and out["depth"][0, 100] == R
    assert out["cls"][0, 0] == 0 and out["depth"][0, 0] == R


def _box_depth(beta, x0, x1, hw):
    """Ray from the origin at angle beta against the box [x0, x1] x [-hw, hw]."""
    t = np.abs(np.tan(beta))
    front = (np.cos(beta) > 0) & (t * x0 <= hw)
    xs = hw / np.where(t > 0, t, 1)
    sb = np.where(np.sin(beta) != 0, np.abs(np.sin(beta)), 1)
    side = ~front & (np.cos(beta) > 0) & (t > 0) & (xs >= x0) & (xs <= x1)
    d = np.where(front, x0 / np.cos(beta), np.where(side, hw / sb, R))
    return d, np.where(front | side, 1, 0)


def test_box_closed_form_head_on_and_turned():
    n, fov = 601, 2 * math.pi / 3
    beta = _angles(0.0, n, fov)
    # box of 4.5 x 2 m centred 10 m ahead, aligned with the ego
    sc = tiny_scene([([_ego(), (10.0, 0.0, 0.0, 0.0, 4.5, 2.0, 0.0, 0.0, 0)], [])])
    out = Oracle(sc, CFG).lidar(n, fov, agents=[0])
    d, c = _box_depth(beta, 7.75, 12.25, 1.0)
    assert out["depth"][0, 300] == 7.75 and out["cls"][0, 300] == 1
    np.testing.assert_allclose(out["depth"][0], d, rtol=1e-12)
    np.testing.assert_array_equal(out["cls"][0], c)
    # the same box turned by 90 degrees: 2 m deep, 4.5 m wide
    sc = tiny_scene([([_ego(), (10.0, 0.0, math.pi / 2, 0.0, 4.5, 2.0, 0.0, 0.0, 0)], [])])
    out = Oracle(sc, CFG).lidar(n, fov, agents=[0])
    d, c = _box_depth(beta, 9.0, 11.0, 2.25)
    # float32(pi/2) turns the box by 4e-8 rad more: corners move by about 1e-7 m
    np.testing.assert_allclose(out["depth"][0], d, rtol=1e-9, atol=1e-6)
    np.testing.assert_array_equal(out["cls"][0][out["fragile"][0] == 0], c[out["fragile"][0] == 0])


def test_inside_a_box_every_ray_stops_at_zero():
    sc = tiny_scene([([_ego(), (1.0, 0.5, 0.4, 0.0, 4.5, 2.0, 0.0, 0.0, 0)],
                      [(5.0, -10.0, 1, 0), (5.0, 10.0, 1, 0)])])
    out = Oracle(sc, CFG).lidar(360, agents=[0])
    assert (out["depth"][0] == 0).all() and (out["cls"][0] == 1).all()


def test_occlusion_and_done_agents():
    n, fov = 101, 0.5
    agents = [_ego(), (10.0, 0.0, 0.0, 0.0, 4.5, 2.0, 0.0, 0.0, 0), (20.0, 0.0, 0.0, 0.0, 4.5, 6.0, 0.0, 0.0, 0)]
    sc = tiny_scene([(agents, [])])
    orc = Oracle(sc, CFG)
    out = orc.lidar(n, fov, agents=[0])
    d1, _ = _box_depth(_angles(0.0, n, fov), 7.75, 12.25, 1.0)
    d2, _ = _box_depth(_angles(0.0, n, fov), 17.75, 22.25, 3.0)
    exp = np.minimum(d1, d2)
    np.testing.assert_allclose(out["depth"][0], exp, rtol=1e-12)
    assert (d2 < d1).any() and (d1 < d2).any()           # both boxes are seen, the far one only past the near
    # the near agent is done: it has left the scene and the far box shows through
    orc.set_state(flags=np.array([0, 1, 0], np.uint8))
    out = orc.lidar(n, fov, agents=[0, 1])
    np.testing.assert_allclose(out["depth"][0], d2, rtol=1e-12)
    assert (out["depth"][1] == 0).all() and (out["cls"][1] == 0).all()   # a done agent sees nothing


def _outline_scene(sc, ego):
    """Scene with only agent `ego`; every other agent's box becomes a closed
    road-edge polyline along its outline."""
    ag = [(float(sc.x[ego]), float(sc.y[ego]), float(sc.theta[ego]), 0.0, float(sc.length[ego]),
           float(sc.width[ego]), 900.0, 900.0, 0)]
    road, poly = [], 0
    for j in range(sc.num_agents):
        if j == ego:
            continue
        c, s = math.cos(float(sc.theta[j])), math.sin(float(sc.theta[j]))
        hl, hw = float(sc.length[j]) / 2, float(sc.width[j]) / 2
        pts = [(hl, hw), (-hl, hw), (-hl, -hw), (hl, -hw), (hl, hw)]
        for (u, v) in pts:
            road.append((float(sc.x[j]) + c * u - s * v, float(sc.y[j]) + s * u + c * v, 1, poly))
        poly += 1
    return tiny_scene([(ag, road)])


def test_box_outline_as_road_edges_gives_the_same_depths():
    sc = scenes.make_scene(np.array([12]), np.array([400]), 3)
    orc = Oracle(sc, CFG)
    n = 1440
    box_scan = orc.lidar(n)
    checked = 0
    for ego in range(sc.num_agents):
        # road-free copy: the boxes alone against their outlines
        alone = tiny_scene([([(float(sc.x[j]), float(sc.y[j]), float(sc.theta[j]), 0.0, float(sc.length[j]),
                                float(sc.width[j]), 900.0, 900.0, 0) for j in range(sc.num_agents)], [])])
        a = Oracle(alone, CFG).lidar(n, agents=[ego])
        b = Oracle(_outline_scene(sc, ego), CFG).lidar(n)
        ok = (a["fragile"][0] == 0) & (b["fragile"][0] == 0) & (a["depth"][0] > 0)
        # outline vertices are float32 (about 4e-6 m off): the depth moves by
        # that over the sine of the incidence angle, 1 + sens / depth at most
        tol = 1e-5 * (1 + a["sens"][0] / np.maximum(a["depth"][0], 1.0))
        assert (np.abs(a["depth"][0] - b["depth"][0]) <= tol)[ok].all()
        np.testing.assert_array_equal(np.where(a["cls"][0][ok] == 1, 2, 0), b["cls"][0][ok])
        checked += int(ok.sum() and (a["cls"][0][ok] == 1).sum())
    assert checked > 0
    assert box_scan["depth"].shape == (sc.num_agents, n)


def test_view_cone_with_head_rotation_equals_the_full_scan():
    sc = scenes.make_scene(np.array([9, 14]), np.array([700, 1200]), 5)
    orc = Oracle(sc, CFG)
    n_full, n_cone, fov = 3000, 1000, 2 * math.pi / 3     # same ray spacing
    full = orc.lidar(n_full)
    step = 2 * math.pi / n_full
    rng = np.random.default_rng(5)
    j = rng.integers(-400, 400, sc.num_agents)
    head = (j * step).astype(np.float32)
    cone = orc.lidar(n_cone, fov, head=head)
    hd = head.astype(np.float64) - j * step               # float32 rounding of the head angle
    idx = (np.arange(n_cone)[None, :] + 1000 + j[:, None]) % n_full
    fd = np.take_along_axis(full["depth"], idx, 1)
    fc = np.take_along_axis(full["cls"], idx, 1)
    ok = (cone["fragile"] == 0) & (np.take_along_axis(full["fragile"], idx, 1) == 0)
    tol = 1e-9 + np.abs(hd)[:, None] * (cone["sens"] + 1) * 2
    assert (np.abs(cone["depth"] - fd) <= tol)[ok].all()
    assert (cone["cls"] == fc)[ok].all()
    assert ok.mean() > 0.99 and (fc[ok] == 2).mean() > 0.05 and (fc[ok] == 1).any()


def test_rigid_motion_leaves_the_scan_unchanged():
    sc = scenes.make_scene(np.array([10, 16]), np.array([800, 1500]), 7)
    n = 2000
    a = Oracle(sc, CFG).lidar(n)
    b = Oracle(sc.transformed(0.7, 31.0, -12.0), CFG).lidar(n)
    ok = (a["fragile"] == 0) & (b["fragile"] == 0)
    # moved coordinates are rounded to float32 (about 1e-5 m)
    tol = 1e-4 + 1e-5 * a["sens"]
    assert (np.abs(a["depth"] - b["depth"]) <= tol)[ok].all()
    assert (a["cls"] == b["cls"])[ok].all()
    assert ok.mean() > 0.99
    print(f"rigid motion: {ok.size} rays, {(~ok).sum()} fragile, classes {np.bincount(a['cls'].ravel())}")
