"""GPU parity of the Visvalingam-Whyatt decimation (Sec. 3.1) against the
oracle, through the C ABI.  Both take every elimination decision in float32
with the same rounding, so the keep masks must be identical bit for bit:
random polylines (lengths 0 to 3 included, collinear runs, tied areas),
0.1 m-sampled synthetic roads, and the 256 x 64 dense-road workload at full
size.  A decimated scene then runs through the library with the oracle
teacher-forced on the same decimated scene."""
import numpy as np
import pytest

from oracle import OracleConfig
from oracle.oracle import decimate
from paper_2408_01584_b300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _gpu(off, x, y, tol):
    from paper_2408_01584_b300 import gd
    keep = torch.empty(len(x), dtype=torch.uint8, device="cuda")
    gd.gd_decimate(torch.from_numpy(off).cuda(), torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), tol, keep)
    torch.cuda.synchronize()
    return keep.cpu().numpy()


def test_random_polylines_bitwise():
    rng = np.random.default_rng(1)
    # short ones (a warp each, shared memory) and ones past 1,024 points (a
    # thread each, heap in global scratch), both forms in one call
    lens = np.concatenate([[0, 1, 2, 3, 3], rng.integers(3, 400, 300), [1023, 1024, 1025, 2500]])
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    pts = []
    for k, n in enumerate(lens):
        p = np.cumsum(rng.normal(size=(n, 2)) * np.array([1.0, 0.2]), axis=0)
        if k % 4 == 1:
            p = np.round(p * 4) / 4                 # ties
        if k % 4 == 2 and n:
            p[:, 1] = 0.5 * p[:, 0]                 # collinear
        pts.append(p)
    xy = np.concatenate(pts).astype(np.float32)
    for tol in (0.0, 1e-3, 0.05, 1.0):
        np.testing.assert_array_equal(_gpu(off, xy[:, 0].copy(), xy[:, 1].copy(), tol),
                                      decimate(off, xy[:, 0], xy[:, 1], tol), err_msg=f"tol {tol}")


def test_dense_workload_full_size_bitwise():
    from paper_2408_01584_b300 import gd
    sc = scenes.workload_scene("dense_roads_256x64", 0)
    off = gd.polylines(sc)
    g = _gpu(off, sc.road_x, sc.road_y, gd.DECIMATE_AREA)
    o = decimate(off, sc.road_x, sc.road_y, gd.DECIMATE_AREA)
    np.testing.assert_array_equal(g, o)
    ratio = len(g) / g.sum()
    print(f"dense roads: {len(g)} -> {int(g.sum())} points ({ratio:.1f}x) over {len(off) - 1} polylines")
    assert 10.0 <= ratio <= 15.0


def test_decimated_scene_runs_and_matches_oracle():
    from paper_2408_01584_b300 import gd
    from tests.test_parity_gpu import teacher_forced
    sc = scenes.make_scene(np.array([6, 17, 30]), np.array([8000, 12000, 20000]), 4, n_poly=np.array([8, 12, 20]),
                           spacing=0.1)
    dsc, keep = gd.decimate_scene(sc)
    assert dsc.num_road == int(keep.sum()) and dsc.num_road < sc.num_road / 8
    np.testing.assert_array_equal(dsc.road_x, sc.road_x[keep == 1])
    ocfg = OracleConfig(k_road=64, n_partners=16, episode_len=12, term_collision=True, term_offroad=True,
                        auto_reset=True)
    acts = scenes.make_actions(15, dsc.num_agents, 4)
    _, ex = teacher_forced(dsc, ocfg, 15, acts, obs_every=3)
    print("exceptions:", ex.items)


def test_decimate_scene_c_abi_full_size():
    # gd_decimate_scene: the polylines split (maximal runs of one world's
    # points with one id), decimated and compacted behind the C ABI, on the
    # full 256 x 64 dense-road workload; keep mask bitwise against the
    # oracle's on polylines split here independently, compaction against
    # numpy masking
    from paper_2408_01584_b300 import gd
    sc = scenes.workload_scene("dense_roads_256x64", 0)
    starts = [p for w in range(sc.num_worlds) for p in range(sc.road_off[w], sc.road_off[w + 1])
              if p == sc.road_off[w] or sc.road_poly[p] != sc.road_poly[p - 1]]
    off = np.array(starts + [sc.num_road], np.int32)
    ref = decimate(off, sc.road_x, sc.road_y, gd.DECIMATE_AREA)
    dsc, keep = gd.decimate_scene(sc)
    np.testing.assert_array_equal(keep, ref)
    m = ref.astype(bool)
    np.testing.assert_array_equal(dsc.road_x, sc.road_x[m])
    np.testing.assert_array_equal(dsc.road_y, sc.road_y[m])
    np.testing.assert_array_equal(dsc.road_type, sc.road_type[m])
    np.testing.assert_array_equal(dsc.road_poly, sc.road_poly[m])
    world = np.repeat(np.arange(sc.num_worlds), np.diff(sc.road_off))
    np.testing.assert_array_equal(np.diff(dsc.road_off), np.bincount(world[m], minlength=sc.num_worlds))
    np.testing.assert_array_equal(dsc.x, sc.x)          # agents untouched
    print(f"gd_decimate_scene: {sc.num_road} -> {dsc.num_road} points over {len(off) - 1} polylines")
