"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/gd.h declares, its structs have the layout the
binding assumes, and bad arguments are rejected before any CUDA call."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2408_01584_b300 import gd, scenes
from paper_2408_01584_b300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gd.h")


@pytest.fixture(scope="module")
def lib():
    build()
    return gd.load_library()


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gd_[a-z_]+)\s*\(", src)))


def test_header_and_binding_agree(lib):
    names = declared()
    assert set(names) == set(gd.SYMBOLS), set(names) ^ set(gd.SYMBOLS)
    for n in names:
        assert hasattr(lib, n), n


def test_exported_symbols_with_nm(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", gd.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gd_[a-z_]+)$", out, flags=re.M))
    assert set(declared()) <= exported


def test_struct_layout_matches_header(tmp_path):
    prog = tmp_path / "layout.c"
    fields = {"gd_config": [f for f, _ in gd.gd_config._fields_],
              "gd_scene_batch": [f for f, _ in gd.gd_scene_batch._fields_],
              "gd_info": [f for f, _ in gd.gd_info._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for s, fs in fields.items():
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f in fs:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", str(prog), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n") if l)
    for s, cls in (("gd_config", gd.gd_config), ("gd_scene_batch", gd.gd_scene_batch), ("gd_info", gd.gd_info)):
        assert int(got[s]) == C.sizeof(cls), s
        for f in fields[s]:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, (s, f)


def test_default_config(lib):
    c = gd.gd_default_config()
    assert (c.k_road, c.n_partners, c.episode_len, c.ckpt_every) == (200, 63, 91, 10)
    assert abs(c.obs_radius - 50) < 1e-6 and abs(c.goal_radius - 2) < 1e-6 and abs(c.dt - 0.1) < 1e-7
    assert c.lidar_rays == 0 and abs(c.lidar_fov - 2 * np.pi) < 1e-6


def _expect(status, fn, *a):
    with pytest.raises(gd.GdError) as e:
        fn(*a)
    assert e.value.status == status, str(e.value)
    return str(e.value)


def test_rejects_bad_arguments_before_any_launch(lib):
    sc = scenes.workload_scene("plain_4x8", 0)
    INV, CAP = 1, 4
    _expect(CAP, gd.gd_create, gd.gd_default_config(k_road=257), sc)
    _expect(CAP, gd.gd_create, gd.gd_default_config(n_partners=128), sc)
    _expect(INV, gd.gd_create, gd.gd_default_config(episode_len=0), sc)
    _expect(INV, gd.gd_create, gd.gd_default_config(obs_radius=0.0), sc)
    _expect(INV, gd.gd_create, gd.gd_default_config(dt=-0.1), sc)
    _expect(INV, gd.gd_create, gd.gd_default_config(block_size=96), sc)
    _expect(INV, gd.gd_create, gd.gd_default_config(flags=gd.GD_DIFFERENTIABLE | gd.GD_AUTO_RESET), sc)
    _expect(CAP, gd.gd_create, gd.gd_default_config(lidar_rays=gd.GD_MAX_LIDAR_RAYS + 1), sc)
    _expect(CAP, gd.gd_create, gd.gd_default_config(lidar_rays=-1), sc)
    _expect(INV, gd.gd_create, gd.gd_default_config(lidar_rays=100, lidar_fov=1e-4), sc)
    _expect(INV, gd.gd_create, gd.gd_default_config(lidar_rays=100, lidar_fov=7.0), sc)
    _expect(INV, gd.gd_create, gd.gd_default_config(lidar_rays=100, lidar_block_size=512), sc)
    _expect(INV, gd.gd_create, gd.gd_default_config(lidar_rays=100, lidar_no_tile=2), sc)
    _expect(INV, gd.gd_create, gd.gd_default_config(lidar_rays=100, lidar_split=3), sc)
    _expect(INV, gd.gd_create, gd.gd_default_config(dynamics=2), sc)
    _expect(INV, gd.gd_create, gd.gd_default_config(nontrivial_dist=-1.0), sc)
    _expect(INV, gd.gd_create, gd.gd_default_config(road_no_tile=2), sc)
    _expect(INV, gd.gd_create, gd.gd_default_config(obs_split=2), sc)
    assert gd.gd_default_config().obs_split == 1      # split observation by default
    big = scenes.make_scene(np.array([129]), np.array([500]), 0)
    _expect(CAP, gd.gd_create, gd.gd_default_config(), big)
    bad = scenes.workload_scene("plain_4x8", 0)
    bad.agent_off = bad.agent_off.copy()
    bad.agent_off[2] = bad.agent_off[1] - 1
    _expect(INV, gd.gd_create, gd.gd_default_config(), bad)
    nan = scenes.workload_scene("plain_4x8", 0)
    nan.theta = nan.theta.copy()
    nan.theta[3] = np.nan
    msg = _expect(INV, gd.gd_create, gd.gd_default_config(), nan)
    assert "agent 3" in msg
    assert "agent 3" in gd.gd_last_error(None)
    neg = scenes.workload_scene("plain_4x8", 0)
    neg.length = neg.length.copy()
    neg.length[0] = 0.0
    _expect(INV, gd.gd_create, gd.gd_default_config(), neg)
    # decimation: validated before any CUDA call
    assert lib.gd_decimate(-1, 10, None, None, None, C.c_float(1e-3), None, None) == INV
    assert lib.gd_decimate(1, 10, None, None, None, C.c_float(float("nan")), None, None) == INV
    assert lib.gd_decimate(1, 10, None, None, None, C.c_float(1e-3), None, None) == INV
    assert lib.gd_decimate(0, 0, None, None, None, C.c_float(1e-3), None, None) == 0
    assert "NULL" in gd.gd_last_error(None) or "must" in gd.gd_last_error(None)
    # scene-level decimation: validated before any CUDA call
    arrs = gd._scene_arrays(sc)
    sb = gd.gd_scene_batch(num_worlds=sc.num_worlds, **{k: a.ctypes.data for k, a in arrs.items()})
    off = np.zeros(sc.num_worlds + 1, np.int32)
    kept = C.c_int32(0)
    pv = lambda a: a.ctypes.data_as(C.c_void_p)
    assert lib.gd_decimate_scene(None, C.c_float(1e-3), None, None, pv(off), None, None, None, None,
                                 C.byref(kept)) == INV
    assert lib.gd_decimate_scene(C.byref(sb), C.c_float(-1.0), None, None, pv(off), None, None, None, None,
                                 C.byref(kept)) == INV
    assert lib.gd_decimate_scene(C.byref(sb), C.c_float(1e-3), None, None, pv(off), None, None, None, None,
                                 C.byref(kept)) == INV                     # output arrays missing
    assert "road_x_out" in gd.gd_last_error(None)
    bad_off = arrs["road_off"].copy()
    bad_off[2] = bad_off[1] - 1
    sb2 = gd.gd_scene_batch(num_worlds=sc.num_worlds, **dict({k: a.ctypes.data for k, a in arrs.items()},
                                                              road_off=bad_off.ctypes.data))
    assert lib.gd_decimate_scene(C.byref(sb2), C.c_float(1e-3), None, None, pv(off), None, None, None, None,
                                 C.byref(kept)) == INV
    assert "non-decreasing" in gd.gd_last_error(None)
    # NULL out pointer
    cfg = gd.gd_default_config()
    assert lib.gd_create(C.byref(cfg), None, None, None) == INV
    assert lib.gd_destroy(None) == 0
