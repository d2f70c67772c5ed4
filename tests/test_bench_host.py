"""Host-side logic of bench.py (no GPU): the active and controlled agent-step
counts on hand-made done traces, and the throughput arithmetic."""
import numpy as np

import bench


def test_active_agent_steps_hand_trace():
    # two worlds: [0, 1] and [2]; T = 4
    off = np.array([0, 2, 3])
    done = np.array([[0, 1, 0],      # after step 0: agent 1 done
                     [0, 1, 0],
                     [1, 1, 1],      # after step 2: everyone done -> both worlds restart
                     [0, 0, 0]], np.uint8)
    # step 0: 3 in; step 1: agent 1 out -> 2; step 2: 2; step 3: worlds ended -> all 3 back
    assert bench.active_agent_steps(done, off) == 3 + 2 + 2 + 3


def test_controlled_agent_steps_excludes_uncontrolled_agents():
    off = np.array([0, 3, 5])
    static = np.array([False, True, False, True, True])       # world 1 has no controlled agent
    done = np.array([[0, 1, 0, 1, 1],
                     [1, 1, 0, 1, 1],
                     [1, 1, 1, 1, 1],                        # world 0's controlled agents both done: restart
                     [0, 1, 0, 1, 1]], np.uint8)
    # controlled agents: 0 and 2; step 0: 2; step 1: 2; step 2: agent 0 out -> 1; step 3: restart -> 2
    assert bench.controlled_agent_steps(done, static, off) == 2 + 2 + 1 + 2
    # with nobody static it is the active count
    assert bench.controlled_agent_steps(done, np.zeros(5, bool), off) == bench.active_agent_steps(done, off)


def test_whole_job_rate_single_rank():
    t, rate = bench.whole_job_rate(1000, 250.0, 1, None)
    assert t == 250.0 and rate == 1000 / 0.25


def test_kernel_record_arithmetic():
    # 1 GB per launch in 1 ms is 1,000 GB/s: half of a 2,000 GB/s peak
    r = bench.kernel_record("k", 4, 4.0, 1e9, 2000.0, "n")
    assert r["launches"] == 4 and abs(r["avg_launch_us"] - 1000.0) < 1e-9
    assert abs(r["achieved_gbs"] - 1000.0) < 1e-6 and abs(r["frac"] - 0.5) < 1e-9 and r["note"] == "n"


def test_measured_traffic_keyed_on_sources_and_shape(tmp_path, monkeypatch):
    import json
    import os
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench._kernel_source_hash("k_observe_split")
    shape = {"block_size": 128, "road_cell_m": 8.0, "road_tile": 0, "obs_split": 1}
    with open(prof / "k_observe_split_w.traffic.json", "w") as f:
        json.dump({"dram_bytes_per_launch": 5.0, "source_hash": h, "shape": shape}, f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_kernel_source_hash", lambda k: h)
    assert bench._measured_traffic("w", "k_observe_split", shape) == 5.0
    assert bench._measured_traffic("w", "k_observe_split", dict(shape, road_cell_m=12.0)) is None
    monkeypatch.setattr(bench, "_kernel_source_hash", lambda k: "other")
    assert bench._measured_traffic("w", "k_observe_split", shape) is None


def test_observation_traffic_record_is_current():
    # the bench's roofline line carries the DRAM traffic of the observation
    # launch from the committed ncu capture only while that capture was taken
    # of the current kernel sources at the tuned shape; a kernel edit must
    # come with a new capture (profiles/k_observe_split_plain_1024x64.*)
    import json
    import os
    path = os.path.join(bench.ROOT, "profiles", "k_observe_split_plain_1024x64.traffic.json")
    rec = json.load(open(path))
    assert rec["source_hash"] == bench._kernel_source_hash("k_observe_split")
    got = bench._measured_traffic("plain_1024x64", "k_observe_split", rec["shape"])
    assert got == rec["dram_bytes_per_launch"] > 0
