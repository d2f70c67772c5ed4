"""Throughput benchmark: agent-steps/s of the batched driving step on B300.

Agent-steps/s (ASPS) = S * sum_k |A_k| / dT  (Sec. 4.1, Eq. ASPS): S steps of
every world, all agents counted.  One benchmark "step" is one full episode
(T = 91 simulator steps of every world: reset, dynamics, collision,
off-road, reward/done and the observation) over one batch of seeded
synthetic actions.  Inputs are resident in HBM when the timed region starts
(`value`); `e2e` repeats the measurement through gd_rollout with host
buffers and the copies inside the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload plain_1024x64] [--no-cpu-baseline] [--no-extras]
       python bench.py --profile [--shape B,C,T] [--lidar N [--fov DEG]] [--worlds W] [--fwdbwd]
                       (one leg alone, for ncu captures)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "agent-steps/s"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")


# Device headers each profiled kernel is compiled from.
KERNEL_SOURCES = {
    "k_observe_split": ("gd_device.cuh", "observe_kernel.cuh"),
    # the fused kernel also embeds the LiDAR arguments in its parameter block
    "k_world": ("gd_device.cuh", "observe_kernel.cuh", "world_kernel.cuh", "lidar_kernel.cuh"),
}


def _kernel_source_hash(kernel="k_world"):
    """Hash of what `kernel` is compiled from: its device headers and the
    constants (#define lines) of the C header.  The header's structs are
    host-side and do not enter the kernel."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2408_01584_b300", "csrc")
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(ROOT, "include", "gd.h")) as fh:
        h.update("".join(l for l in fh if l.startswith("#define GD_")).encode())
    return h.hexdigest()[:16]


def _measured_traffic(workload, kernel="k_world", shape=None):
    """DRAM bytes per launch of `kernel` from the committed ncu capture of
    this workload, or None when the kernel sources changed since the capture
    or the capture's kernel shape (CTA size, road cell, tile, split) is not
    the one in use."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("source_hash") != _kernel_source_hash(kernel):
        return None
    if shape is not None and rec.get("shape") != shape:
        return None
    return rec["dram_bytes_per_launch"]


def _peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class Clocks:
    """SM clock and throttle-reason sampling (NVML, every 5 ms) during a
    timed region; the device is matched to the CUDA device by PCI bus id."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, torch_device):
        import threading
        self.dev = torch_device
        self.samples = []
        self.stop = threading.Event()
        self.thread = None
        self.err = None

    def _handle(self):
        import pynvml
        import torch
        pynvml.nvmlInit()
        p = torch.cuda.get_device_properties(self.dev)
        bus = f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
        return pynvml, pynvml.nvmlDeviceGetHandleByPciBusId(bus)

    def _run(self, nv, h):
        while not self.stop.is_set():
            try:
                self.samples.append((nv.nvmlDeviceGetClockInfo(h, nv.NVML_CLOCK_SM),
                                     nv.nvmlDeviceGetMaxClockInfo(h, nv.NVML_CLOCK_SM),
                                     nv.nvmlDeviceGetCurrentClocksEventReasons(h),
                                     nv.nvmlDeviceGetPowerUsage(h) / 1000.0))
            except Exception as e:  # keep timing even if one read fails
                self.err = repr(e)
            self.stop.wait(0.005)

    def _smi(self):
        """Fallback: nvidia-smi every 20 ms for the same PCI bus id."""
        import subprocess
        import torch
        p = torch.cuda.get_device_properties(self.dev)
        bus = f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        self.proc = subprocess.Popen(["nvidia-smi", f"--id={bus}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                      "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)

    def __enter__(self):
        import threading
        self.proc = None
        try:
            nv, h = self._handle()
            self.thread = threading.Thread(target=self._run, args=(nv, h), daemon=True)
            self.thread.start()
        except Exception as e:
            self.err = repr(e)
            try:
                self._smi()
            except Exception as e2:
                self.err += " / " + repr(e2)
        return self

    def __exit__(self, *a):
        self.stop.set()
        if self.thread is not None:
            self.thread.join(timeout=2)
        if self.proc is not None:
            self.proc.terminate()
            out, _ = self.proc.communicate(timeout=5)
            bits = (0x8, 0x40, 0x20, 0x4)
            for line in out.splitlines():
                f = [x.strip() for x in line.split(",")]
                if len(f) < 7:
                    continue
                try:
                    r = sum(b for b, v in zip(bits, f[3:7]) if v.lower() == "active")
                    self.samples.append((float(f[0]), float(f[1]), r, float(f[2])))
                except ValueError:
                    pass

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [f"no samples ({self.err})"]}
        sm = [x[0] for x in self.samples]
        reasons = sorted({name for x in self.samples for bit, name in self.REASONS.items() if x[2] & bit})
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(x[1] for x in self.samples),
               "reasons": reasons, "samples": len(self.samples),
               "power_w_max": max(x[3] for x in self.samples),
               "source": "nvml 5 ms" if self.proc is None else "nvidia-smi 20 ms"}
        if self.proc is not None and self.err:
            out["nvml_error"] = self.err[:200]
        return out


def workload_description(name, seed=0):
    """The workload keys of the JSON line's config, shared by both arms."""
    from paper_2408_01584_b300 import scenes
    wl = scenes.WORKLOADS[name]
    sc = scenes.workload_scene(name, seed)
    return {"workload": name, "worlds": sc.num_worlds, "agents": sc.num_agents, "road_points": sc.num_road,
            "k_road": wl["k_road"], "n_partners": wl["n_partners"], "episode_steps": wl["steps"],
            "feat": 8 + 8 * wl["n_partners"] + 4 * wl["k_road"], "step": f"one {wl['steps']}-step episode of every world"}


def workload_cfg(name):
    from paper_2408_01584_b300 import gd, scenes
    wl = scenes.WORKLOADS[name]
    fl = (gd.GD_TERM_COLLISION if wl["term_collision"] else 0) | (gd.GD_TERM_OFFROAD if wl["term_offroad"] else 0) \
        | (gd.GD_AUTO_RESET if wl["auto_reset"] else 0) | (gd.GD_NONTRIVIAL_INIT if wl.get("nontrivial_init") else 0)
    return dict(k_road=wl["k_road"], n_partners=wl["n_partners"], episode_len=wl["steps"], flags=fl)


# Observation launch of the split form, per agent besides the row (4F) and
# the road: the agent's state (16 B), extents and goal (16 B) and flags (1 B).
OBS_AGENT_BYTES = 33.0
# Step launch per agent: reads state 16, extents and goal 16, flags 1, type 1,
# action 8; writes state 16, flags 1, reward 4, done 1.  The road-edge
# segments the off-road test reads are not counted (they are not in the
# algorithmic byte formula; the step's DRAM traffic is about 3.6x this).
STEP_AGENT_BYTES = 64.0
# Checkpoint copy per agent: state and flags read and written.
SNAPSHOT_AGENT_BYTES = 34.0


def kernel_record(name, launches, total_ms, bytes_per_launch, peak, note=None):
    """One kernel's roofline line: average launch duration (CUDA events) and
    algorithmic bytes per launch against the HBM peak."""
    us = total_ms * 1e3 / max(launches, 1)
    gbs = bytes_per_launch / (us * 1e-6) / 1e9 if us > 0 else None
    rec = {"kernel": name, "launches": int(launches), "avg_launch_us": us,
           "algorithmic_bytes_per_launch": bytes_per_launch, "achieved_gbs": gbs,
           "frac": gbs / peak if gbs else None, "bound": "hbm"}
    if note:
        rec["note"] = note
    return rec


def per_kernel_launch_us(env, actions, T, stream, flush):
    """Average duration of the step launch and of the observation launch of
    the split form, from CUDA events around each launch of one episode issued
    call by call (gd_step, then gd_observe) after an L2 flush."""
    import torch
    from paper_2408_01584_b300 import gd
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(T)]
    gd.gd_reset(env.h, None)
    flush_l2(flush)
    for t in range(T):
        ev[t][0].record(stream)
        gd.gd_step(env.h, actions[t], env.reward, env.done, env.world_done)
        ev[t][1].record(stream)
        gd.gd_observe(env.h, env.obs)
        ev[t][2].record(stream)
    stream.synchronize()
    gd.gd_sync(env.h)
    step = statistics.mean(e[0].elapsed_time(e[1]) for e in ev) * 1e3
    obs = statistics.mean(e[1].elapsed_time(e[2]) for e in ev) * 1e3
    return {"step": step, "observe": obs}


def forward_kernels(env, info, actions, T, stream, flush, ms_episode, road_bytes, peak):
    """Roofline lines of the forward launches of a batched env: the step and
    the observation launch of the split form (CUDA events around each launch
    of one extra episode issued call by call), or the fused launch (episode
    time / T).  Returns (kernels, dominant)."""
    A, F = env.A, env.F
    if info.obs_split:
        us = per_kernel_launch_us(env, actions, T, stream, flush)
        step = kernel_record("k_world (step only)", T, us["step"] * T / 1e3, STEP_AGENT_BYTES * A, peak,
                             "road-edge segments read by the off-road test are not in the algorithmic bytes")
        obs = kernel_record("k_observe_split (radial observation of every agent)", T, us["observe"] * T / 1e3,
                            (4.0 * F + OBS_AGENT_BYTES + road_bytes) * A, peak)
        obs["timing"] = step["timing"] = ("CUDA events around each launch of one extra episode issued call by call "
                                          "(gd_step, then gd_observe)")
        return [step, obs], obs
    fused = kernel_record("k_world (fused step + observation)", T, ms_episode,
                          (4.0 * F + 70.0 + road_bytes) * A, peak)
    fused["timing"] = "episode time of the timed graph replays / steps"
    return [fused], fused


def algorithmic_bytes_per_agent_step(scene, F, radius=50.0, max_worlds=None):
    """Observation write 4F + state/action/flags ~70 B, and the road: 12 B
    (x, y, type/index) for every distinct road point of a world within the
    observation radius of at least one of its agents, per agent.  The road
    set is taken at the initial state, with every agent in the scene, so it
    bounds the set of any later step from above.  max_worlds: count the road
    over the first max_worlds worlds only and scale by their agents (for
    the largest workloads)."""
    import numpy as np
    from scipy.spatial import cKDTree
    pts = 0
    nw = scene.num_worlds if max_worlds is None else min(scene.num_worlds, max_worlds)
    for w in range(nw):
        a0, a1 = scene.agent_off[w], scene.agent_off[w + 1]
        r0, r1 = scene.road_off[w], scene.road_off[w + 1]
        if a1 == a0 or r1 == r0:
            continue
        tree = cKDTree(np.stack([scene.road_x[r0:r1], scene.road_y[r0:r1]], 1).astype(np.float64))
        near = tree.query_ball_point(np.stack([scene.x[a0:a1], scene.y[a0:a1]], 1).astype(np.float64), radius)
        pts += len(set().union(*near))
    road = 12.0 * pts / max(int(scene.agent_off[nw]), 1)
    return 4.0 * F + 70.0, road


def cpu_baseline(workload, seed, budget_s=12.0, scene=None, dynamics=0, actions=None):
    """The oracle as it stands, on a bounded sample of the same workload: the
    first 64 worlds, stepped (step + observe, episodes repeating the same
    action sequence) until budget_s of wall-clock has passed.  scene: the
    workload's scene when the caller has it already."""
    import numpy as np
    from oracle import Oracle, OracleConfig
    from oracle.oracle import num_threads
    from paper_2408_01584_b300 import scenes
    wl = scenes.WORKLOADS[workload]
    sc = (scene if scene is not None else scenes.workload_scene(workload, seed)).subset(0, min(64, wl["worlds"]))
    cfg = OracleConfig(k_road=wl["k_road"], n_partners=wl["n_partners"], episode_len=wl["steps"],
                       term_collision=wl["term_collision"], term_offroad=wl["term_offroad"],
                       auto_reset=wl["auto_reset"], nontrivial_init=bool(wl.get("nontrivial_init", False)),
                       dynamics=dynamics)
    o = Oracle(sc, cfg)
    acts = scenes.make_actions(wl["steps"], sc.num_agents, seed) if actions is None else actions[:, :sc.num_agents]
    t0 = time.perf_counter()
    steps = 0
    while (time.perf_counter() - t0) < budget_s:
        o.step(acts[steps % wl["steps"]])
        o.observe()
        steps += 1
    dt = time.perf_counter() - t0
    return {"value": steps * sc.num_agents / dt, "unit": METRIC, "cores": num_threads(), "kind": "oracle",
            "sample": f"first {sc.num_worlds} worlds ({sc.num_agents} agents) of {workload}, {steps} steps of "
                      f"step+observe, float64 brute force, OpenMP over worlds, {dt:.1f} s"}


def cpu_baseline_fwdbwd(workload, scene, worlds, steps, seed=0):
    """The oracle's forward + backward as it stands (oracle/gradient.py: the
    float64 C++ oracle rollout, then float64 autograd along its decisions)
    on the first `worlds` worlds of the workload for `steps` steps."""
    import numpy as np
    from oracle import OracleConfig
    from oracle.gradient import objective_gradient
    from oracle.oracle import num_threads
    from paper_2408_01584_b300 import scenes
    wl = scenes.WORKLOADS[workload]
    sc = scene.subset(0, worlds)
    cfg = OracleConfig(k_road=wl["k_road"], n_partners=wl["n_partners"], episode_len=wl["steps"],
                       term_collision=wl["term_collision"], term_offroad=wl["term_offroad"],
                       auto_reset=wl["auto_reset"])
    acts = scenes.make_actions(steps, sc.num_agents, seed)
    w = np.random.default_rng(seed).uniform(0, 1, cfg.feat)
    t0 = time.perf_counter()
    objective_gradient(sc, cfg, acts, w, 1.0)
    dt = time.perf_counter() - t0
    return {"value": steps * sc.num_agents / dt, "unit": METRIC + " (forward+backward)", "cores": num_threads(),
            "kind": "oracle", "sample": f"first {worlds} worlds ({sc.num_agents} agents) of {workload}, {steps} steps: "
                                        f"float64 brute-force rollout + float64 autograd gradient, {dt:.1f} s"}


def whole_job_rate(units_per_rank, local_ms, world, device):
    """Max time over ranks (ms) and whole-job throughput: the units every
    rank processed divided by that time (weak scaling, no data exchange)."""
    t = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        x = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return t, units_per_rank * world / (t / 1e3)


def flush_l2(flush, k=0):
    """Flush L2 (126 MB) on the current stream: write the first half of
    `flush` (256 MB), then read the second half, so that the write's dirty
    lines go back to HBM here and not inside the timed kernel that follows,
    and L2 holds clean lines of neither its inputs nor its outputs."""
    half = flush.numel() // 2
    flush[:half].fill_(float(k))
    flush[half:].sum()


def _time_rollouts(run, n, stream, flush):
    """Time n calls of run() with CUDA events on `stream`; L2 flushed (see
    flush_l2) before each, outside the timed interval.  Returns ms per call."""
    import torch
    ms = []
    for k in range(n):
        flush_l2(flush, k)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        run()
        s1.record(stream)
        s1.synchronize()
        ms.append(s0.elapsed_time(s1))
    return ms


def active_agent_steps(done, agent_off):
    """Agent-steps of agents still in the scene at the start of each step
    (the controlled-agent analogue of Sec. 4.1): after gd_reset every agent
    is in; an agent done after step t-1 is out at step t unless its whole
    world was done (the world then restarts from its snapshot)."""
    import numpy as np
    T, A = done.shape
    world = np.repeat(np.arange(len(agent_off) - 1), np.diff(agent_off))
    total = A
    for t in range(1, T):
        d = done[t - 1].astype(bool)
        n_out = np.bincount(world, weights=d, minlength=len(agent_off) - 1)
        all_done = (n_out == np.diff(agent_off)) & (np.diff(agent_off) > 0)
        total += int((~d | all_done[world]).sum())
    return total


def controlled_agent_steps(done, static, agent_off):
    """Agent-steps of controlled agents still in the scene at the start of
    each step (the controlled-agent count of Sec. 4.1): uncontrolled agents
    (static) never count; a controlled agent done after step t-1 is out at
    step t unless its world's episode ended (every controlled agent done),
    when the world restarts from its snapshot."""
    import numpy as np
    T, A = done.shape
    W = len(agent_off) - 1
    world = np.repeat(np.arange(W), np.diff(agent_off))
    ctrl = ~static
    n_ctrl = np.bincount(world, weights=ctrl, minlength=W)
    total = int(ctrl.sum())
    for t in range(1, T):
        d = done[t - 1].astype(bool) & ctrl
        n_out = np.bincount(world, weights=d, minlength=W)
        ended = (n_out == n_ctrl) & (n_ctrl > 0)
        total += int((ctrl & (~d | ended[world])).sum())
    return total


def bench_batched_forward(workload, steps, warmup, dev, stream, flush, seed=0, road_worlds=256, cpu_s=8.0):
    """Batched rollouts (persistent kernels, CUDA graph) of another
    workload, with each forward kernel's roofline line and the oracle on
    its first 64 worlds."""
    import torch
    from paper_2408_01584_b300 import gd, scenes
    wl = scenes.WORKLOADS[workload]
    T = wl["steps"]
    sc = scenes.workload_scene(workload, seed)
    cfg = workload_cfg(workload)
    hbm, peak_kind = _peaks()
    with torch.cuda.stream(stream):
        env = gd.Env(sc, stream=stream, **dict(cfg, flags=cfg["flags"] | gd.GD_BATCHED))
        gd.gd_autotune(env.h)
        info = gd.gd_get_info(env.h)
        A = env.A
        static = (env.get_state()[1].cpu().numpy() & gd.GD_FLAG_STATIC) != 0
        actions = torch.from_numpy(scenes.make_actions(T, A, seed)).to(dev)
        rew = torch.empty(T, A, device=dev)
        done = torch.empty(T, A, dtype=torch.uint8, device=dev)

        def run():
            gd.gd_reset(env.h, None)
            gd.gd_rollout(env.h, T, actions, env.obs, False, rew, done)

        for _ in range(warmup):
            run()
        ms = _time_rollouts(run, steps, stream, flush)
        gd.gd_sync(env.h)
        done_h = done.cpu().numpy()
        _, road = algorithmic_bytes_per_agent_step(sc, env.F, float(env.cfg.obs_radius), road_worlds)
        kernels, dom = forward_kernels(env, info, actions, T, stream, flush, statistics.mean(ms), road, hbm)
        gd.gd_sync(env.h)
    act = active_agent_steps(done_h, sc.agent_off)
    ctl = controlled_agent_steps(done_h, static, sc.agent_off)
    out = {"workload": workload, "worlds": sc.num_worlds, "agents": A, "road_points": sc.num_road,
           "value": T * A * steps / (sum(ms) / 1e3), "unit": METRIC, "ms_per_episode": statistics.mean(ms),
           "active_agent_steps_per_s": act * steps / (sum(ms) / 1e3),
           "controlled_agent_steps_per_s": ctl * steps / (sum(ms) / 1e3),
           "uncontrolled_agents": int(static.sum()),
           "autotuned": {"block_size": info.block_size, "road_cell_m": round(float(info.road_cell), 3),
                         "topk_strategy": info.topk_strategy, "road_tile": info.road_tile, "obs_split": info.obs_split},
           "roofline": dict(dom, peak=hbm, peak_kind=peak_kind, unit="GB/s",
                            road_bytes_per_agent=road,
                            road_bytes_sample=f"road points within R of the agents of the first "
                                              f"{min(road_worlds, sc.num_worlds)} worlds"),
           "kernels": kernels}
    env.close()
    out["cpu_baseline"] = cpu_baseline(workload, seed, budget_s=cpu_s, scene=sc)
    return out


def bench_fwdbwd(workload, steps, warmup, dev, stream, flush, seed=0, road_worlds=256, cpu_worlds=8, cpu_steps=91,
                 shape=None):
    """Differentiable rollouts: objective forward (checkpoints every 10
    steps) + adjoint backward over the whole episode, each a captured CUDA
    graph (batched form), against the same kernels issued from the host
    (plain form); each kernel's roofline line from a launch-by-launch pass
    under CUDA events; the oracle's forward + backward on a sample.
    `shape`: gd_config fields that replace the autotuner (profiling runs,
    where the tuner's trials are timed under the profiler)."""
    import numpy as np
    import torch
    from paper_2408_01584_b300 import gd, scenes
    wl = scenes.WORKLOADS[workload]
    T = wl["steps"]
    sc = scenes.workload_scene(workload, seed)
    cfg = workload_cfg(workload)
    hbm, peak_kind = _peaks()
    res = {}
    with torch.cuda.stream(stream):
        for form in ("batched", "plain"):
            fl = cfg["flags"] | gd.GD_DIFFERENTIABLE | (gd.GD_BATCHED if form == "batched" else 0)
            env = gd.Env(sc, stream=stream, **dict(cfg, flags=fl), **(shape or {}))
            if not shape:
                gd.gd_autotune(env.h)
            info = gd.gd_get_info(env.h)
            A, F = env.A, env.F
            actions = torch.from_numpy(scenes.make_actions(T, A, seed)).to(dev)
            w = torch.from_numpy(np.random.default_rng(seed).uniform(0, 1, F).astype(np.float32)).to(dev)
            ell = torch.empty(T, A, device=dev)
            d_act = torch.empty(T, A, 2, device=dev)
            d_s0 = torch.empty(A, 4, device=dev)

            def fwd():
                gd.gd_reset(env.h, None)
                gd.gd_rollout_objective(env.h, T, actions, w, 1.0, ell, env.obs)

            def fwdbwd():
                fwd()
                gd.gd_rollout_backward(env.h, w, 1.0, None, d_act, d_s0)

            for _ in range(warmup):
                fwdbwd()
            ms_f = _time_rollouts(fwd, steps, stream, flush)
            ms = _time_rollouts(fwdbwd, steps, stream, flush)
            gd.gd_sync(env.h)
            res[form] = {"value": T * A * steps / (sum(ms) / 1e3), "unit": METRIC + " (forward+backward)",
                         "ms_per_episode": statistics.mean(ms), "forward_only_ms_per_episode": statistics.mean(ms_f),
                         "autotuned": {"block_size": info.block_size, "road_cell_m": round(float(info.road_cell), 3),
                                       "topk_strategy": info.topk_strategy, "road_tile": info.road_tile,
                                       "obs_split": info.obs_split, "adjoint_split": info.adjoint_split,
                                       "adjoint_road_tile": info.adjoint_road_tile}}
            if form == "batched":
                # launch by launch under events: one objective rollout, one backward pass
                flush_l2(flush)
                gd.gd_reset(env.h, None)
                ms_o, n_o = gd.gd_time_objective(env.h, T, actions, w, 1.0, ell, env.obs)
                flush_l2(flush)
                ms_b, n_b = gd.gd_time_backward(env.h, w, 1.0, None, d_act, d_s0)
                # a split adjoint launch covers a whole segment: bytes per
                # launch are the agent-step bytes of all T steps over the launches
                seg = lambda per_agent_step, n: per_agent_step * A * T / max(n, 1)
                _, road = algorithmic_bytes_per_agent_step(sc, F, float(env.cfg.obs_radius), road_worlds)
                n_w = float((np.diff(sc.agent_off) ** 2).sum()) / A          # agents of an agent's world, averaged
                kern = []
                if n_o[0]:
                    kern.append(kernel_record("k_copy_snapshot (checkpoint)", n_o[0], ms_o[0], SNAPSHOT_AGENT_BYTES * A,
                                              hbm))
                if info.obs_split:
                    kern.append(kernel_record("k_world (step only, writes r_s)", n_o[1], ms_o[1],
                                              (STEP_AGENT_BYTES + 4) * A, hbm))
                    kern.append(kernel_record("k_observe_split<LOSS> (observation + objective term)", n_o[2], ms_o[2],
                                              (4.0 * F + OBS_AGENT_BYTES + 12 + road) * A, hbm,
                                              "row 4F, own state 33 B, ell read+write 8 B, K-th distance 4 B, road; "
                                              "the selection record (2K B per agent in the scene) is not counted"))
                else:
                    kern.append(kernel_record("k_world (fused step + observation + objective)", n_o[2], ms_o[2],
                                              (4.0 * F + 70.0 + 8 + road) * A, hbm))
                kern.append(kernel_record("k_copy_snapshot (segment start)", n_b[0], ms_b[0], SNAPSHOT_AGENT_BYTES * A,
                                          hbm))
                if info.adjoint_recompute:
                    kern.append(kernel_record(
                        "k_recompute (a segment's states from the forward's recorded decisions)", n_b[1], ms_b[1],
                        seg(8 + 1 + 16 + 1, n_b[1]) + 17 * A, hbm,
                        "per agent-step: reads the action and the recorded flags, writes state and flags; the "
                        "segment's first state and flags once"))
                else:
                    kern.append(kernel_record("k_world (recomputed step, out of place)", n_b[1], ms_b[1],
                                              STEP_AGENT_BYTES * A, hbm))
                if info.adjoint_split:
                    kern.append(kernel_record(
                        "k_adj_observer (a segment's recorded selections, observer-side gradients, slot rows)",
                        n_b[2], ms_b[2], seg(16 + 16 + 1 + 2 * env.K + 16 + 8 + 128 + road * 8 / 12, n_b[2]), hbm,
                        "per agent-step: reads post state, extents, flags, the forward's selection record (2K B) and "
                        "the selected points' coordinates (bounded by 8 B per road point within R of the world's "
                        "agents); writes gradient, (cos, sin), 128-byte slot row"))
                    kern.append(kernel_record(
                        "k_adj_dynamics (a segment's partner sides, rewards, dynamics adjoints)", n_b[3], ms_b[3],
                        seg(16 + 16 + 16 + 1 + 1 + 8 + 8 + n_w + 8, n_b[3]) + 2 * 16 * A, hbm,
                        "per agent-step: reads gradient, post and pre state, flags, action, (cos, sin), its slot "
                        "column; writes the action gradient; the adjoint is read and written once per segment"))
                else:
                    kern.append(kernel_record("k_adjoint (fused)", n_b[2], ms_b[2],
                                              (16 + 16 + 1 + 16 + 1 + 8 + 16 + 4 + 16 + 8 + road) * A, hbm))
                res[form]["kernels"] = kern
                res[form]["road_bytes_per_agent"] = road
                # dominant backward kernel
                bwd = [k for k in kern if k["kernel"].startswith(("k_adj", "k_adjoint"))]
                top = max(bwd, key=lambda k: k["avg_launch_us"] * k["launches"])
                res[form]["roofline"] = dict(top, peak=hbm, peak_kind=peak_kind, unit="GB/s")
            env.close()
            del env
    out = {"workload": workload, "worlds": sc.num_worlds, "agents": A, "road_points": sc.num_road,
           "value": res["batched"]["value"], "unit": METRIC + " (forward+backward)",
           "ms_per_episode": res["batched"]["ms_per_episode"],
           "forward_only_ms_per_episode": res["batched"]["forward_only_ms_per_episode"], "ckpt_every": 10,
           "form": "batched: objective rollout and backward pass each one captured CUDA graph",
           "autotuned": res["batched"]["autotuned"], "roofline": res["batched"]["roofline"],
           "kernels": res["batched"]["kernels"],
           "plain": dict(res["plain"], form="plain: the same kernels issued from the host launch by launch, no graph")}
    if cpu_worlds:
        out["cpu_baseline"] = cpu_baseline_fwdbwd(workload, sc, cpu_worlds, cpu_steps, seed)
    return out


def bench_lidar(workload, n_rays, fov, head, steps, warmup, dev, stream, flush, seed=0, cpu_s=8.0):
    """Batched rollouts with the LiDAR / view-cone observation (Sec. 3.2
    "Sensor modalities") instead of the radius filter: n_rays rays over fov
    radians per agent per step, autotuned, one CUDA graph per episode; head
    rotations (when `head`) drawn per step and agent in [-1, 1] rad.  The
    oracle's scan of the first world's agents gives the CPU rate."""
    import math
    import numpy as np
    import torch
    from oracle import Oracle, OracleConfig
    from oracle.oracle import num_threads
    from paper_2408_01584_b300 import gd, scenes
    wl = scenes.WORKLOADS[workload]
    T = wl["steps"]
    sc = scenes.workload_scene(workload, seed)
    cfg = workload_cfg(workload)
    with torch.cuda.stream(stream):
        env = gd.Env(sc, stream=stream, lidar_rays=n_rays, lidar_fov=fov,
                     **dict(cfg, flags=cfg["flags"] | gd.GD_BATCHED))
        gd.gd_autotune(env.h)
        info = gd.gd_get_info(env.h)
        A = env.A
        actions = torch.from_numpy(scenes.make_actions(T, A, seed)).to(dev)
        hd = torch.from_numpy(np.random.default_rng(seed).uniform(-1, 1, (T, A)).astype(np.float32)).to(dev) \
            if head else None

        def run():
            gd.gd_reset(env.h, None)
            gd.gd_rollout_lidar(env.h, T, actions, hd, env.depth, env.cls, False)

        for _ in range(warmup):
            run()
        ms = _time_rollouts(run, steps, stream, flush)
        gd.gd_sync(env.h)
    hbm, peak_kind = _peaks()
    step_s = statistics.mean(ms) / T / 1e3
    algo = 5.0 * n_rays + 70.0                      # depth float + class byte per ray, state/action/flags
    achieved = algo * A / step_s / 1e9
    # CPU: the oracle's brute-force scan of the first world's agents
    orc = Oracle(sc.subset(0, 1), OracleConfig())
    na = int(sc.agent_off[1])
    t0 = time.perf_counter()
    reps = 0
    while time.perf_counter() - t0 < cpu_s or reps == 0:
        orc.lidar(n_rays, fov)
        reps += 1
    cpu_dt = time.perf_counter() - t0
    out = {"workload": workload, "observation": f"LiDAR {n_rays} rays over {math.degrees(fov):.0f} deg"
           + (" with head rotation" if head else ""), "agents": A,
           "value": T * A * steps / (sum(ms) / 1e3), "unit": METRIC, "ms_per_episode": statistics.mean(ms),
           "autotuned": {"lidar_block_size": info.lidar_block_size, "road_tile": info.lidar_road_tile,
                         "split": info.lidar_split, "road_cell_m": round(float(info.road_cell), 3)},
           "roofline": {"kernel": "k_lidar_group (split form) or k_world<LIDAR> (fused), as tuned", "bound": "hbm",
                        "achieved": achieved, "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s",
                        "frac": achieved / hbm, "algorithmic_bytes_per_agent_step": algo,
                        "timing": "episode time of the timed graph replays / steps (both launches of a step)"},
           "cpu_baseline": {"value": reps * na / cpu_dt, "unit": "agent-scans/s", "cores": num_threads(),
                            "kind": "oracle", "sample": f"{na} agents of world 0, {reps} scans, {cpu_dt:.1f} s"}}
    env.close()
    return out


def bench_invertible(workload, steps, warmup, dev, stream, flush, seed=0):
    """The simplified invertible model (Sec. 3.2 "Agent dynamics"): batched
    rollouts of the workload under it, and gd_invert_actions over a 91-step
    trajectory of every agent (expert-action inversion), against HBM: the
    inversion reads each state once (16 B per agent-step plus the lengths)
    and writes 8 B of actions."""
    import numpy as np
    import torch
    from paper_2408_01584_b300 import gd, scenes
    wl = scenes.WORKLOADS[workload]
    T = wl["steps"]
    sc = scenes.workload_scene(workload, seed)
    cfg = workload_cfg(workload)
    with torch.cuda.stream(stream):
        env = gd.Env(sc, stream=stream, dynamics=gd.GD_DYN_INVERTIBLE, **dict(cfg, flags=cfg["flags"] | gd.GD_BATCHED))
        gd.gd_autotune(env.h)
        A = env.A
        acts_h = scenes.make_actions(T, A, seed)
        acts_h[:, :, 1] *= 0.2 / 0.7                     # curvature U[-0.2, 0.2] 1/m
        actions = torch.from_numpy(acts_h).to(dev)

        def run():
            gd.gd_reset(env.h, None)
            gd.gd_rollout(env.h, T, actions, env.obs, False, None, None)

        for _ in range(warmup):
            run()
        ms = _time_rollouts(run, steps, stream, flush)
        hbm, peak_kind = _peaks()
        _, road = algorithmic_bytes_per_agent_step(sc, env.F, float(env.cfg.obs_radius), 256)
        kernels, _ = forward_kernels(env, gd.gd_get_info(env.h), actions, T, stream, flush, statistics.mean(ms), road,
                                     hbm)
        # a trajectory of every agent (no agent leaves: per-stage steps without termination)
        envt = gd.Env(sc, stream=stream, goal_radius=0.0, dynamics=gd.GD_DYN_INVERTIBLE, k_road=0, n_partners=0)
        states = torch.empty(T + 1, A, 4, device=dev)
        states[0] = envt.get_state()[0]
        for t in range(T):
            gd.gd_step(envt.h, actions[t])
            states[t + 1] = envt.get_state()[0]
        rec = torch.empty(T, A, 2, device=dev)

        def inv():
            gd.gd_invert_actions(envt.h, T, states, rec)

        for _ in range(warmup):
            inv()
        # a single launch of ~30 us: the median of 9 (each after an L2 flush)
        ms_inv = _time_rollouts(inv, max(steps, 9), stream, flush)
        gd.gd_sync(env.h)
        gd.gd_sync(envt.h)
    # recovered vs. applied actions where the vehicle moved (curvature is
    # undefined at rest and ill-conditioned near it)
    moving = np.abs(states[:-1, :, 3].cpu().numpy() * float(envt.cfg.dt)) > 0.05
    d = np.abs(rec.cpu().numpy() - acts_h)
    err = [float(d[..., 0].max()), float(d[..., 1][moving].max())]
    inv_s = statistics.median(ms_inv) / 1e3
    algo = (T + 1) * A * 16 + A * 16 + T * A * 8
    inv_rec = kernel_record("k_invert (expert-action inversion, 91 steps of every agent)", 1, statistics.median(ms_inv),
                            algo, hbm)
    kernels.append(inv_rec)
    # the oracle's inversion of the first 4,096 agents' trajectories (float64)
    from oracle import OracleConfig
    from oracle.oracle import invert as oracle_invert, num_threads
    n_cpu = min(A, 4096)
    st_h = states[:, :n_cpu].cpu().numpy().astype(np.float64)
    t0 = time.perf_counter()
    oracle_invert(OracleConfig(dynamics=1), st_h, sc.length[:n_cpu])
    cpu_inv_s = time.perf_counter() - t0
    out = {"workload": workload, "dynamics": "simplified invertible model", "agents": A,
           "roofline": dict(inv_rec, peak=hbm, peak_kind=peak_kind, unit="GB/s"), "kernels": kernels,
           "value": T * A * steps / (sum(ms) / 1e3), "unit": METRIC, "ms_per_episode": statistics.mean(ms),
           "inversion": {"value": T * A / inv_s, "unit": "agent-steps/s", "ms": statistics.median(ms_inv),
                         "timing": f"median of {len(ms_inv)} launches, each after an L2 flush",
                         "max_abs_error_accel_curvature": err,
                         "note": "curvature error over steps that moved more than 5 cm",
                         "hbm": {"achieved": algo / inv_s / 1e9, "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s",
                                 "frac": algo / inv_s / 1e9 / hbm, "algorithmic_bytes": algo},
                         "cpu_baseline": {"value": T * n_cpu / cpu_inv_s, "unit": "agent-steps/s",
                                          "cores": num_threads(), "kind": "oracle",
                                          "sample": f"{n_cpu} agents x {T} steps, float64, {cpu_inv_s:.2f} s"}}}
    env.close()
    envt.close()
    out["cpu_baseline"] = cpu_baseline(workload, seed, budget_s=6.0, scene=sc, dynamics=1, actions=acts_h)
    return out


def bench_decimation(workload, steps, warmup, dev, stream, flush, seed=0):
    """Scene-load decimation (Sec. 3.1): gd_decimate over every polyline of
    the 0.1 m-sampled workload, and batched rollouts on the raw and on the
    decimated roads (the paper's claim: 10-15x fewer points, faster steps)."""
    import numpy as np
    import torch
    from paper_2408_01584_b300 import gd, scenes
    wl = scenes.WORKLOADS[workload]
    T = wl["steps"]
    sc = scenes.workload_scene(workload, seed)
    cfg = workload_cfg(workload)
    off = gd.polylines(sc)
    with torch.cuda.stream(stream):
        t_off = torch.from_numpy(off).to(dev)
        tx = torch.from_numpy(sc.road_x).to(dev)
        ty = torch.from_numpy(sc.road_y).to(dev)
        keep = torch.empty(sc.num_road, dtype=torch.uint8, device=dev)

        def dec():
            gd.gd_decimate(t_off, tx, ty, gd.DECIMATE_AREA, keep, stream.cuda_stream)

        for _ in range(warmup):
            dec()
        ms_dec = _time_rollouts(dec, max(steps, 3), stream, flush)
        dsc, k = gd.decimate_scene(sc, stream=stream.cuda_stream)
        rates = {}
        for name, scene in (("raw", sc), ("decimated", dsc)):
            env = gd.Env(scene, stream=stream, **dict(cfg, flags=cfg["flags"] | gd.GD_BATCHED))
            gd.gd_autotune(env.h)
            actions = torch.from_numpy(scenes.make_actions(T, env.A, seed)).to(dev)

            def run():
                gd.gd_reset(env.h, None)
                gd.gd_rollout(env.h, T, actions, env.obs, False, None, None)

            for _ in range(warmup):
                run()
            ms = _time_rollouts(run, steps, stream, flush)
            gd.gd_sync(env.h)
            rates[name] = {"value": T * env.A * steps / (sum(ms) / 1e3), "unit": METRIC,
                           "ms_per_episode": statistics.mean(ms), "road_points": scene.num_road,
                           "device_bytes": int(gd.gd_get_info(env.h).device_bytes)}
            env.close()
    hbm, peak_kind = _peaks()
    # the oracle's decimation of the first 32 worlds' polylines (float32, OpenMP over polylines)
    from oracle.oracle import decimate as oracle_decimate, num_threads
    n_poly_cpu = int(np.searchsorted(off, sc.road_off[min(32, sc.num_worlds)]))
    t0 = time.perf_counter()
    oracle_decimate(off[:n_poly_cpu + 1], sc.road_x[:off[n_poly_cpu]], sc.road_y[:off[n_poly_cpu]], gd.DECIMATE_AREA)
    cpu_dec_s = time.perf_counter() - t0
    # k_vw reads each point's x, y once and writes its keep byte, plus the offsets
    vw = kernel_record("k_vw_warp (Visvalingam-Whyatt, a warp per polyline)", len(ms_dec), sum(ms_dec),
                       9.0 * sc.num_road + 4.0 * len(off), hbm,
                       "bound by instruction issue over each polyline's sequential eliminations, not by HBM")
    return {"workload": workload, "decimation": {"points_in": sc.num_road, "points_kept": int(k.sum()),
                                                 "reduction": sc.num_road / max(int(k.sum()), 1),
                                                 "polylines": len(off) - 1, "area_tol_m2": gd.DECIMATE_AREA,
                                                 "ms": statistics.mean(ms_dec),
                                                 "points_per_s": sc.num_road / (statistics.mean(ms_dec) / 1e3),
                                                 "roofline": dict(vw, peak=hbm, peak_kind=peak_kind, unit="GB/s")},
            "value": rates["decimated"]["value"], "unit": METRIC, "rollout": rates,
            "roofline": dict(vw, peak=hbm, peak_kind=peak_kind, unit="GB/s"),
            "cpu_baseline": {"value": int(off[n_poly_cpu]) / cpu_dec_s, "unit": "points/s (decimation)", "cores": num_threads(),
                             "kind": "oracle", "sample": f"{n_poly_cpu} polylines ({int(off[n_poly_cpu])} points) of the "
                                                         f"first 32 worlds, {cpu_dec_s:.2f} s"}}


def run_profile(args):
    """Batched rollouts only (no tuner, no other legs), so that a profiler
    sees warm-up + timed k_world launches and nothing else.  --shape
    B,C,T: CTA size B, road cell C m, road tile T (0/1) instead of the
    library's default shape; --lidar N: the LiDAR rollout (N rays over --fov
    degrees, split form: k_world step + k_lidar_group scan per simulator step)
    instead of the radial one; --worlds W: the first W worlds of the
    workload only."""
    import math
    import torch
    from paper_2408_01584_b300 import gd, scenes
    from paper_2408_01584_b300.build import build
    build()
    dev = torch.device("cuda", 0)
    if args.fwdbwd:
        stream = torch.cuda.Stream(dev)
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # see flush_l2
        shape = None
        if args.shape:
            b, c, t = args.shape.split(",")
            shape = dict(block_size=int(b), road_cell=float(c), road_no_tile=0 if int(t) else 1, obs_split=1,
                         adjoint_split=1)
        return dict(bench_fwdbwd(args.workload, args.steps, args.warmup, dev, stream, flush, shape=shape,
                                 cpu_worlds=0 if shape else 8), profile=args.workload)
    wl = scenes.WORKLOADS[args.workload]
    T = wl["steps"]
    sc = scenes.workload_scene(args.workload, 0)
    if args.worlds:
        sc = sc.subset(0, args.worlds)
    cfg = workload_cfg(args.workload)
    stream = torch.cuda.Stream(dev)
    lidar = dict(lidar_rays=args.lidar, lidar_fov=math.radians(args.fov), lidar_split=1) if args.lidar else {}
    shape = {}
    if args.shape:
        b, c, t = args.shape.split(",")
        shape = dict(block_size=int(b), road_cell=float(c), road_no_tile=0 if int(t) else 1)
    with torch.cuda.stream(stream):
        env = gd.Env(sc, stream=stream, **dict(cfg, flags=cfg["flags"] | gd.GD_BATCHED), **lidar, **shape)
        actions = torch.from_numpy(scenes.make_actions(T, env.A, 0)).to(dev)
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # see flush_l2

        def run():
            gd.gd_reset(env.h, None)
            if args.lidar:
                gd.gd_rollout_lidar(env.h, T, actions, None, env.depth, env.cls, False)
            else:
                gd.gd_rollout(env.h, T, actions, env.obs, False, None, None)

        for _ in range(args.warmup):
            run()
        ms = _time_rollouts(run, args.steps, stream, flush)
        gd.gd_sync(env.h)
    return {"profile": args.workload, "shape": args.shape or "default", "worlds": sc.num_worlds, "lidar_rays": args.lidar,
            "ms_per_episode": statistics.mean(ms), "launches_per_episode": T * (2 if args.lidar else 1)}


def run_ours(args, rank, world):
    import numpy as np
    import torch
    from paper_2408_01584_b300 import gd, scenes
    from paper_2408_01584_b300.build import build

    build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wl = scenes.WORKLOADS[args.workload]
    T = wl["steps"]
    sc = scenes.workload_scene(args.workload, seed=rank)
    stream = torch.cuda.Stream(dev)
    cfg = workload_cfg(args.workload)
    with torch.cuda.stream(stream):
        env_b = gd.Env(sc, stream=stream, **dict(cfg, flags=cfg["flags"] | gd.GD_BATCHED))
        env_p = gd.Env(sc, stream=stream, **cfg)
        A, F = env_b.A, env_b.F
        actions_h = torch.from_numpy(scenes.make_actions(T, A, seed=rank)).pin_memory()
        actions = actions_h.to(dev, non_blocking=True)
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # see flush_l2
        reward_d = torch.empty(T, A, dtype=torch.float32, device=dev)
        done_d = torch.empty(T, A, dtype=torch.uint8, device=dev)
    n_plain_launch = 6 + (1 if cfg["flags"] & gd.GD_AUTO_RESET else 0) + 1

    def batched_rollout():
        # reset + one CUDA graph of T simulator steps (fused: one launch per step; split: two)
        gd.gd_reset(env_b.h, None)
        gd.gd_rollout(env_b.h, T, actions, env_b.obs, False, reward_d, done_d)

    def plain_rollout():
        # per-stage form: one launch per stage, issued from the host every step
        gd.gd_reset(env_p.h, None)
        for t in range(T):
            gd.gd_step(env_p.h, actions[t], env_p.reward, env_p.done, env_p.world_done)
            gd.gd_observe(env_p.h, env_p.obs)

    with torch.cuda.stream(stream):
        gd.gd_autotune(env_b.h)
        info = gd.gd_get_info(env_b.h)
        tuned = {"block_size": info.block_size, "road_cell_m": round(float(info.road_cell), 3),
                 "topk_strategy": {1: "bucket rank", 2: "bitonic sort"}[info.topk_strategy],
                 "road_tile": info.road_tile, "obs_split": info.obs_split}
        for _ in range(args.warmup):
            batched_rollout()
            plain_rollout()
        torch.cuda.synchronize()
        gd.gd_sync(env_b.h)
        gd.gd_sync(env_p.h)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with Clocks(dev) as clk:
            ms = _time_rollouts(batched_rollout, args.steps, stream, flush)
        gd.gd_sync(env_b.h)
        total_ms, _ = whole_job_rate(T * A * args.steps, sum(ms), world, dev)
        plain_ms = _time_rollouts(plain_rollout, max(2, min(args.steps, 5)), stream, flush)
        gd.gd_sync(env_p.h)

        # e2e: the public rollout call on host buffers (gd_rollout_host); the
        # copies of actions in and rewards / done out are in the timed region
        reward_h = torch.empty(T, A, dtype=torch.float32).pin_memory()
        done_h = torch.empty(T, A, dtype=torch.uint8).pin_memory()

        def e2e_rollout():
            # the host-buffer rollout: the copies in and out run inside its
            # graph, overlapped with the steps
            gd.gd_reset(env_b.h, None)
            gd.gd_rollout_host(env_b.h, T, actions_h, env_b.obs, reward_h, done_h)

        # untimed warm-up like the device-resident leg: the first call also
        # captures the call's graph
        for _ in range(max(1, args.warmup)):
            e2e_rollout()
        gd.gd_sync(env_b.h)
        e2e_ms = _time_rollouts(e2e_rollout, max(2, min(args.steps, 5)), stream, flush)
        gd.gd_sync(env_b.h)
        bytes_obs, bytes_road = algorithmic_bytes_per_agent_step(sc, F, float(env_b.cfg.obs_radius))
        hbm, peak_kind = _peaks()
        kernels, dom = forward_kernels(env_b, info, actions, T, stream, flush, statistics.mean(ms), bytes_road, hbm)
        gd.gd_sync(env_b.h)
    agent_steps = T * A * world
    value = agent_steps * args.steps / (total_ms / 1e3)
    launches = (2 if info.obs_split else 1) * args.steps * T
    shape = {"block_size": info.block_size, "road_cell_m": round(float(info.road_cell), 3),
             "road_tile": info.road_tile, "obs_split": info.obs_split}
    out = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload,
                   "form": ("batched, split: per step a persistent step kernel over worlds and a persistent "
                            "observation kernel over agents; 91-step CUDA graph") if info.obs_split else
                           "batched, fused: one persistent kernel per simulator step; 91-step CUDA graph",
                   "autotuned": tuned,
                   "worlds": sc.num_worlds, "agents": A, "road_points": sc.num_road, "k_road": cfg["k_road"],
                   "n_partners": cfg["n_partners"], "episode_steps": T, "feat": F,
                   "step": "one 91-step episode of every world",
                   "l2": "flushed (256 MB write, then 256 MB read) before each timed episode; observation output "
                         f"{A * F * 4 / 1e6:.0f} MB per simulator step > 126 MB L2",
                   "parallelism": f"independent worlds, {world} GPU(s), no collective"},
        "e2e": {"value": agent_steps / world * len(e2e_ms) / (sum(e2e_ms) / 1e3), "unit": METRIC,
                "h2d_bytes_per_step": int(T * A * 8), "d2h_bytes_per_step": int(T * A * 5),
                "note": "gd_rollout_host: actions in from pinned host memory, reward and done out, copies inside the "
                        "timed region; the observations stay on the device (the C ABI's design: a learner on the "
                        "same GPU reads them there)"},
        "gpu_launches": int(launches),
        "roofline": dict(dom, peak=hbm, peak_kind=peak_kind, unit="GB/s",
                         traffic=_measured_traffic(args.workload, "k_observe_split" if info.obs_split else "k_world",
                                                   shape),
                         road_bytes_per_agent=bytes_road),
        "kernels": kernels,
        "active_agent_steps_per_s": active_agent_steps(done_d.cpu().numpy(), sc.agent_off) * args.steps
        / (total_ms / 1e3),
        "plain": {"value": T * A * len(plain_ms) / (sum(plain_ms) / 1e3), "unit": METRIC,
                  "ms_per_step": statistics.mean(plain_ms), "launches_per_sim_step": n_plain_launch,
                  "form": "per-stage launches from the host, no graph"},
        "clocks": clk.summary(),
    }
    env_b.close()
    env_p.close()
    del env_b, env_p
    if args.extras and world == 1:
        torch.cuda.empty_cache()
        import math
        out["workloads"] = [bench_batched_forward("uneven_4096", 3, 1, dev, stream, flush),
                            bench_batched_forward("nontrivial_1024x64", 3, 1, dev, stream, flush),
                            bench_fwdbwd("diff_512x32", 3, 1, dev, stream, flush, cpu_worlds=8),
                            bench_fwdbwd("fwdbwd_8192", 2, 1, dev, stream, flush, cpu_worlds=4),
                            bench_lidar(args.workload, 3000, 2 * math.pi, False, 3, 1, dev, stream, flush),
                            bench_lidar(args.workload, 3000, 2 * math.pi / 3, True, 3, 1, dev, stream, flush),
                            bench_invertible(args.workload, 3, 1, dev, stream, flush),
                            bench_decimation("dense_roads_256x64", 3, 1, dev, stream, flush)]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plain_1024x64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="batched rollouts of the workload only, default tuning (for ncu captures)")
    ap.add_argument("--shape", default="", help="with --profile: k_world shape 'block,cell_m,tile', e.g. 256,12,0")
    ap.add_argument("--lidar", type=int, default=0, help="with --profile: LiDAR rollout with this many rays")
    ap.add_argument("--fov", type=float, default=360.0, help="with --profile --lidar: fan width (degrees)")
    ap.add_argument("--worlds", type=int, default=0, help="with --profile: only the first W worlds")
    ap.add_argument("--fwdbwd", action="store_true",
                    help="with --profile: the workload's forward+backward leg (objective rollout + adjoint), autotuned")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the uneven, differentiable, forward+backward, LiDAR, invertible-model and decimation workloads")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        cb = cpu_baseline(args.workload, 0, budget_s=max(3.0, 20.0 / max(args.steps, 1)))
        out = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": METRIC, "n_gpus": args.gpus,
               "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": dict(workload_description(args.workload), form="the oracle on the host cores (see cpu_baseline)"),
               "cpu_baseline": cb,
               "e2e": {"value": cb["value"], "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return
    if args.profile:
        print(json.dumps(run_profile(args)))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            out["cpu_baseline"] = cpu_baseline(args.workload, 0)
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
