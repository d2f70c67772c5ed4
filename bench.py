"""Throughput benchmark: agent-steps/s of the batched driving step on B300.

Agent-steps/s (ASPS) = S * sum_k |A_k| / dT  (Sec. 4.1, Eq. ASPS): S steps of
every world, all agents counted.  One benchmark "step" is one full episode
(T = 91 simulator steps of every world: reset, dynamics, collision,
off-road, reward/done and the observation) over one batch of seeded
synthetic actions.  Inputs are resident in HBM when the timed region starts
(`value`); `e2e` repeats the measurement through gd_rollout with host
buffers and the copies inside the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload plain_1024x64] [--form plain|batched]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "agent-steps/s"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")


def _peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.p = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def workload_cfg(name):
    from paper_2408_01584_b300 import gd, scenes
    wl = scenes.WORKLOADS[name]
    fl = (gd.GD_TERM_COLLISION if wl["term_collision"] else 0) | (gd.GD_TERM_OFFROAD if wl["term_offroad"] else 0) \
        | (gd.GD_AUTO_RESET if wl["auto_reset"] else 0)
    return dict(k_road=wl["k_road"], n_partners=wl["n_partners"], episode_len=wl["steps"], flags=fl)


def algorithmic_bytes_per_agent_step(scene, F):
    """Observation write 4F + state/action/flags ~70 B + the world's road
    tile read once per step (12 B per point: x, y, type/index) / A_w."""
    import numpy as np
    A_w = np.diff(scene.agent_off).astype(np.float64)
    N_w = np.diff(scene.road_off).astype(np.float64)
    road = float((12.0 * N_w).sum() / max(A_w.sum(), 1.0))
    return 4.0 * F + 70.0, road


def cpu_baseline(workload, seed, budget_s=12.0):
    """The oracle as it stands, on a bounded sample of the same workload: the
    first 64 worlds, as many steps (step + observe) as fit in budget_s."""
    import numpy as np
    from oracle import Oracle, OracleConfig
    from oracle.oracle import num_threads
    from paper_2408_01584_b300 import scenes
    wl = scenes.WORKLOADS[workload]
    sc = scenes.workload_scene(workload, seed).subset(0, min(64, wl["worlds"]))
    cfg = OracleConfig(k_road=wl["k_road"], n_partners=wl["n_partners"], episode_len=wl["steps"],
                       term_collision=wl["term_collision"], term_offroad=wl["term_offroad"],
                       auto_reset=wl["auto_reset"])
    o = Oracle(sc, cfg)
    acts = scenes.make_actions(wl["steps"], sc.num_agents, seed)
    t0 = time.perf_counter()
    steps = 0
    while steps < wl["steps"] and (time.perf_counter() - t0) < budget_s:
        o.step(acts[steps])
        o.observe()
        steps += 1
    dt = time.perf_counter() - t0
    return {"value": steps * sc.num_agents / dt, "unit": METRIC, "cores": num_threads(), "kind": "oracle",
            "sample": f"first {sc.num_worlds} worlds ({sc.num_agents} agents) of {workload}, {steps} steps of "
                      f"step+observe, float64 brute force, {dt:.1f} s"}


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
        env = gd.Env(sc, stream=stream, **cfg)
        A, F = env.A, env.F
        actions_h = torch.from_numpy(scenes.make_actions(T, A, seed=rank)).pin_memory()
        actions = actions_h.to(dev, non_blocking=True)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    n_launch_step = 6 + (1 if cfg["flags"] & gd.GD_AUTO_RESET else 0)

    def rollout(events=None):
        # plain form: one launch per stage, driven from the host
        gd.gd_reset(env.h, None)
        for t in range(T):
            gd.gd_step(env.h, actions[t], env.reward, env.done, env.world_done)
            if events is not None:
                events[t][0].record(stream)
            gd.gd_observe(env.h, env.obs)
            if events is not None:
                events[t][1].record(stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            rollout()
        torch.cuda.synchronize()
        gd.gd_sync(env.h)
        if world > 1:
            torch.distributed.barrier()
        ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(T)]
              for _ in range(args.steps)]
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        with Clocks(dev.index) as clk:
            torch.cuda.synchronize()
            for k in range(args.steps):
                flush.fill_(float(k))               # L2 flush between timed rollouts (not timed)
                starts[k].record(stream)
                rollout(ev[k])
                ends[k].record(stream)
            torch.cuda.synchronize()
        gd.gd_sync(env.h)
        ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        obs_ms = [a.elapsed_time(b) for row in ev for (a, b) in row]
        total_ms = sum(ms)
        if world > 1:
            t = torch.tensor([total_ms], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            total_ms = float(t.item())
        # e2e: public rollout call with host buffers, copies inside the timed region
        reward_h = torch.empty(T, A, dtype=torch.float32).pin_memory()
        done_h = torch.empty(T, A, dtype=torch.uint8).pin_memory()
        reward_d = torch.empty(T, A, dtype=torch.float32, device=dev)
        done_d = torch.empty(T, A, dtype=torch.uint8, device=dev)
        e2e_ms = []
        for k in range(max(2, min(args.steps, 5))):
            flush.fill_(float(k))
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            actions.copy_(actions_h, non_blocking=True)
            gd.gd_reset(env.h, None)
            gd.gd_rollout(env.h, T, actions, env.obs, False, reward_d, done_d)
            reward_h.copy_(reward_d, non_blocking=True)
            done_h.copy_(done_d, non_blocking=True)
            s1.record(stream)
            s1.synchronize()
            e2e_ms.append(s0.elapsed_time(s1))
        gd.gd_sync(env.h)
    agent_steps = T * A * world
    value = agent_steps * args.steps / (total_ms / 1e3)
    bytes_obs, bytes_road = algorithmic_bytes_per_agent_step(sc, F)
    obs_avg_s = statistics.mean(obs_ms) / 1e3
    hbm, peak_kind = _peaks()
    achieved = (bytes_obs + bytes_road) * A / obs_avg_s / 1e9
    out = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "form": "plain", "worlds": sc.num_worlds, "agents": A,
                   "road_points": sc.num_road, "k_road": cfg["k_road"], "n_partners": cfg["n_partners"],
                   "episode_steps": T, "feat": F, "l2": "flushed (256 MB write) before each timed episode; "
                   f"observation output {A * F * 4 / 1e6:.0f} MB per step > 126 MB L2",
                   "parallelism": f"independent worlds, {world} GPU(s), no collective"},
        "e2e": {"value": agent_steps * len(e2e_ms) / (sum(e2e_ms) / 1e3) / world * world, "unit": METRIC,
                "h2d_bytes_per_step": int(T * A * 8), "d2h_bytes_per_step": int(T * A * 5)},
        "gpu_launches": int(args.steps * T * (n_launch_step + 1)),
        "roofline": {"bound": "hbm", "kernel": "k_observe", "achieved": achieved, "peak": hbm,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                     "algorithmic_bytes_per_agent_step": bytes_obs + bytes_road,
                     "avg_launch_us": obs_avg_s * 1e6, "launches_timed": len(obs_ms)},
        "clocks": clk.summary(),
    }
    env.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plain_1024x64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
               "config": {"workload": args.workload}, "cpu_baseline": cb,
               "e2e": {"value": cb["value"], "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
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
