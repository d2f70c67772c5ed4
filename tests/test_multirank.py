"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): each rank
takes its own seeded copy of the workload, the timing is the maximum over
ranks and the whole-job rate counts the units of every rank."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2408_01584_b300 import scenes
    local_ms = 100.0 + 50.0 * rank                  # rank 1 is the slow one
    t, rate = bench.whole_job_rate(1000, local_ms, world, "cpu")
    sc = scenes.workload_scene("plain_4x8", seed=rank)
    out[rank] = (t, rate, float(sc.x[0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_time_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    (t0, r0, x0), (t1, r1, x1) = out[0], out[1]
    assert t0 == t1 == 150.0                         # max over ranks
    assert r0 == r1 == pytest.approx(2 * 1000 / 0.150)
    assert x0 != x1                                  # each rank has its own worlds


def test_single_rank_needs_no_process_group():
    import bench
    t, rate = bench.whole_job_rate(500, 250.0, 1, "cpu")
    assert t == 250.0 and rate == pytest.approx(2000.0)
