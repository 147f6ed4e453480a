"""The benchmark's multi-GPU path runs independent replicas: each rank times
its own simulation, the job's time is the slowest rank's and its throughput
counts every rank's site updates.  This checks that aggregation with two
gloo ranks on the CPU (no GPU involved)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, times, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(times[rank], dist)
        glups = bench.whole_job_glups(2.0e9, world, slowest)
        out[rank] = (slowest, glups)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_timing_is_max_over_ranks_and_value_is_whole_job():
    world = 2
    times = [1.5, 2.0]
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, times, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        slowest, glups = out[r]
        assert slowest == 2.0
        assert abs(glups - world * 2.0e9 / 2.0 / 1e9) < 1e-12


def test_single_process_aggregation_is_local():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, None) == 3.25
    assert bench.whole_job_glups(1e9, 1, 0.5) == 2.0
