"""The benchmark's multi-rank arithmetic on CPU: world-size-2 gloo ranks run independent
replicas (no data-path collective); the job's step time is the slowest rank's and the job's
throughput counts every rank's frames (weak scaling)."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, per_rank_ms, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.world_max_ms(per_rank_ms[rank], dist, torch.device("cpu"))
    out[rank] = (ms, bench.job_rate(255, world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank_and_the_whole_job():
    world = 2
    per_rank = [120.0, 150.0]
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), per_rank, out), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        ms, rate = out[r]
        assert ms == 150.0
        assert rate == pytest.approx(2 * 255 / 0.150)


def test_single_process_needs_no_collective():
    import bench
    assert bench.world_max_ms(42.0, None, None) == 42.0
    assert bench.job_rate(255, 1, 100.0) == pytest.approx(2550.0)
