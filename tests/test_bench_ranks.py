"""Multi-rank aggregation of bench.py on CPU: two gloo ranks stand in for two GPUs.

With N replicas ("replicas only": the method has no data-parallel exchange at the benchmark
size), bench.py reports all steps of all ranks over the slowest rank's time.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    dist.barrier()
    value, ms_max = bench.aggregate_throughput(10.0 * (rank + 1), world)   # rank 1 is the slower one
    out[rank] = (value, ms_max)
    dist.destroy_process_group()


def test_two_ranks_report_all_steps_over_the_slowest_time():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        value, ms_max = out[r]
        assert ms_max == 20.0
        assert abs(value - world * 1000.0 / 20.0) < 1e-12


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_throughput(8.0, 1) == (125.0, 8.0)
