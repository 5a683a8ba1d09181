"""Multi-process (world size 2, gloo, CPU) test of bench.py's replica logic:
each rank times its own replica; the job's time is the max over ranks and
the value counts the steps of every rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [1500.0, 2500.0][rank]
    ms = bench.reduce_max(local_ms, dist)
    out[rank] = (ms, bench.job_value(world, 4, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    world = 2
    port = _free_port()
    # the manager process is spawned too: forking a process that already
    # runs threads (OpenMP, torch) can deadlock the child
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, value = out[r]
        assert ms == 2500.0
        assert abs(value - 2 * 4 / 2.5) < 1e-12


def test_single_process_is_identity():
    import bench
    assert bench.reduce_max(3.0, None) == 3.0
    assert abs(bench.job_value(1, 3, 1500.0) - 2.0) < 1e-15
