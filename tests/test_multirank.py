"""The multi-rank part of bench.py on CPU (gloo, world size 2): ranks run
independent replicas, the job time is the slowest rank's, and the reported
value aggregates every rank's site updates."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank            # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, dist)
    value = bench.aggregate_mlups(world, 1000, 16 * 60, ms_max)
    out[rank] = (ms_max, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction_gloo():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 150.0
    expect = 2 * 1000 * 16 * 60 / 0.150 / 1e6
    assert abs(out[0][1] - expect) < 1e-9 and out[0][1] == out[1][1]


def test_single_rank_reduction_is_identity():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert abs(bench.aggregate_mlups(1, 4194304, 16, 2.0) - 4194304 * 16 / 2e-3 / 1e6) < 1e-6
