"""Multi-rank logic of bench.py on CPU: two gloo ranks, each timing its own
replica.  The job value must use the slowest rank's time and count every
rank's points (weak scaling, no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [120.0, 150.0][rank]
    ms = bench.reduce_max(local_ms, dist, torch.device("cpu"))
    out[rank] = (ms, bench.weak_throughput(world, 240 ** 3, 1000, 10, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    assert out[0][0] == out[1][0] == 150.0
    expect = 2 * 240 ** 3 * 1000 * 10 / 0.150 / 1e9
    assert out[0][1] == pytest.approx(expect)


def test_single_process_is_identity():
    assert bench.reduce_max(3.5, None, None) == 3.5
    assert bench.weak_throughput(1, 100, 10, 2, 1000.0) == pytest.approx(2e-6)
