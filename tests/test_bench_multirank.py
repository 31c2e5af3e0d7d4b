"""bench.py's N > 1 path on CPU: two gloo ranks reduce their timings with
the same helpers the GPU run uses (max over ranks, weak-scaling rate)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 20.0][rank]
    m = bench.reduce_max(ms, "cpu", world)
    v = bench.whole_job_rate(4096 * 2048, 100, world, m * 1e-3)
    out[rank] = (m, v)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reduce_max_and_weak_scaling_rate():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    assert out[0] == out[1]
    m, v = out[0]
    assert m == 20.0
    assert abs(v - 4096 * 2048 * 100 * 2 / 0.020) < 1e-6 * v
