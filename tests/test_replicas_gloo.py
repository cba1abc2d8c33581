"""Multi-GPU is replicas only: each rank transforms its own segments and the
only cross-rank step is the timing reduction (max over ranks).  Checked with
two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = bench.rank_seeds(rank, 4)
        t = bench.reduce_max(1.5 + rank, dist, "cpu")
        out[rank] = (seeds, t)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_disjoint_work_and_max_time():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    s0, t0 = out[0]
    s1, t1 = out[1]
    assert set(s0).isdisjoint(s1) and len(s0) == len(s1) == 4
    assert t0 == t1 == 2.5


def test_single_rank_identity():
    assert bench.reduce_max(3.25, None) == 3.25
    assert bench.rank_seeds(0, 3) == [0, 1, 2]
