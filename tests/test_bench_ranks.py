"""Host logic of the multi-GPU benchmark on CPU processes (gloo, world size 2).

Each rank runs its own disorder realisation (no exchange of data); the only
collectives are the barrier and the max over ranks of the timings, and the
whole-job value counts the steps of every rank.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) seconds of device time and 10 - r of wall time
        t_dev, t_wall = bench.reduce_max([rank + 1.0, 10.0 - rank], dist, torch.device("cpu"))
        dist.barrier()
        out[rank] = (t_dev, t_wall, bench.rank_seed(rank), bench.job_value(world, 5, t_dev))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    res = [out[r] for r in range(world)]
    for t_dev, t_wall, _, value in res:
        assert t_dev == 2.0 and t_wall == 10.0   # the slowest rank sets the job time
        assert value == pytest.approx(2 * 5 / 2.0)
    assert res[0][2] != res[1][2]                # independent realisations


def test_single_rank_reduce_is_identity():
    assert bench.reduce_max([1.5, 2.5], None, torch.device("cpu")) == [1.5, 2.5]
    assert bench.job_value(1, 10, 0.5) == 20.0
