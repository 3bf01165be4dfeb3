"""The multi-process path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Under torchrun every rank solves its own copy of the instance (replicas, no
collective on the data path); the only communication is the aggregation of
the timing and of the residual gate across ranks.  These tests drive exactly
those helpers with gloo in place of NCCL."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [7.0, 9.5][rank]                       # the slower rank sets the job time
        t = bench.max_over_ranks(ms, world, "cpu")
        ok_all = bench.all_ranks(True, world, "cpu")
        ok_one_fails = bench.all_ranks(rank == 0, world, "cpu")
        out[rank] = (t, ok_all, ok_one_fails, bench.job_rate(world, 1024, t))
    finally:
        dist.destroy_process_group()


def test_timing_and_gate_aggregate_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, ok_all, ok_one_fails, rate = res[rank]
        assert t == 9.5
        assert ok_all is True and ok_one_fails is False
        assert rate == pytest.approx(2 * 1024 / 9.5e-3)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.25, 1, "cpu") == 3.25
    assert bench.all_ranks(False, 1, "cpu") is False
    assert bench.job_rate(1, 1024, 6.4) == pytest.approx(1024 / 6.4e-3)
