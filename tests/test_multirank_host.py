"""The N > 1 path of the benchmark (independent replicas, one per rank, timed by
the slowest) on CPU ranks of a world_size-2 gloo group."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_setup()
        local_s = 1.0 + rank                       # rank 1 is the slow replica
        slowest = bench.max_over_ranks(local_s, dist, device="cpu")
        rate = bench.whole_job_rate(1000.0, w, slowest)
        out[rank] = (w, r, local, slowest, rate)
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_and_the_whole_job():
    world = 2
    with mp.get_context("spawn").Manager() as m:   # no fork of a threaded process
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        w, r, local, slowest, rate = res[rank]
        assert (w, r, local) == (world, rank, rank)
        assert slowest == 2.0                      # max over ranks, same on every rank
        assert rate == pytest.approx(1000.0 * world / 2.0)


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
