"""The multi-GPU form of the step is independent replicas (one gap batch
per rank, no exchange on the data path); bench.py's host logic times the
slowest rank and counts every rank's units.  Checked with world_size 2 on
the CPU (gloo)."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 100.0 + 50.0 * rank  # rank 1 is the slower one
    ms = bench.max_over_ranks(ms_local, dist)
    dist.barrier()
    q.put((rank, ms, bench.job_throughput(1000, 10, ms, world), bench.rank_info()))
    dist.destroy_process_group()


def test_two_replicas_time_the_slowest_rank_and_count_all_units():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, info in out:
        assert ms == 150.0                       # every rank sees the max
        assert value == pytest.approx(2 * 1000 * 10 / 0.150)
        assert info[0] == rank and info[1] == world


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_throughput(10, 4, 2.0, 1) == pytest.approx(20000.0)
