"""Host-side logic of bench.py's multi-GPU mode, on CPU with gloo ranks: every
rank builds an independent problem (distinct seeds), the step time is the
slowest rank's (max all-reduce), and the reported throughput counts the points
of all ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = bench.max_over_ranks(times[rank], world, "cpu")
        out[rank] = (m, bench.problem_seed(2, rank))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_seeds_gloo():
    world, times = 2, [120.0, 345.5]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, _free_port(), times, out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    assert [res[r][0] for r in range(world)] == [345.5, 345.5]
    assert len({res[r][1] for r in range(world)}) == world
    assert bench.aggregate_value(1 << 20, world, 345.5) == pytest.approx(2 * (1 << 20) / 0.3455)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
