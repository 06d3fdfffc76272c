"""The benchmark's multi-rank host logic on CPU with the gloo backend, world size 2:
every rank ends with the slowest rank's time, the whole-job value counts the units of
all ranks against it, and the replicas draw independent instances."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [10.0 + 5.0 * rank, 3.0 - rank]  # per-rank step and e2e times (ms)
        got = bench.max_over_ranks(mine, world, "cpu")
        out[rank] = (got, bench.whole_job_value(world, 1000.0, got[0]), bench.replica_seed(rank))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_replicas_gloo():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        got, value, _ = res[r]
        assert got == [15.0, 3.0]  # the maxima over both ranks
        assert value == pytest.approx(2 * 1000.0 / 0.015)
    assert res[0][2] != res[1][2]  # independent instances per replica


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks([1.5, 2.5], 1, "cpu") == [1.5, 2.5]
    assert bench.whole_job_value(1, 100.0, 10.0) == pytest.approx(10000.0)
