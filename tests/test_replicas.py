"""The N > 1 path of bench.py (replicas only: every rank solves its own
Hamiltonian, no data-path collective) on CPU with two gloo ranks: the
per-rank seeds differ, the reported time is the slowest rank's, and the
whole-job throughput counts every rank's solves."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.replica_seed(0, rank))
        local_ms = 100.0 * (rank + 1)            # rank 1 is the slow one
        ms_max = bench.slowest(local_ms, dist)
        out[rank] = (seeds, ms_max, bench.replica_throughput(world, 2, ms_max))
    finally:
        dist.destroy_process_group()


def test_two_replicas_on_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        seeds, ms_max, tput = res[r]
        assert seeds == [0, 1]                   # a different Hamiltonian per rank
        assert ms_max == 200.0                   # the slowest rank's time, on every rank
        assert tput == pytest.approx(2 * 2 / 0.2)


def test_single_process_defaults():
    assert bench.slowest(12.5) == 12.5
    assert bench.replica_seed(7, 0) == 7
    assert bench.replica_throughput(1, 3, 1500.0) == pytest.approx(2.0)
