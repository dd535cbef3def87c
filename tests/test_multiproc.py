"""The N>1 path of bench.py on CPU: world_size-2 gloo ranks (replicas).

Each rank evaluates its own copy of the workload (weak scaling, no data-path
collective); the job's time is the slowest rank's, taken with an all-reduce
MAX, and its rate counts every rank's units. Here the ranks time a host-only
plan build of their own seeded graph, so the test needs no GPU.
"""
import os
import socket
import sys
from pathlib import Path

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = Path(__file__).resolve().parents[1]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, str(ROOT))
    import bench
    from paper_2204_06045_gb300 import qtgb, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # a different amount of work per rank: the slowest decides
        n, p = 30 + 10 * rank, 3
        edges = synth.random_regular_graph(n, 1000 + rank)
        with qtgb.plan(n, edges, p, host_only=True) as pl:
            st = pl.stats()
        mine = 0.010 * (rank + 1)  # seconds this rank "took"
        job = bench.max_over_ranks(mine, dist, torch)
        rate = bench.job_throughput(world, 5, job)
        dist.barrier()
        out[rank] = (mine, job, rate, st["n_networks"])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_every_rank():
    from paper_2204_06045_gb300 import build
    build.build()
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for r in range(world):
        mine, job, rate, nets = res[r]
        assert job == pytest.approx(0.020)  # the slower rank's time, seen by both
        assert rate == pytest.approx(world * 5 / 0.020)
    assert res[0][3] == 45 and res[1][3] == 60  # each rank planned its own graph
