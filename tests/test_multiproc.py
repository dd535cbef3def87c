"""The N>1 paths of bench.py on CPU, with gloo ranks.

* Sharded (the default for N>1): one graph's networks, or their slices, split
  over the ranks by longest processing time on their cost; each rank
  contracts its share and one all-reduce of the partial energies completes E.
  Here a rank contracts its share from the arrays the kernels read
  (qt_plan_export_device, emulated on the CPU) or from the exported plan.
* Replicas (--replicas): each rank evaluates its own copy of the workload
  (weak scaling, no data-path collective); the job's time is the slowest
  rank's, taken with an all-reduce MAX, and its rate counts every rank's units.
"""
import os
import socket
import sys
from pathlib import Path

import numpy as np
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
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for r in range(world):
        mine, job, rate, nets = res[r]
        assert job == pytest.approx(0.020)  # the slower rank's time, seen by both
        assert rate == pytest.approx(world * 5 / 0.020)
    assert res[0][3] == 45 and res[1][3] == 60  # each rank planned its own graph


def _shard_rank(rank, world, port, out):
    """One rank of a sharded energy: plan this rank's networks (LPT by cost),
    contract them with the test-side numpy evaluator, reduce the partial
    energies with one all-reduce."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, str(ROOT))
    sys.path.insert(0, str(ROOT / "tests"))
    from plan_eval import evaluate
    from paper_2204_06045_gb300 import qtgb, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, p = 14, 2
        edges = synth.random_regular_graph(n, 22)
        g, b = synth.angles(p, 22)
        with qtgb.plan_shard(n, edges, p, world, rank, host_only=True) as pl:
            mine = pl.shard_edges
            cost = float(pl.stats()["sum_2w"])
            if mine.size:
                B, O = pl.export()
                zz = evaluate(B, O, g, b, fixed=pl.export_fixed()).real
            else:
                zz = np.zeros(0)
        part = torch.tensor([0.5 * float(np.sum(1.0 - zz))], dtype=torch.float64)
        dist.all_reduce(part, op=dist.ReduceOp.SUM)
        out[rank] = (mine.tolist(), zz.tolist(), float(part.item()), cost)
    finally:
        dist.destroy_process_group()


def test_sharded_energy_over_gloo_ranks_matches_oracle():
    """One graph's networks split over ranks by LPT on their cost; the
    ranks' partial energies sum to the oracle's energy, every edge is held by
    exactly one rank, and the loads are balanced."""
    import oracle
    from paper_2204_06045_gb300 import build, synth
    build.build()
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_shard_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    n, p = 14, 2
    edges = synth.random_regular_graph(n, 22)
    g, b = synth.angles(p, 22)
    held = sorted(e for r in range(world) for e in res[r][0])
    assert held == list(range(edges.shape[0]))
    E = res[0][2]
    assert res[1][2] == pytest.approx(E, abs=1e-14)
    assert E == pytest.approx(oracle.sv_energy(n, edges, g, b), abs=1e-10)
    zz = oracle.sv_zz(n, edges, g, b)
    for r in range(world):
        np.testing.assert_allclose(res[r][1], zz[res[r][0]], atol=1e-12)
    costs = [res[r][3] for r in range(world)]
    assert max(costs) <= 1.5 * min(costs)


def _slice_shard_rank(rank, world, port, out):
    """One rank's units (network slices) of a sliced graph, contracted with the
    test-side evaluator; per-edge partial values summed over ranks."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, str(ROOT))
    sys.path.insert(0, str(ROOT / "tests"))
    from plan_eval import evaluate
    from paper_2204_06045_gb300 import qtgb, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, p = 14, 3
        edges = synth.random_regular_graph(n, 22)
        g, b = synth.angles(p, 22)
        dense = torch.zeros(edges.shape[0], dtype=torch.float64)
        units = []
        with qtgb.plan_shard(n, edges, p, world, rank, host_only=True, slice_width=7) as pl:
            mine = pl.shard_edges
            cost = float(pl.stats()["sum_2w"])
            if mine.size:
                B, O = pl.export()
                zz = evaluate(B, O, g, b, fixed=pl.export_fixed()).real
                dense[torch.as_tensor(mine, dtype=torch.long)] = torch.as_tensor(zz)
                units = sorted({(int(mine[net]), int(s)) for net, s in zip(B["network"], B["slice"])})
        dist.all_reduce(dense, op=dist.ReduceOp.SUM)
        out[rank] = (units, dense.tolist(), cost)
    finally:
        dist.destroy_process_group()


def test_sliced_networks_sharded_over_gloo_ranks_match_oracle():
    """Balance with slicing: the units are network slices, so one wide
    network's slices may sit on several ranks; each rank's value for an edge
    is the sum over its slices, and the sum over ranks is the oracle's e_jk.
    Every slice of every network is held by exactly one rank."""
    import oracle
    from paper_2204_06045_gb300 import build, qtgb, synth
    build.build()
    world = 3
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_slice_shard_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    n, p = 14, 3
    edges = synth.random_regular_graph(n, 22)
    g, b = synth.angles(p, 22)
    with qtgb.plan(n, edges, p, host_only=True, slice_width=7) as full:
        B, _ = full.export()
    want = sorted({(int(e), int(s)) for e, s in zip(B["network"], B["slice"])})
    held = sorted(u for r in range(world) for u in res[r][0])
    assert held == want  # a partition of all (edge, slice) units
    split = {e for e, _ in want if len({r for r in range(world) for (e2, _) in res[r][0] if e2 == e}) > 1}
    assert split, "some network's slices sit on more than one rank"
    zz = oracle.sv_zz(n, edges, g, b)
    for r in range(world):
        np.testing.assert_allclose(res[r][1], zz, atol=1e-12)
    costs = [res[r][2] for r in range(world)]
    assert max(costs) <= 1.5 * min(costs)


def _dedup_shard_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, str(ROOT))
    sys.path.insert(0, str(ROOT / "tests"))
    from plan_eval import evaluate
    from paper_2204_06045_gb300 import qtgb, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, p = 80, 2
        edges = synth.random_regular_graph(n, 31)
        g, b = synth.angles(p, 31)
        dense = torch.zeros(edges.shape[0], dtype=torch.float64)
        with qtgb.plan_shard(n, edges, p, world, rank, host_only=True, dedup=True) as pl:
            mine = pl.shard_edges
            st = pl.stats()
            if mine.size:
                B, O = pl.export()
                vals = evaluate(B, O, g, b, fixed=pl.export_fixed()).real
                R = pl.export_reps()
                dense[torch.as_tensor(mine, dtype=torch.long)] = torch.as_tensor(
                    np.array([vals[R[i]] for i in range(R.size)]))
        dist.all_reduce(dense, op=dist.ReduceOp.SUM)
        out[rank] = (dense.tolist(), int(st["n_unique"]), int(st["n_networks"]))
    finally:
        dist.destroy_process_group()


def test_deduplicated_shards_over_gloo_ranks_match_oracle():
    """Each rank deduplicates the networks of its own shard (their costs are
    counted undeduplicated when the shards are drawn): the per-edge values
    summed over ranks are the oracle's."""
    import oracle
    from paper_2204_06045_gb300 import build, synth
    build.build()
    world = 3
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_dedup_shard_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    n, p = 80, 2
    edges = synth.random_regular_graph(n, 31)
    g, b = synth.angles(p, 31)
    want = oracle.bucket_zz(n, edges, g, b)[0].real
    for r in range(world):
        np.testing.assert_allclose(res[r][0], want, atol=1e-12)
    assert sum(res[r][1] for r in range(world)) < sum(res[r][2] for r in range(world))


class _CpuPlanStep:
    """Stands in for a device plan in bench.shard_step: the rank's partial energy from the
    device arrays of its host-only shard plan, emulated on the CPU."""

    def __init__(self, pl, p):
        self.pl, self.p = pl, p

    def energy(self, gd, bd, edge_zz=None, energy=None, stream=None):
        from device_eval import emulate
        vals, en = emulate(self.pl, gd.numpy(), bd.numpy(), self.p)
        if edge_zz is not None:
            edge_zz[:] = torch.as_tensor(vals.real)
        energy[0] = float(en[0])


def _device_shard_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, str(ROOT))
    sys.path.insert(0, str(ROOT / "tests"))
    import bench
    from paper_2204_06045_gb300 import qtgb, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, p = 16, 3
        edges = synth.random_regular_graph(n, 40)
        g, b = synth.angles(p, 40)
        with qtgb.plan_shard(n, edges, p, world, rank, host_only=True, slice_width=7) as pl:
            mine = pl.shard_edges
            E = torch.zeros(1, dtype=torch.float64)
            zz = torch.zeros(max(1, mine.size), dtype=torch.float64)
            step = _CpuPlanStep(pl, p)
            gd = torch.tensor(g, dtype=torch.float64)
            bd = torch.tensor(b, dtype=torch.float64)
            bench.shard_step(step, gd, bd, zz if mine.size else None, E, None, dist)
            dense = torch.zeros(edges.shape[0], dtype=torch.float64)
            if mine.size:
                dense[torch.as_tensor(mine, dtype=torch.long)] = zz[:mine.size]
            dist.all_reduce(dense, op=dist.ReduceOp.SUM)
            slow = bench.max_over_ranks(0.001 * (rank + 1), dist, torch)
        out[rank] = (float(E.item()), dense.tolist(), slow, mine.tolist())
    finally:
        dist.destroy_process_group()


def test_bench_shard_step_over_gloo_ranks_matches_oracle():
    """bench.shard_step on two gloo ranks, each rank's share contracted from the
    device arrays of its sliced shard plan: after the step's all-reduce every
    rank holds the oracle's energy, the ranks' per-edge values (sums over their
    slices) add up to the oracle's, and the job's time is the slowest rank's."""
    import oracle
    from paper_2204_06045_gb300 import build, synth
    build.build()
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_device_shard_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    n, p = 16, 3
    edges = synth.random_regular_graph(n, 40)
    g, b = synth.angles(p, 40)
    want_E = oracle.sv_energy(n, edges, g, b)
    for r in range(world):
        assert res[r][0] == pytest.approx(want_E, abs=1e-10)
        np.testing.assert_allclose(res[r][1], oracle.sv_zz(n, edges, g, b), atol=1e-12)
        assert res[r][2] == pytest.approx(0.002)
    assert res[0][3] and res[1][3]  # both ranks hold networks
