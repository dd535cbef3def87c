"""The device layout of plans, checked on the CPU.

tests/device_eval.py contracts every bucket from the arrays the kernels read
(arena offsets, masks over tile outputs, which operands pair over the summed
variable, merged pair sums) and forms the epilogue from its factor lists and
owned networks. Its values must be the oracle's for every kind of plan: plain,
merged, sliced, deduplicated, batched and sharded.
"""
import numpy as np
import pytest

import oracle
from device_eval import emulate
from paper_2204_06045_gb300 import qtgb, synth


def _check(pl, n, edges, g, b, p, atol=1e-12):
    vals, energies = emulate(pl, g, b, p)
    ref = oracle.sv_zz(n, edges, g, b)
    np.testing.assert_allclose(vals.real, ref, rtol=0, atol=atol)
    assert np.abs(vals.imag).max() < atol
    assert energies[0] == pytest.approx(oracle.energy_from_zz(ref), abs=1e-10)


@pytest.mark.parametrize("kw", [dict(slice_width=-1, merge=False), dict(slice_width=-1), dict(slice_width=12),
                                dict(slice_width=8), dict(slice_width=10, merge=False)])
def test_layout_of_one_graph_matches_state_vector(kw):
    """Plain, merged, merged and sliced, and more heavily sliced plans."""
    n, seed, p = 16, 23, 3
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    with qtgb.plan(n, edges, p, host_only=True, dtype="c128", **kw) as pl:
        st = pl.stats()
        if kw.get("merge", True) and kw.get("slice_width", 0) == -1:
            assert (pl.export()[0]["n_sum"] > 1).any()
        if kw.get("slice_width", 0) > 0:
            assert st["slice_bits"] > 0
        _check(pl, n, edges, g, b, p)


def test_layout_of_a_deduplicated_batch_matches_oracle():
    """Two graphs (their own angles), duplicates sharing their representatives'
    factors, representatives sliced."""
    graphs = [(16, synth.random_regular_graph(16, 1)), (18, synth.random_regular_graph(18, 2))]
    p = 2
    G = np.array([synth.angles(p, s)[0] for s in (1, 2)])
    Bt = np.array([synth.angles(p, s)[1] for s in (1, 2)])
    with qtgb.plan_batch(graphs, p, host_only=True, dtype="c128", dedup=True, slice_width=4) as pl:
        st = pl.stats()
        assert st["n_unique"] < st["n_networks"] and st["slice_bits"] > 0
        vals, energies = emulate(pl, G, Bt, p)
    first = 0
    for i, (n, e) in enumerate(graphs):
        ref = oracle.sv_zz(n, e, G[i], Bt[i])
        np.testing.assert_allclose(vals[first:first + e.shape[0]].real, ref, rtol=0, atol=1e-12)
        assert energies[i] == pytest.approx(oracle.energy_from_zz(ref), abs=1e-10)
        first += e.shape[0]


def test_layout_of_slice_shards_adds_up():
    """Slice shards: per-edge partial values and energies (slice 0's holder
    counting the edge's 1/2) sum over ranks to the state vector's."""
    n, seed, p, world = 14, 22, 3, 3
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    zz = np.zeros(edges.shape[0])
    E = 0.0
    for r in range(world):
        with qtgb.plan_shard(n, edges, p, world, r, host_only=True, dtype="c128", slice_width=7) as pl:
            mine = pl.shard_edges
            if mine.size == 0:
                continue
            vals, energies = emulate(pl, g, b, p)
        zz[mine] += vals.real
        E += energies[0]
    ref = oracle.sv_zz(n, edges, g, b)
    np.testing.assert_allclose(zz, ref, rtol=0, atol=1e-12)
    assert E == pytest.approx(oracle.energy_from_zz(ref), abs=1e-10)


@pytest.mark.parametrize("kw", [dict(), dict(slice_width=-1), dict(slice_width=8)])
def test_operands_without_the_summed_variable_are_folded(kw):
    """The kernels read an operand that lacks the bucket's summed variable
    (a merged bucket's consumer gates) only from the gate table: every such
    operand of the device layout is folded, and has rank <= 2."""
    n, seed, p = 18, 5, 4
    edges = synth.random_regular_graph(n, seed)
    with qtgb.plan(n, edges, p, host_only=True, **kw) as pl:
        B, O = pl.export()
        DB, DO, _, _, _ = pl.export_device()
    seen = 0
    for k in range(len(B)):
        for t in range(int(B["op_begin"][k]), int(B["op_begin"][k]) + int(B["n_ops"][k])):
            if not DO["pairs_x"][t]:
                seen += 1
                assert (int(B["folded"][k]) >> (t - int(B["op_begin"][k]))) & 1
                assert O["rank"][t] <= 2 and DO["leaf"][t] == 1
    assert (seen > 0) == bool((B["n_sum"] > 1).any())


def test_symmetric_graphs_deduplicate_to_one_network():
    """K4 and the prism at p=1: every edge's lightcone is the whole graph and
    all are isomorphic (edge-transitive graphs), so one network is contracted."""
    for n, edges in ((4, synth.complete_graph(4)), (6, synth.prism_graph())):
        with qtgb.plan(n, edges, 1, host_only=True, dedup=True) as pl:
            st = pl.stats()
        if n == 4:
            assert st["n_unique"] == 1
        else:  # the prism's triangle edges and its rung edges are two edge orbits
            assert st["n_unique"] == 2


def test_more_ranks_than_units():
    """With more ranks than slices, some ranks hold nothing; the rest hold
    every (edge, slice) unit exactly once."""
    n, seed, p = 10, 3, 1
    edges = synth.random_regular_graph(n, seed)
    world = edges.shape[0] + 5
    held = []
    for r in range(world):
        with qtgb.plan_shard(n, edges, p, world, r, host_only=True, slice_width=3) as pl:
            mine = pl.shard_edges
            if mine.size:
                B, _ = pl.export()
                held += sorted({(int(mine[net]), int(s)) for net, s in zip(B["network"], B["slice"])})
    with qtgb.plan(n, edges, p, host_only=True, slice_width=3) as full:
        B, _ = full.export()
    assert sorted(held) == sorted({(int(e), int(s)) for e, s in zip(B["network"], B["slice"])})


@pytest.mark.parametrize("kw", [dict(), dict(slice_width=6)])
def test_layout_of_energy_passes_adds_up(kw):
    """opts.energy_budget_bytes: each pass's own device arrays, emulated, give
    partial per-edge values and energies (a network's slice 0 in one pass
    counting the edge's 1/2) that sum to the state vector's."""
    n, seed, p = 14, 22, 3
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    with qtgb.plan(n, edges, p, host_only=True, dtype="c128", **kw) as whole:
        budget = whole.stats()["arena_bytes"] // 6
    zz = np.zeros(edges.shape[0])
    E = 0.0
    with qtgb.plan(n, edges, p, host_only=True, dtype="c128", energy_budget_bytes=budget, **kw) as pl:
        passes = pl.passes()
        assert len(passes) == pl.stats()["n_passes"] > 1
        for part, pe in passes:
            vals, energies = emulate(part, g, b, p)
            zz[pe] += vals.real
            E += energies[0]
    ref = oracle.sv_zz(n, edges, g, b)
    np.testing.assert_allclose(zz, ref, rtol=0, atol=1e-12)
    assert E == pytest.approx(oracle.energy_from_zz(ref), abs=1e-10)


@pytest.mark.parametrize("dtype,scratch", [("c64", 1024), ("c128", 512)])
def test_fused_unit_programs_match_plain_contraction(dtype, scratch):
    """The fused units' programs (steps of one bucket, or of up to four
    independent small buckets sharing the warp's lanes), interpreted as the
    kernel runs them -- every member of a step reading before any writes, the
    intermediates in a scratch array of the stage's size -- give the values of
    the bucket-by-bucket contraction, and no step writes scratch that one of
    its members reads."""
    graphs = synth.batch(3, 3, lo=50, hi=200, base_seed=1000)
    spec = [(n, e) for n, e, _, _ in graphs]
    G = np.array([gg for _, _, gg, _ in graphs])
    Bt = np.array([bb for _, _, _, bb in graphs])
    with qtgb.plan_batch(spec, 3, host_only=True, dtype=dtype) as pl:
        assert pl.stats()["n_units"] > 0
        units, recs = pl.export_units()
        steps = (recs["a"] & (1 << 18)) != 0
        assert steps.any(), "no step packs several buckets"
        v_units, e_units = emulate(pl, G, Bt, 3, with_units=True, scratch_elems=scratch)
        v_plain, e_plain = emulate(pl, G, Bt, 3)
    np.testing.assert_allclose(v_units, v_plain, rtol=0, atol=1e-12)
    np.testing.assert_allclose(e_units, e_plain, rtol=1e-12)
