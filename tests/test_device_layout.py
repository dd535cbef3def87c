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
