"""GPU parity of lightcone deduplication (opts.dedup).

Within one graph, networks whose lightcones are isomorphic are contracted
once; the others take that network's value (the epilogue reads the
representative's results). These tests run deduplicated plans against the
state vector, the full plans and the oracle's bucket elimination, with the
tolerances of the other GPU parity tests (1e-10 complex128, 1e-5 complex64
per edge, as in test_gpu_energy).
"""
import numpy as np
import pytest

import oracle
from paper_2204_06045_gb300 import qtgb, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 1e-5}


def scaled_err(x, ref):
    x, ref = np.asarray(x, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    d = np.abs(x - ref)
    return float(max(np.max(d / np.abs(1.0 - ref)), np.max(d)))


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_06045_gb300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("sched", ["persistent", "per_bucket"])
def test_deduplicated_small_graph_matches_state_vector(dtype, sched):
    n, seed, p = 20, 3, 1
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    with qtgb.plan(n, edges, p, dtype=dtype, sched=sched, dedup=True) as pl:
        assert pl.stats()["n_unique"] < edges.shape[0]
        zz, E = pl.energy(g, b)
    ref = oracle.sv_zz(n, edges, g, b)
    assert scaled_err(zz, ref) <= TOL[dtype]
    assert abs(E - oracle.energy_from_zz(ref)) <= TOL[dtype] * abs(E)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_deduplicated_batch_matches_full_plan_and_oracle(dtype):
    """A batch like the 64-graph workload (p=3, N in [50, 300]): deduplicated
    and full plans agree per edge and per graph; sampled edges match the
    oracle."""
    graphs = synth.batch(8, 3, lo=50, hi=300, base_seed=1000)
    spec = [(n, e) for n, e, _, _ in graphs]
    G = np.array([gg for _, _, gg, _ in graphs])
    Bt = np.array([bb for _, _, _, bb in graphs])
    with qtgb.plan_batch(spec, 3, dtype=dtype, dedup=True) as pl:
        st = pl.stats()
        e_d, zz_d = pl.energy_batch(G, Bt)
    with qtgb.plan_batch(spec, 3, dtype=dtype) as pl:
        e_f, zz_f = pl.energy_batch(G, Bt)
    assert st["n_unique"] < st["n_networks"]
    assert scaled_err(zz_d, zz_f) <= TOL[dtype]
    assert np.all(np.abs(e_d - e_f) <= TOL[dtype] * np.abs(e_f))
    first = np.cumsum([0] + [e.shape[0] for _, e, _, _ in graphs])
    rng = np.random.default_rng(3)
    for f in np.sort(rng.choice(first[-1], size=20, replace=False)):
        gi = int(np.searchsorted(first, f, side="right") - 1)
        n, edges, gg, bb = graphs[gi]
        ref, _ = oracle.edge_bucket(n, edges, gg, bb, int(f - first[gi]), seed=int(f))
        assert scaled_err([zz_d[f]], [ref.real]) <= TOL[dtype]


def test_deduplicated_sliced_representatives():
    """Representatives may be sliced: duplicates take the sum over the
    representative's slices."""
    n, seed, p = 60, 3, 2
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    with qtgb.plan(n, edges, p, dtype="c128", dedup=True, slice_width=4) as pl:
        st = pl.stats()
        zz, E = pl.energy(g, b)
    with qtgb.plan(n, edges, p, dtype="c128", slice_width=-1) as pl:
        zz_f, E_f = pl.energy(g, b)
    assert st["n_unique"] < edges.shape[0] and st["slice_bits"] > 0
    assert scaled_err(zz, zz_f) <= TOL["c128"]
    assert abs(E - E_f) <= TOL["c128"] * abs(E_f)


def test_deduplicated_plan_without_device_allocation():
    n, seed, p = 20, 3, 1
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    with qtgb.plan(n, edges, p, dtype="c128", host_only=True, dedup=True) as pl:
        energies, zz = pl.energy_noalloc(g, b)
    ref = oracle.sv_zz(n, edges, g, b)
    assert scaled_err(zz, ref) <= TOL["c128"]
