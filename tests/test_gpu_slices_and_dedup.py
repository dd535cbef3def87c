"""GPU parity of plans that split or share networks.

Index slicing (opts.slice_width): a network wider than the target has
variables fixed; its value is the sum, over the 2^s assignments of the fixed
variables, of networks without them. Gates left with one free variable read
the entry pair at 2 * (fixed value) of their table; gates with every variable
fixed are scalars the epilogue multiplies into their slice's product before
the slices are summed. Slices may be split over shards or passes.

Lightcone deduplication (opts.dedup): within one graph, networks whose
lightcones are isomorphic are contracted once; the others take that
network's value (the epilogue reads the representative's results).

These tests run such plans against the state vector, the stored goldens, the
full plans and the oracle's bucket elimination, with the tolerances of the
other GPU parity tests (1e-10 complex128, 1e-5 complex64 per edge, as in
test_gpu_energy).
"""
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_2204_06045_gb300 import qtgb, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = Path(__file__).parent / "golden"
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
@pytest.mark.parametrize("sched,order", [("persistent", "simulated"), ("persistent", "ready_queue"),
                                         ("per_bucket", "simulated")])
@pytest.mark.parametrize("n,seed,p,width", [(14, 22, 3, 8), (18, 5, 4, 14)])
def test_sliced_small_graphs_match_state_vector(dtype, sched, order, n, seed, p, width):
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    with qtgb.plan(n, edges, p, dtype=dtype, sched=sched, order=order, slice_width=width) as pl:
        st = pl.stats()
        zz, E = pl.energy(g, b)
        im = pl.last_imag()
    assert st["slice_bits"] > 0 and st["n_slices"] > edges.shape[0]
    ref = oracle.sv_zz(n, edges, g, b)
    assert scaled_err(zz, ref) <= TOL[dtype]
    assert abs(E - oracle.energy_from_zz(ref)) <= TOL[dtype] * abs(E)
    assert np.abs(im).max() <= 10 * TOL[dtype]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_sliced_c2_n30_p4_matches_statevector_golden(dtype):
    """Networks of greedy width up to 26 sliced to width 20 or less."""
    if not (GOLDEN / "c2_n30_p4_statevector.txt").exists():
        pytest.skip("golden not generated")
    rows, zz_ref = {}, []
    for line in (GOLDEN / "c2_n30_p4_statevector.txt").read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        parts = line.split()
        if parts[0] == "edge":
            zz_ref.append(float(parts[4]))
        else:
            rows[parts[0]] = [float(x) for x in parts[1:]]
    n, p = 30, 4
    edges = synth.random_regular_graph(n, 1000)
    g, b = np.array(rows["gamma"]), np.array(rows["beta"])
    with qtgb.plan(n, edges, p, dtype=dtype, slice_width=20) as pl:
        st = pl.stats()
        zz, E = pl.energy(g, b)
    assert st["max_width"] <= 20 and st["slice_bits"] > 0
    assert scaled_err(zz, np.array(zz_ref)) <= TOL[dtype]
    assert abs(E - rows["energy"][0]) <= TOL[dtype] * abs(E)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_sliced_c4_wide_networks_match_min_fill_golden(dtype):
    """The N=1000 p=5 networks of greedy width 26..28, sliced to width 24."""
    path = GOLDEN / "c4_n1000_p5_bucket.txt"
    if not path.exists():
        pytest.skip("golden not generated")
    ref = {}
    for line in path.read_text().splitlines():
        parts = line.split()
        if parts and parts[0] == "edge":
            ref[int(parts[1])] = float(parts[4])
    n, p = 1000, 5
    edges = synth.random_regular_graph(n, 1000)
    g, b = synth.angles(p, 1000)
    with qtgb.plan(n, edges, p, host_only=True, merge=False, slice_width=-1, restarts=-1) as hp:
        B, _ = hp.export()
    mw = np.zeros(edges.shape[0], dtype=np.int64)
    np.maximum.at(mw, B["network"], B["width"])
    sel = np.nonzero((mw >= 26) & (mw <= 28))[0]
    with qtgb.plan_subset(n, edges, p, sel, dtype=dtype, slice_width=24) as pl:
        st = pl.stats()
        zz, _ = pl.energy(g, b)
    assert st["max_width"] <= 24 and st["slice_bits"] > 0
    assert scaled_err(zz, np.array([ref[int(e)] for e in sel])) <= TOL[dtype]


def test_sliced_batch_with_fused_units_matches_oracle():
    """A batch whose slices are small enough to run as fused units."""
    graphs = synth.batch(6, 2, lo=30, hi=80, base_seed=900)
    spec = [(n, e) for n, e, _, _ in graphs]
    G = np.array([gg for _, _, gg, _ in graphs])
    Bt = np.array([bb for _, _, _, bb in graphs])
    with qtgb.plan_batch(spec, 2, dtype="c128", slice_width=5) as pl:
        st = pl.stats()
        energies, zz = pl.energy_batch(G, Bt)
    assert st["slice_bits"] > 0 and st["n_units"] > 0
    first = np.cumsum([0] + [e.shape[0] for _, e, _, _ in graphs])
    rng = np.random.default_rng(5)
    for f in np.sort(rng.choice(first[-1], size=20, replace=False)):
        gi = int(np.searchsorted(first, f, side="right") - 1)
        n, edges, gg, bb = graphs[gi]
        ref, _ = oracle.edge_bucket(n, edges, gg, bb, int(f - first[gi]), seed=int(f))
        assert scaled_err([zz[f]], [ref.real]) <= TOL["c128"]


def test_sliced_plan_without_device_allocation():
    """qt_energy_noalloc uploads the epilogue's factor lists into its static array too."""
    n, seed, p = 14, 22, 3
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    with qtgb.plan(n, edges, p, dtype="c128", host_only=True, slice_width=8) as pl:
        energies, zz = pl.energy_noalloc(g, b)
    ref = oracle.sv_zz(n, edges, g, b)
    assert scaled_err(zz, ref) <= TOL["c128"]
    assert abs(energies[0] - oracle.energy_from_zz(ref)) <= TOL["c128"] * abs(energies[0])


def test_slice_shards_add_up_to_the_full_plan():
    """qt_plan_shard with slicing: the ranks' plans (run one after another on
    this GPU) hold subsets of the networks' slices; their per-edge values and
    partial energies (the rank holding slice 0 counts the edge's 1/2) add up to
    the unsharded plan's."""
    n, seed, p, world = 16, 23, 3, 3
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    with qtgb.plan(n, edges, p, dtype="c128", slice_width=8) as full:
        zz_full, E_full = full.energy(g, b)
    zz_sum = np.zeros(edges.shape[0])
    E_sum = 0.0
    holders = np.zeros(edges.shape[0], dtype=int)
    for r in range(world):
        with qtgb.plan_shard(n, edges, p, world, r, dtype="c128", slice_width=8) as pl:
            mine = pl.shard_edges
            zz, E = pl.energy(g, b)
        zz_sum[mine] += zz
        holders[mine] += 1
        E_sum += E
    assert holders.max() > 1  # some network's slices are spread over ranks
    np.testing.assert_allclose(zz_sum, zz_full, rtol=0, atol=1e-10)
    assert abs(E_sum - E_full) <= 1e-10 * abs(E_full)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_energy_budget_passes_match_the_whole_plan(dtype):
    """opts.energy_budget_bytes: the N=30 p=4 plan run in passes over its
    slices (one shared arena a tenth of the whole plan's) gives the whole
    plan's per-edge values and energy; a subset plan in passes returns its
    networks' values in its own order."""
    n, p = 30, 4
    edges = synth.random_regular_graph(n, 1000)
    g, b = synth.angles(p, 1000)
    with qtgb.plan(n, edges, p, dtype=dtype) as pl:
        full = pl.stats()["arena_bytes"]
        zz_f, E_f = pl.energy(g, b)
    with qtgb.plan(n, edges, p, dtype=dtype, energy_budget_bytes=full // 10) as pl:
        st = pl.stats()
        zz, E = pl.energy(g, b)
    assert st["n_passes"] > 1 and st["pass_arena_bytes"] <= full // 10
    assert scaled_err(zz, zz_f) <= TOL[dtype]
    assert abs(E - E_f) <= TOL[dtype] * abs(E_f)
    sel = np.array([3, 17, 40, 8])
    with qtgb.plan_subset(n, edges, p, sel, dtype=dtype, energy_budget_bytes=full // 20) as pl:
        assert pl.stats()["n_passes"] > 1
        zz_s, _ = pl.energy(g, b)
    assert scaled_err(zz_s, zz_f[sel]) <= TOL[dtype]


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


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_deduplicated_gradient_matches_the_full_plan(dtype):
    """opts.dedup with gradients: the reverse sweep seeds each representative
    once for its whole class; energy and derivatives equal the full plan's."""
    n, seed, p = 60, 3, 2
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    with qtgb.plan(n, edges, p, dtype=dtype, with_grad=True, dedup=True) as pl:
        assert pl.stats()["n_unique"] < edges.shape[0]
        E, dg, db = pl.energy_grad(g, b)
    with qtgb.plan(n, edges, p, dtype=dtype, with_grad=True) as pl:
        E_f, dg_f, db_f = pl.energy_grad(g, b)
    tol = {"c128": 1e-9, "c64": 1e-4}[dtype]
    assert abs(E[0] - E_f[0]) <= tol * abs(E_f[0])
    np.testing.assert_allclose(dg, dg_f, rtol=0, atol=tol * max(1.0, np.abs(dg_f).max()))
    np.testing.assert_allclose(db, db_f, rtol=0, atol=tol * max(1.0, np.abs(db_f).max()))


def test_deduplicated_gradient_matches_oracle_finite_differences():
    """The N=60 p=2 graph whose lightcones repeat, complex128, deduplicated:
    energy and gradient against central differences (h = 1e-5) of the
    oracle's bucket-elimination energy (stored values)."""
    rows = {}
    for line in (Path(__file__).parent / "golden" / "dedup_n60_p2_fd.txt").read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            k, *v = line.split()
            rows[k] = np.array([float(x) for x in v])
    n, seed, p = 60, 3, 2
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    with qtgb.plan(n, edges, p, dtype="c128", with_grad=True, dedup=True) as pl:
        assert pl.stats()["n_unique"] < edges.shape[0]
        E, dg, db = pl.energy_grad(g, b)
    ref = np.concatenate([rows["dE_dgamma"], rows["dE_dbeta"]])
    assert np.abs(np.concatenate([dg, db]) - ref).max() <= 1e-6
    assert abs(E[0] - rows["energy"][0]) <= 1e-10 * abs(rows["energy"][0])


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_deduplicated_batch_gradient_matches_full_plans(dtype):
    """A batch gradient plan with deduplication over three graphs of
    different sizes (duplicates in each): per graph, energy and derivatives
    equal those of the full batch plan, and those of each graph planned alone."""
    p = 2
    graphs = [(60, synth.random_regular_graph(60, 3)), (40, synth.random_regular_graph(40, 8)),
              (80, synth.random_regular_graph(80, 11))]
    G = np.array([synth.angles(p, s)[0] for s in (3, 8, 11)])
    B = np.array([synth.angles(p, s)[1] for s in (3, 8, 11)])
    with qtgb.plan_batch(graphs, p, dtype=dtype, with_grad=True, dedup=True) as pl:
        st = pl.stats()
        E, dg, db = pl.energy_grad(G, B)
    with qtgb.plan_batch(graphs, p, dtype=dtype, with_grad=True) as pl:
        E_f, dg_f, db_f = pl.energy_grad(G, B)
    assert st["n_unique"] < st["n_networks"]
    tol = {"c128": 1e-9, "c64": 1e-4}[dtype]
    for i, (n, e) in enumerate(graphs):
        with qtgb.plan(n, e, p, dtype=dtype, with_grad=True, dedup=True) as one:
            E1, dg1, db1 = one.energy_grad(G[i], B[i])
        sl = slice(i * p, (i + 1) * p)
        for a, b_ in ((E[i], E_f[i]), (E[i], E1[0])):
            assert abs(a - b_) <= tol * abs(b_)
        scale = max(1.0, np.abs(np.concatenate([dg_f[sl], db_f[sl]])).max())
        for got_g, got_b in ((dg[sl], db[sl]), (dg1, db1)):
            np.testing.assert_allclose(got_g, dg_f[sl], rtol=0, atol=tol * scale)
            np.testing.assert_allclose(got_b, db_f[sl], rtol=0, atol=tol * scale)
