"""GPU parity: qt_energy / qt_energy_batch through the C ABI against the oracle.

Per edge, two measures must stay within tol (1e-10 for complex128, 1e-5 for
complex64 with FP32 arithmetic):
* the relative error of the per-edge energy <C_jk> = (1 - e_jk)/2, the edge's
  term in E = sum_jk (1 - e_jk)/2 (§II-B edge decomposition);
* the absolute error of e_jk = <Z_jZ_k>, a quantity bounded by 1.
The energy E must match to tol relative, and |Im| of every network value must
stay within 10 * tol.
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
    """Larger of: relative error of (1 - e)/2 per edge, absolute error of e per edge."""
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
def test_c1_p1_matches_state_vector_and_closed_form(dtype, sched):
    n, p, seed = 10, 1, 1000
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    with qtgb.plan(n, edges, p, dtype=dtype, sched=sched) as pl:
        zz, E = pl.energy(g, b)
        im = pl.last_imag()
    ref = oracle.sv_zz(n, edges, g, b)
    assert scaled_err(zz, ref) <= TOL[dtype]
    assert scaled_err(zz, oracle.p1_closed_form(n, edges, g[0], b[0])) <= TOL[dtype]
    assert abs(E - oracle.energy_from_zz(ref)) <= TOL[dtype] * abs(E)
    assert np.abs(im).max() <= 10 * TOL[dtype]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,seed,p", [(12, 21, 2), (14, 22, 3), (16, 23, 3), (20, 1020, 4), (18, 5, 4)])
def test_small_graphs_match_state_vector(dtype, n, seed, p):
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    with qtgb.plan(n, edges, p, dtype=dtype) as pl:
        zz, E = pl.energy(g, b)
    ref = oracle.sv_zz(n, edges, g, b)
    assert scaled_err(zz, ref) <= TOL[dtype]
    assert abs(E - oracle.energy_from_zz(ref)) <= TOL[dtype] * abs(E)


@pytest.mark.parametrize("name,n,edges", [("K4", 4, synth.complete_graph(4)), ("prism", 6, synth.prism_graph()),
                                          ("petersen", 10, synth.petersen_graph()), ("ring", 9, synth.ring_graph(9))])
def test_degenerate_small_graphs(name, n, edges):
    for p in (1, 2, 3):
        g, b = synth.angles(p, 4)
        ref = oracle.sv_zz(n, edges, g, b)
        with qtgb.plan(n, edges, p, dtype="c128") as pl:
            zz, _ = pl.energy(g, b)
        assert scaled_err(zz, ref) <= TOL["c128"]


def test_single_edge_graph():
    edges = np.array([[0, 1]])
    g, b = [0.3, 0.8], [0.5, 0.1]
    ref = oracle.sv_zz(2, edges, g, b)
    with qtgb.plan(2, edges, 2, dtype="c128") as pl:
        zz, E = pl.energy(g, b)
    assert scaled_err(zz, ref) <= TOL["c128"]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_invariants(dtype):
    n, p = 30, 4
    edges = synth.random_regular_graph(n, 1000)
    m = edges.shape[0]
    with qtgb.plan(n, edges, p, dtype=dtype) as pl:
        zz, E = pl.energy(np.zeros(p), np.zeros(p))
        assert np.abs(zz).max() <= TOL[dtype] and abs(E - m / 2) <= TOL[dtype] * m
        g, _ = synth.angles(p, 1000)
        zz, E = pl.energy(g, np.zeros(p))
        assert np.abs(zz).max() <= 10 * TOL[dtype]
        g, b = synth.angles(p, 1000)
        zz, E = pl.energy(g, b)
        assert np.all(np.abs(zz) <= 1 + 10 * TOL[dtype]) and -1e-9 <= E <= m + 1e-9
        zz2, _ = pl.energy(g + np.pi, b + np.pi)
        assert scaled_err(zz2, zz) <= 10 * TOL[dtype]


def _golden_edges(name):
    rows = {}
    zz = []
    for line in (GOLDEN / name).read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        parts = line.split()
        if parts[0] == "edge":
            zz.append(float(parts[4]))
        else:
            rows[parts[0]] = [float(x) for x in parts[1:]]
    return rows, np.array(zz)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("sched,order", [("persistent", "simulated"), ("persistent", "ready_queue"),
                                         ("per_bucket", "simulated")])
def test_c2_n30_p4_matches_statevector_golden(dtype, sched, order):
    if not (GOLDEN / "c2_n30_p4_statevector.txt").exists():
        pytest.skip("golden not generated")
    rows, ref = _golden_edges("c2_n30_p4_statevector.txt")
    n, p = 30, 4
    edges = synth.random_regular_graph(n, 1000)
    g, b = np.array(rows["gamma"]), np.array(rows["beta"])
    np.testing.assert_array_equal((g, b), synth.angles(p, 1000))
    with qtgb.plan(n, edges, p, dtype=dtype, sched=sched, order=order) as pl:
        zz, E = pl.energy(g, b)
        im = pl.last_imag()
    assert scaled_err(zz, ref) <= TOL[dtype]
    assert abs(E - rows["energy"][0]) <= TOL[dtype] * abs(E)
    assert np.abs(im).max() <= 10 * TOL[dtype]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_autotuned_plan_matches_state_vector(dtype):
    """opts.autotune: every candidate layout is uploaded and timed; the plan
    left behind must still give the oracle's values."""
    n, p = 20, 4
    edges = synth.random_regular_graph(n, 1020)
    g, b = synth.angles(p, 1020)
    with qtgb.plan(n, edges, p, dtype=dtype, autotune=2) as pl:
        st = pl.stats()
        zz, E = pl.energy(g, b)
    assert st["tune_candidates"] > 1 and st["tune_seconds"] > 0
    assert all(6 <= c <= 11 for c in st["tile_cap"]) and st["run_tiles"] in (8, 12, 16, 32)
    ref = oracle.sv_zz(n, edges, g, b)
    assert scaled_err(zz, ref) <= TOL[dtype]
    assert abs(E - oracle.energy_from_zz(ref)) <= TOL[dtype] * abs(E)


def _c4_golden():
    rows, ref = {}, {}
    with open(GOLDEN / "c4_n1000_p5_bucket.txt") as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if parts[0] == "edge":
                ref[int(parts[1])] = (float(parts[4]), float(parts[5]))
            else:
                rows[parts[0]] = [float(x) for x in parts[1:]]
    return rows, ref


def _c4_inputs():
    n, p = 1000, 5
    edges = synth.random_regular_graph(n, 1000)
    g, b = synth.angles(p, 1000)
    return n, p, edges, g, b


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_c4_wide_networks_match_min_fill_golden(dtype):
    """The networks whose greedy order reaches width 26..28 (buckets of up to
    2^27 outputs) against the oracle's complex128 elimination in its own
    min-fill order."""
    if not (GOLDEN / "c4_n1000_p5_bucket.txt").exists():
        pytest.skip("golden not generated")
    rows, ref = _c4_golden()
    n, p, edges, g, b = _c4_inputs()
    np.testing.assert_array_equal((g, b), (np.array(rows["gamma"]), np.array(rows["beta"])))
    with qtgb.plan(n, edges, p, host_only=True, slice_width=-1, restarts=-1) as hp:
        B, _ = hp.export()
    mw = np.zeros(edges.shape[0], dtype=np.int64)
    np.maximum.at(mw, B["network"], B["width"])
    sel = np.nonzero((mw >= 26) & (mw <= 28))[0]
    assert sel.size == 15
    with qtgb.plan_subset(n, edges, p, sel, dtype=dtype) as pl:
        zz, _ = pl.energy(g, b)
        im = pl.last_imag()
    want = np.array([ref[int(e)][0] for e in sel])
    assert scaled_err(zz, want) <= TOL[dtype]
    assert np.abs(im).max() <= 10 * TOL[dtype]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_c4_whole_graph_energy_matches_golden(dtype):
    """All 1500 lightcone networks of the N=1000 p=5 graph in one launch."""
    if not (GOLDEN / "c4_n1000_p5_bucket.txt").exists():
        pytest.skip("golden not generated")
    rows, ref = _c4_golden()
    n, p, edges, g, b = _c4_inputs()
    with qtgb.plan(n, edges, p, dtype=dtype) as pl:
        zz, E = pl.energy(g, b)
    want = np.array([ref[e][0] for e in range(edges.shape[0])])
    assert scaled_err(zz, want) <= TOL[dtype]
    assert abs(E - rows["energy"][0]) <= TOL[dtype] * abs(E)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_c5_n50_p4_matches_bucket_golden(dtype):
    if not (GOLDEN / "c5_n50_p4_bucket.txt").exists():
        pytest.skip("golden not generated")
    rows, ref = _golden_edges("c5_n50_p4_bucket.txt")
    n, p = 50, 4
    edges = synth.random_regular_graph(n, 1000)
    g, b = np.array(rows["gamma"]), np.array(rows["beta"])
    with qtgb.plan(n, edges, p, dtype=dtype) as pl:
        zz, E = pl.energy(g, b)
    assert scaled_err(zz, ref) <= TOL[dtype]


def _c3_sample(graphs, n_sample, seed):
    """(flat network index, graph, edge) of a seeded sample of the batch's edges."""
    rng = np.random.default_rng(seed)
    first = np.cumsum([0] + [e.shape[0] for _, e, _, _ in graphs])
    flat = np.sort(rng.choice(first[-1], size=n_sample, replace=False))
    gi = np.searchsorted(first, flat, side="right") - 1
    return [(int(f), int(g), int(f - first[g])) for f, g in zip(flat, gi)]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_c3_full_batch_sampled_edges_match_oracle(dtype):
    """The 64-graph, N in [50, 1000], p=3 batch at full size, in the persistent
    launch with fused units that the benchmark times: 100 sampled edges against
    the oracle's bucket elimination of their networks."""
    p = 3
    graphs = synth.batch(64, p, lo=50, hi=1000, base_seed=1000)
    G = np.array([gg for _, _, gg, _ in graphs])
    Bt = np.array([bb for _, _, _, bb in graphs])
    with qtgb.plan_batch([(n, e) for n, e, _, _ in graphs], p, dtype=dtype) as pl:
        assert pl.stats()["n_units"] > 0
        energies, zz = pl.energy_batch(G, Bt)
    for f, g, e in _c3_sample(graphs, 100, 7):
        n, edges, gg, bb = graphs[g]
        ref, _ = oracle.edge_bucket(n, edges, gg, bb, e, seed=f)
        assert scaled_err([zz[f]], [ref.real]) <= TOL[dtype]
        assert abs(ref.imag) < 1e-12


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("order", ["simulated", "ready_queue"])
def test_fused_units_match_unfused_and_oracle(dtype, order):
    """A batch with enough small buckets to form fused units (subtrees run in
    one warp's shared memory) against the same plan without units and the
    oracle's bucket elimination."""
    p = 3
    graphs = synth.batch(12, p, lo=50, hi=300, base_seed=2000)
    spec = [(n, e) for n, e, _, _ in graphs]
    G = np.array([gg for _, _, gg, _ in graphs])
    Bt = np.array([bb for _, _, _, bb in graphs])
    with qtgb.plan_batch(spec, p, dtype=dtype, order=order) as pl:
        assert pl.stats()["n_units"] > 0
        e_f, zz_f = pl.energy_batch(G, Bt)
    with qtgb.plan_batch(spec, p, dtype=dtype, order=order, fuse=False) as pl:
        assert pl.stats()["n_units"] == 0
        e_u, zz_u = pl.energy_batch(G, Bt)
    assert scaled_err(zz_f, zz_u) <= TOL[dtype]
    first = 0
    for gi, (n, e, gg, bb) in enumerate(graphs[:3]):
        ref, _ = oracle.bucket_zz(n, e, gg, bb, seed=1)
        m = e.shape[0]
        assert scaled_err(zz_f[first:first + m], ref.real) <= TOL[dtype]
        first += m


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("sched", ["persistent", "per_bucket"])
def test_graphs_without_edges(dtype, sched):
    """An edgeless graph has energy 0 (no networks); in a batch it leaves the
    other graphs' energies unchanged."""
    empty = np.zeros((0, 2), dtype=np.int32)
    g, b = synth.angles(2, 5)
    with qtgb.plan(6, empty, 2, dtype=dtype, sched=sched) as pl:
        zz, E = pl.energy(g, b)
    assert zz.size == 0 and E == 0.0
    n, edges = 10, synth.random_regular_graph(10, 1)
    graphs = [(6, empty), (n, edges), (3, empty)]
    G = np.tile(g, (3, 1))
    Bt = np.tile(b, (3, 1))
    with qtgb.plan_batch(graphs, 2, dtype=dtype, sched=sched) as pl:
        energies, zz = pl.energy_batch(G, Bt)
    ref = oracle.sv_zz(n, edges, g, b)
    assert energies[0] == 0.0 and energies[2] == 0.0
    assert scaled_err(zz, ref) <= TOL[dtype]
    assert abs(energies[1] - oracle.energy_from_zz(ref)) <= TOL[dtype] * abs(energies[1])


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_whole_networks_as_fused_units(dtype):
    """p=1 networks are small enough that each network's whole bucket tree is
    one fused unit, its root the network's scalar: energies against the p=1
    closed form."""
    graphs = synth.batch(200, 1, lo=20, hi=60, base_seed=4000)
    spec = [(n, e) for n, e, _, _ in graphs]
    with qtgb.plan_batch(spec, 1, dtype=dtype) as pl:
        st = pl.stats()
        assert st["n_units"] == st["n_networks"] and st["n_fused"] == st["n_buckets"]
        G = np.array([gg for _, _, gg, _ in graphs])
        Bt = np.array([bb for _, _, _, bb in graphs])
        _, zz = pl.energy_batch(G, Bt)
    first = 0
    for n, e, gg, bb in graphs[:20]:
        m = e.shape[0]
        assert scaled_err(zz[first:first + m], oracle.p1_closed_form(n, e, gg[0], bb[0])) <= TOL[dtype]
        first += m


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("order", ["simulated", "ready_queue"])
def test_batch_of_graphs_matches_oracle(dtype, order):
    p = 3
    graphs = synth.batch(6, p, lo=50, hi=120, base_seed=1000)
    with qtgb.plan_batch([(n, e) for n, e, _, _ in graphs], p, dtype=dtype, order=order) as pl:
        G = np.array([gg for _, _, gg, _ in graphs])
        B = np.array([bb for _, _, _, bb in graphs])
        energies, zz = pl.energy_batch(G, B)
    at = 0
    for i, (n, e, gg, bb) in enumerate(graphs):
        vals, _ = oracle.bucket_zz(n, e, gg, bb, seed=3)
        part = zz[at:at + e.shape[0]]
        at += e.shape[0]
        assert scaled_err(part, vals.real) <= TOL[dtype]
        assert abs(energies[i] - oracle.energy_from_zz(vals.real)) <= TOL[dtype] * abs(energies[i])


def test_device_buffers_and_stream():
    n, p = 16, 3
    edges = synth.random_regular_graph(n, 8)
    g, b = synth.angles(p, 8)
    ref = oracle.sv_zz(n, edges, g, b)
    s = torch.cuda.Stream()
    with qtgb.plan(n, edges, p, dtype="c128") as pl:
        gd = torch.tensor(g, dtype=torch.float64, device="cuda")
        bd = torch.tensor(b, dtype=torch.float64, device="cuda")
        zz = torch.zeros(edges.shape[0], dtype=torch.float64, device="cuda")
        E = torch.zeros(1, dtype=torch.float64, device="cuda")
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            pl.energy(gd, bd, edge_zz=zz, energy=E, stream=s)
        pl.sync(s)
        assert scaled_err(zz.cpu().numpy(), ref) <= TOL["c128"]
        assert abs(E.item() - oracle.energy_from_zz(ref)) <= 1e-10 * abs(E.item())


def test_repeat_calls_are_bitwise_identical():
    n, p = 30, 4
    edges = synth.random_regular_graph(n, 1000)
    g, b = synth.angles(p, 1000)
    with qtgb.plan(n, edges, p, dtype="c64") as pl:
        first, _ = pl.energy(g, b)
        for _ in range(3):
            again, _ = pl.energy(g, b)
            np.testing.assert_array_equal(first, again)


def test_stalled_dependency_times_out_and_context_survives():
    n, p = 12, 2
    edges = synth.random_regular_graph(n, 3)
    g, b = synth.angles(p, 3)
    # without fused units every bucket waits on its producers' counters
    with qtgb.plan(n, edges, p, dtype="c64", spin_limit=2000, fuse=False) as pl:
        B, _ = pl.export()
        victim = int(np.nonzero(B["parent"] >= 0)[0][-1])  # a producer: its consumer can never start
        pl.debug_stall_bucket(victim)
        with pytest.raises(qtgb.QTError) as ei:
            pl.energy(g, b)
        assert ei.value.code == qtgb.QT_ETIMEOUT
    # the context is still usable
    with qtgb.plan(n, edges, p, dtype="c128") as pl:
        zz, _ = pl.energy(g, b)
    assert scaled_err(zz, oracle.sv_zz(n, edges, g, b)) <= TOL["c128"]


def test_kernel_time_counts_launches():
    n, p = 20, 3
    edges = synth.random_regular_graph(n, 2)
    g, b = synth.angles(p, 2)
    with qtgb.plan(n, edges, p) as pl:
        pl.kernel_time(reset=True)
        for _ in range(5):
            pl.energy(g, b)
        ms, cnt = pl.kernel_time(reset=True)
        assert cnt == 5 and ms > 0
