"""GPU parity of merged eliminations (the default; opts.no_merge turns them off).

A bucket whose consumer only extends it by its own summed variable is merged
with that consumer: one bucket sums two variables (s0, then s1) and the
intermediate result is never written. The persistent kernel contracts it as
the bucket of s0 with outputs (o, s1), the consumer's gate tensors folded into
its gate table, and adds each lane's two outputs (s1 = 0, 1) into result o
(inside the unrolled tile loop for complex64, in a compact loop of its own for
complex128).
These tests run merged (unsliced) plans against the state vector, the stored
goldens and the oracle's own bucket elimination, with the tolerances of the other GPU
parity tests (1e-10 complex128, 1e-5 complex64 per edge, as in
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


def _merged_tiles(n, edges, p, **kw):
    """Tile bits of the merged buckets of the plan these options give."""
    with qtgb.plan(n, edges, p, host_only=True, merge=True, **kw, slice_width=-1) as hp:
        B, _ = hp.export()
    return B["tile_log2"][B["n_sum"] > 1]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("order", ["simulated", "ready_queue"])
@pytest.mark.parametrize("n,seed,p", [(16, 23, 3), (18, 5, 4), (20, 1020, 4)])
def test_merged_small_graphs_match_state_vector(dtype, order, n, seed, p):
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    assert _merged_tiles(n, edges, p, dtype=dtype).size > 0
    with qtgb.plan(n, edges, p, dtype=dtype, order=order, merge=True, slice_width=-1) as pl:
        zz, E = pl.energy(g, b)
        im = pl.last_imag()
    ref = oracle.sv_zz(n, edges, g, b)
    assert scaled_err(zz, ref) <= TOL[dtype]
    assert abs(E - oracle.energy_from_zz(ref)) <= TOL[dtype] * abs(E)
    assert np.abs(im).max() <= 10 * TOL[dtype]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("cap", [2, 3, 5, 6, 7, 11])
def test_merged_tile_shapes(dtype, cap):
    """Tile caps below 6 send merged tiles through the generic tile loop (2 to
    32 active lanes), 6..11 through the unrolled one (1 to 32 iterations of 64
    outputs); the gate table then sees the consumer's gates inside and above
    the tile."""
    n, seed, p = 18, 5, 4
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    tiles = _merged_tiles(n, edges, p, dtype=dtype, tile_cap=[cap] * 5)
    assert tiles.size > 0 and tiles.max() <= cap
    if cap <= 6:
        assert tiles.max() == cap
    with qtgb.plan(n, edges, p, dtype=dtype, merge=True, tile_cap=[cap] * 5, slice_width=-1) as pl:
        zz, E = pl.energy(g, b)
    ref = oracle.sv_zz(n, edges, g, b)
    assert scaled_err(zz, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("order", ["simulated", "ready_queue"])
def test_merged_c2_n30_p4_matches_statevector_golden(dtype, order):
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
    # the plain greedy order (no restarts), on which merging halves the bytes
    with qtgb.plan(n, edges, p, dtype=dtype, order=order, merge=True, slice_width=-1, restarts=-1) as pl:
        st = pl.stats()
        zz, E = pl.energy(g, b)
        im = pl.last_imag()
    with qtgb.plan(n, edges, p, dtype=dtype, host_only=True, merge=False, slice_width=-1, restarts=-1) as hp:
        st1 = hp.stats()
    assert st["n_buckets"] < st1["n_buckets"] and st["alg_bytes"] < 0.6 * st1["alg_bytes"]
    assert scaled_err(zz, np.array(zz_ref)) <= TOL[dtype]
    assert abs(E - rows["energy"][0]) <= TOL[dtype] * abs(E)
    assert np.abs(im).max() <= 10 * TOL[dtype]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_merged_c4_wide_networks_match_min_fill_golden(dtype):
    """The N=1000 p=5 networks of greedy width 26..28 (merged buckets of up to
    2^26 outputs) against the oracle's complex128 values."""
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
    with qtgb.plan(n, edges, p, host_only=True, slice_width=-1, restarts=-1) as hp:
        B, _ = hp.export()
    mw = np.zeros(edges.shape[0], dtype=np.int64)
    np.maximum.at(mw, B["network"], B["width"])
    sel = np.nonzero((mw >= 26) & (mw <= 28))[0]
    with qtgb.plan_subset(n, edges, p, sel, dtype=dtype, merge=True, slice_width=-1) as pl:
        zz, _ = pl.energy(g, b)
        im = pl.last_imag()
    assert scaled_err(zz, np.array([ref[int(e)] for e in sel])) <= TOL[dtype]
    assert np.abs(im).max() <= 10 * TOL[dtype]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_merged_c3_batch_sampled_edges_match_oracle(dtype):
    """The 64-graph N in [50, 1000] p=3 batch with merging and fused units: 60
    sampled edges against the oracle's bucket elimination of their networks."""
    p = 3
    graphs = synth.batch(64, p, lo=50, hi=1000, base_seed=1000)
    G = np.array([gg for _, _, gg, _ in graphs])
    Bt = np.array([bb for _, _, _, bb in graphs])
    spec = [(n, e) for n, e, _, _ in graphs]
    with qtgb.plan_batch(spec, p, dtype=dtype, merge=True, slice_width=-1) as pl:
        assert pl.stats()["n_units"] > 0
        energies, zz = pl.energy_batch(G, Bt)
    rng = np.random.default_rng(11)
    first = np.cumsum([0] + [e.shape[0] for _, e, _, _ in graphs])
    for f in np.sort(rng.choice(first[-1], size=60, replace=False)):
        gi = int(np.searchsorted(first, f, side="right") - 1)
        n, edges, gg, bb = graphs[gi]
        ref, _ = oracle.edge_bucket(n, edges, gg, bb, int(f - first[gi]), seed=int(f))
        assert scaled_err([zz[f]], [ref.real]) <= TOL[dtype]


def test_merged_and_unmerged_agree_on_a_batch():
    """Same batch, merged and not: per-graph energies within the complex64
    tolerance of each other (both against the complex128 merged values)."""
    graphs = synth.batch(8, 3, lo=40, hi=200, base_seed=500)
    G = np.array([gg for _, _, gg, _ in graphs])
    Bt = np.array([bb for _, _, _, bb in graphs])
    spec = [(n, e) for n, e, _, _ in graphs]
    out = {}
    for dtype, merge in [("c128", True), ("c64", True), ("c64", False)]:
        with qtgb.plan_batch(spec, 3, dtype=dtype, merge=merge, slice_width=-1) as pl:
            out[(dtype, merge)] = pl.energy_batch(G, Bt)
    e_ref, zz_ref = out[("c128", True)]
    for key in [("c64", True), ("c64", False)]:
        e, zz = out[key]
        assert scaled_err(zz, zz_ref) <= TOL["c64"]
        assert np.all(np.abs(e - e_ref) <= TOL["c64"] * np.abs(e_ref))
