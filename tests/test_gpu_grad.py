"""GPU parity of the adjoint: qt_energy_grad through the C ABI.

References: the published p=1 closed form's derivative, the oracle's exact
parameter-shift gradient on a 2^20 state vector (stored values), central
finite differences of the complex128 energy (h = 1e-5), and the oracle's
parameter shift on small graphs. Gradients of the complex128 path must match
to 1e-6 absolute (1e-8 against exact references), those of the complex64
path to 1e-4 relative to the largest component.
"""
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_2204_06045_gb300 import qtgb, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
GOLDEN = Path(__file__).parent / "golden"


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_06045_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def grad_plan(n, edges, p, dtype="c128", **kw):
    return qtgb.plan(n, edges, p, dtype=dtype, with_grad=True, **kw)


@pytest.mark.parametrize("name,n,edges", [("petersen", 10, synth.petersen_graph()), ("prism", 6, synth.prism_graph()),
                                          ("K4", 4, synth.complete_graph(4))])
def test_p1_matches_closed_form_derivative(name, n, edges):
    for g, b in [(0.3, 0.7), (1.9, 0.2)]:
        with grad_plan(n, edges, 1) as pl:
            E, dg, db = pl.energy_grad([g], [b])
        cg, cb = oracle.p1_closed_form_grad(n, edges, g, b)
        assert abs(dg[0] - cg) < 1e-9 and abs(db[0] - cb) < 1e-9
        assert abs(E[0] - oracle.energy_from_zz(oracle.p1_closed_form(n, edges, g, b))) < 1e-10


def _golden_grad():
    rows = {}
    for line in (GOLDEN / "c5_n20_p4_gradient.txt").read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            k, *v = line.split()
            rows[k] = np.array([float(x) for x in v])
    return rows


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-8), ("c64", 1e-4)])
@pytest.mark.parametrize("sched", ["persistent", "per_bucket"])
def test_n20_p4_matches_parameter_shift_golden(dtype, tol, sched):
    rows = _golden_grad()
    n, p = 20, 4
    edges = synth.random_regular_graph(n, 1020)
    with grad_plan(n, edges, p, dtype=dtype, sched=sched) as pl:
        E, dg, db = pl.energy_grad(rows["gamma"], rows["beta"])
    ref = np.concatenate([rows["dE_dgamma"], rows["dE_dbeta"]])
    got = np.concatenate([dg, db])
    scale = 1.0 if dtype == "c128" else np.abs(ref).max()
    assert np.abs(got - ref).max() <= tol * scale, (got, ref)
    assert abs(E[0] - rows["energy"][0]) <= (1e-10 if dtype == "c128" else 1e-5) * abs(E[0])


def _golden_rows(name):
    rows = {}
    for line in (GOLDEN / name).read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            k, *v = line.split()
            rows[k] = np.array([float(x) for x in v])
    return rows


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_c5_n50_p4_sampled_edges_match_oracle_finite_differences(dtype):
    """N=50 p=4 (seed 1000), 8 seeded edges: the adjoint of a subset plan of
    their networks against central differences (h = 1e-5) of their energy
    share computed by the oracle's own bucket elimination (stored values)."""
    rows = _golden_rows("c5_n50_p4_fd.txt")
    n, p = 50, 4
    edges = synth.random_regular_graph(n, 1000)
    g, b = synth.angles(p, 1000)
    np.testing.assert_array_equal(g, rows["gamma"])
    np.testing.assert_array_equal(b, rows["beta"])
    sel = rows["edges"].astype(np.int32)
    with qtgb.plan_subset(n, edges, p, sel, dtype=dtype, with_grad=True) as pl:
        E, dg, db = pl.energy_grad(g, b)
    ref = np.concatenate([rows["dE_dgamma"], rows["dE_dbeta"]])
    got = np.concatenate([dg, db])
    if dtype == "c128":
        assert np.abs(got - ref).max() <= 1e-6, (got, ref)
        assert abs(E[0] - rows["energy"][0]) <= 1e-10 * abs(rows["energy"][0])
    else:
        assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max(), (got, ref)
        assert abs(E[0] - rows["energy"][0]) <= 1e-5 * abs(rows["energy"][0])


def test_c5_n50_p4_adjoint_matches_differences_of_its_own_energy():
    """Self-consistency of the whole N=50 p=4 graph: the complex128 adjoint
    against central differences of this library's own complex128 energy (the
    oracle comparison is the sampled-edge test above)."""
    n, p = 50, 4
    edges = synth.random_regular_graph(n, 1000)
    g, b = synth.angles(p, 1000)
    with grad_plan(n, edges, p) as pl, qtgb.plan(n, edges, p, dtype="c128") as pe:
        E, dg, db = pl.energy_grad(g, b)
        fd = oracle.grad_fd(lambda G, B: pe.energy(G, B)[1], g, b, h=1e-5)
        _, E2 = pe.energy(g, b)
    np.testing.assert_allclose(dg, fd[0], rtol=0, atol=1e-6)
    np.testing.assert_allclose(db, fd[1], rtol=0, atol=1e-6)
    assert abs(E[0] - E2) < 1e-10 * abs(E2)


def test_c5_c64_gradient_close_to_c128():
    n, p = 50, 4
    edges = synth.random_regular_graph(n, 1000)
    g, b = synth.angles(p, 1000)
    with grad_plan(n, edges, p, dtype="c128") as a, grad_plan(n, edges, p, dtype="c64") as c:
        _, dg1, db1 = a.energy_grad(g, b)
        _, dg2, db2 = c.energy_grad(g, b)
    ref = np.concatenate([dg1, db1])
    assert np.abs(np.concatenate([dg2, db2]) - ref).max() <= 1e-4 * np.abs(ref).max()


@pytest.mark.parametrize("order", ["simulated", "ready_queue"])
def test_batch_gradient_matches_parameter_shift(order):
    p = 2
    graphs = [(8, synth.random_regular_graph(8, 3)), (10, synth.random_regular_graph(10, 4)),
              (12, synth.random_regular_graph(12, 5))]
    G = np.array([synth.angles(p, s)[0] for s in (3, 4, 5)])
    B = np.array([synth.angles(p, s)[1] for s in (3, 4, 5)])
    with qtgb.plan_batch(graphs, p, dtype="c128", with_grad=True, order=order) as pl:
        E, dg, db = pl.energy_grad(G, B)
    for i, (n, e) in enumerate(graphs):
        ps = oracle.grad_param_shift(n, e, G[i], B[i])
        np.testing.assert_allclose(dg[i * p:(i + 1) * p], ps[0], rtol=0, atol=1e-9)
        np.testing.assert_allclose(db[i * p:(i + 1) * p], ps[1], rtol=0, atol=1e-9)
        assert abs(E[i] - oracle.sv_energy(n, e, G[i], B[i])) < 1e-10


def test_zero_angles_give_zero_gradient_and_half_edges():
    n, p = 16, 3
    edges = synth.random_regular_graph(n, 6)
    with grad_plan(n, edges, p) as pl:
        E, dg, db = pl.energy_grad(np.zeros(p), np.zeros(p))
    assert abs(E[0] - edges.shape[0] / 2) < 1e-12
    # at gamma = beta = 0 the first-order change in beta still moves E, in gamma it does not
    assert np.abs(dg).max() < 1e-12


def test_torch_autograd_function():
    n, p = 12, 2
    edges = synth.random_regular_graph(n, 9)
    g0, b0 = synth.angles(p, 9)
    with grad_plan(n, edges, p) as pl:
        g = torch.tensor(g0, dtype=torch.float64, requires_grad=True)
        b = torch.tensor(b0, dtype=torch.float64, requires_grad=True)
        E = qtgb.qaoa_energy(pl, g, b)
        (2.0 * E).backward()
    ps = oracle.grad_param_shift(n, edges, g0, b0)
    np.testing.assert_allclose(g.grad.numpy(), 2 * ps[0], atol=1e-9)
    np.testing.assert_allclose(b.grad.numpy(), 2 * ps[1], atol=1e-9)
    assert abs(E.item() - oracle.sv_energy(n, edges, g0, b0)) < 1e-10


def test_torch_autograd_function_on_device(monkeypatch):
    """CUDA angle tensors: the angles, energy and gradient stay on the device
    (no host copy of the angles, no host sync inside forward); the values
    match the oracle's parameter shift once the stream has run."""
    n, p = 12, 2
    edges = synth.random_regular_graph(n, 9)
    g0, b0 = synth.angles(p, 9)
    with grad_plan(n, edges, p) as pl:
        g = torch.tensor(g0, dtype=torch.float64, device="cuda", requires_grad=True)
        b = torch.tensor(b0, dtype=torch.float64, device="cuda", requires_grad=True)

        def no_host(*a, **k):
            raise AssertionError("host copy or host sync inside forward")

        with monkeypatch.context() as m:
            m.setattr(torch.Tensor, "cpu", no_host)
            m.setattr(torch.Tensor, "numpy", no_host)
            m.setattr(torch.Tensor, "item", no_host)
            m.setattr(torch.cuda.Stream, "synchronize", no_host)
            E = qtgb.qaoa_energy(pl, g, b)
            (2.0 * E).backward()
        assert E.is_cuda and g.grad.is_cuda and b.grad.is_cuda
        torch.cuda.synchronize()
        pl.sync()
    ps = oracle.grad_param_shift(n, edges, g0, b0)
    np.testing.assert_allclose(g.grad.cpu().numpy(), 2 * ps[0], atol=1e-9)
    np.testing.assert_allclose(b.grad.cpu().numpy(), 2 * ps[1], atol=1e-9)
    assert abs(E.item() - oracle.sv_energy(n, edges, g0, b0)) < 1e-10


def test_energy_only_plan_refuses_gradient():
    n, p = 10, 1
    edges = synth.random_regular_graph(n, 1)
    with qtgb.plan(n, edges, p) as pl:
        with pytest.raises(qtgb.QTError) as ei:
            pl.energy_grad([0.1], [0.2])
        assert ei.value.code == qtgb.QT_ESTATE


def test_gradient_of_a_graph_without_edges_is_zero():
    empty = np.zeros((0, 2), dtype=np.int32)
    g, b = synth.angles(3, 2)
    with qtgb.plan(4, empty, 3, dtype="c64", with_grad=True) as pl:
        E, dg, db = pl.energy_grad(g, b)
    assert E[0] == 0.0 and not np.any(dg) and not np.any(db)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_sharded_energy_and_gradient_sum_to_the_whole(dtype):
    """Three ranks' shards (LPT by network cost), run one after the other on
    this GPU: their partial energies and gradients add up to the unsharded
    plan's."""
    n, p = 20, 3
    edges = synth.random_regular_graph(n, 1020)
    g, b = synth.angles(p, 1020)
    with qtgb.plan(n, edges, p, dtype=dtype, with_grad=True) as pl:
        E, dg, db = pl.energy_grad(g, b)
    tot_E, tot_g, tot_b, held = 0.0, np.zeros(p), np.zeros(p), []
    for rank in range(3):
        with qtgb.plan_shard(n, edges, p, 3, rank, dtype=dtype, with_grad=True) as sh:
            e_r, g_r, b_r = sh.energy_grad(g, b)
            held += sh.shard_edges.tolist()
        tot_E += e_r[0]
        tot_g += g_r
        tot_b += b_r
    assert sorted(held) == list(range(edges.shape[0]))
    tol = 1e-10 if dtype == "c128" else 1e-5
    assert abs(tot_E - E[0]) <= tol * abs(E[0])
    np.testing.assert_allclose(tot_g, dg, atol=tol * 10)
    np.testing.assert_allclose(tot_b, db, atol=tol * 10)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_gradient_under_a_memory_budget_matches_the_whole(dtype):
    """opts.adjoint_budget_bytes at a quarter of what the plan would hold: the
    networks run in passes on one shared arena; energy, edge values and
    gradient equal the unbudgeted plan's."""
    n, p = 30, 4
    edges = synth.random_regular_graph(n, 1000)
    g, b = synth.angles(p, 1000)
    with qtgb.plan(n, edges, p, dtype=dtype, with_grad=True) as pl:
        need = pl.stats()["arena_bytes"]
        E, dg, db = pl.energy_grad(g, b)
        zz, _ = pl.energy(g, b)
    with qtgb.plan(n, edges, p, dtype=dtype, with_grad=True, adjoint_budget_bytes=need // 4) as pl:
        assert pl.stats()["n_passes"] >= 4
        E2, dg2, db2 = pl.energy_grad(g, b)
        zz2, E3 = pl.energy(g, b)
    tol = 1e-10 if dtype == "c128" else 1e-5
    assert abs(E2[0] - E[0]) <= tol * abs(E[0]) and abs(E3 - E[0]) <= tol * abs(E[0])
    np.testing.assert_allclose(zz2, zz, atol=tol)
    np.testing.assert_allclose(dg2, dg, atol=10 * tol)
    np.testing.assert_allclose(db2, db, atol=10 * tol)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_merged_gradient_plans_match_the_oracle(dtype):
    """Gradient plans with merged eliminations (opt-in): the reverse sweep
    through merged buckets against the N=50 p=4 sampled-edge central
    differences and the N=20 p=4 parameter-shift golden."""
    rows = _golden_rows("c5_n50_p4_fd.txt")
    n, p = 50, 4
    edges = synth.random_regular_graph(n, 1000)
    with qtgb.plan_subset(n, edges, p, rows["edges"].astype(np.int32), dtype=dtype, with_grad=True,
                          merge=True) as pl:
        B, _ = pl.export()
        E, dg, db = pl.energy_grad(rows["gamma"], rows["beta"])
    assert (B["n_sum"] > 1).any()
    ref = np.concatenate([rows["dE_dgamma"], rows["dE_dbeta"]])
    tol = 1e-6 if dtype == "c128" else 1e-4 * np.abs(ref).max()
    assert np.abs(np.concatenate([dg, db]) - ref).max() <= tol
    g20 = _golden_grad()
    edges20 = synth.random_regular_graph(20, 1020)
    with grad_plan(20, edges20, 4, dtype=dtype, merge=True) as pl:
        E, dg, db = pl.energy_grad(g20["gamma"], g20["beta"])
    ref = np.concatenate([g20["dE_dgamma"], g20["dE_dbeta"]])
    tol = 1e-8 if dtype == "c128" else 1e-4 * np.abs(ref).max()
    assert np.abs(np.concatenate([dg, db]) - ref).max() <= tol


def test_gradient_passes_split_a_network_by_slice():
    """A budget below one network's whole arena but above each of its slices:
    the network's slices land in several passes, each seeding its slices from
    their own factors; energy and gradient equal the unbudgeted plan's."""
    n, p = 30, 4
    edges = synth.random_regular_graph(n, 1000)
    g, b = synth.angles(p, 1000)
    kw = dict(dtype="c128", with_grad=True, slice_width=16)
    with qtgb.plan(n, edges, p, **kw) as pl:
        E, dg, db = pl.energy_grad(g, b)
        need = pl.stats()["arena_bytes"]
    with qtgb.plan(n, edges, p, adjoint_budget_bytes=need // 40, **kw) as pl:
        parts = [set(e.tolist()) for _, e in pl.passes()]
        E2, dg2, db2 = pl.energy_grad(g, b)
    split = [e for e in range(edges.shape[0]) if sum(e in s for s in parts) > 1]
    assert len(parts) > 1 and split, "no network's slices were split over passes"
    assert abs(E2[0] - E[0]) <= 1e-10 * abs(E[0])
    np.testing.assert_allclose(dg2, dg, atol=1e-9)
    np.testing.assert_allclose(db2, db, atol=1e-9)
