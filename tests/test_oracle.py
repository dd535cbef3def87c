"""Pins for the CPU oracle against facts other than itself.

* the published p=1 closed form (any graph, triangles included);
* a dense 2^N matrix exponential from scipy (any depth, small N);
* the paper's 0.6924 per-edge optimum at p=1 on 3-regular graphs (§II-A);
* invariants of the QAOA state (γ=β=0, β=0, periodicity, |e| <= 1);
* brute force over all assignments of a network (the definition of a
  contraction) against bucket elimination, and bucket elimination under two
  different orders;
* lightcone shape: 2(p - d) + 1 variables on a qubit at distance d <= p;
* gradients: parameter shift against finite differences and against the
  derivative of the closed form; the closed-form derivative against finite
  differences of the closed form.
A final group plants plausible mistakes in the oracle's inputs and checks that
the pins above would catch them.
"""
import math
from pathlib import Path

import networkx as nx
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2204_06045_gb300 import synth

GOLDEN = Path(__file__).parent / "golden"

SMALL_GRAPHS = {
    "petersen": (10, synth.petersen_graph()),
    "K4": (4, synth.complete_graph(4)),
    "prism": (6, synth.prism_graph()),
    "ring7": (7, synth.ring_graph(7)),
    "rr10": (10, synth.random_regular_graph(10, 1000)),
    "rr12": (12, synth.random_regular_graph(12, 1001)),
}


def _dense_zz(n, edges, gammas, betas):
    """<Z_a Z_b> from scipy's matrix exponential of the full Hamiltonians."""
    dim = 2 ** n
    z = np.arange(dim)
    spins = 1 - 2 * ((z[:, None] >> np.arange(n)[None, :]) & 1)
    hzz = np.zeros(dim)
    for a, b in edges:
        hzz += spins[:, a] * spins[:, b]
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    B = np.zeros((dim, dim), dtype=complex)
    for q in range(n):
        op = np.array([[1.0]], dtype=complex)
        for k in reversed(range(n)):  # qubit q is bit q of the index
            op = np.kron(op, X if k == q else np.eye(2))
        B += op
    psi = np.full(dim, 2 ** (-n / 2), dtype=complex)
    for g, b in zip(gammas, betas):
        psi = np.exp(-1j * g * hzz) * psi
        psi = scipy.linalg.expm(-1j * b * B) @ psi
    pr = np.abs(psi) ** 2
    return np.array([np.sum(pr * spins[:, a] * spins[:, b]) for a, b in edges])


@pytest.mark.parametrize("name", list(SMALL_GRAPHS))
@pytest.mark.parametrize("gb", [(0.37, 0.91), (2.9, 0.05), (1.1, 1.4), (-0.6, 0.3)])
def test_state_vector_matches_p1_closed_form(name, gb):
    n, edges = SMALL_GRAPHS[name]
    g, b = gb
    sv = oracle.sv_zz(n, edges, [g], [b])
    cf = oracle.p1_closed_form(n, edges, g, b)
    np.testing.assert_allclose(sv, cf, rtol=0, atol=1e-13)


@pytest.mark.parametrize("n,seed,p", [(6, 11, 2), (8, 12, 3), (8, 13, 4)])
def test_state_vector_matches_dense_expm(n, seed, p):
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    np.testing.assert_allclose(oracle.sv_zz(n, edges, g, b), _dense_zz(n, edges, g, b), rtol=0, atol=1e-12)


def test_ring_matches_dense_expm():
    n, edges = 6, synth.ring_graph(6)
    g, b = [0.4, 1.3], [0.2, 0.7]
    np.testing.assert_allclose(oracle.sv_zz(n, edges, g, b), _dense_zz(n, edges, g, b), rtol=0, atol=1e-12)


def _golden(name):
    vals = {}
    for line in (GOLDEN / name).read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_p1_triangle_free_optimum_is_paper_value():
    gold = _golden("p1_three_regular_optimum.txt")
    n, edges = SMALL_GRAPHS["petersen"]
    # optimum of <C_uv> = 1/2 - 1/2 sin4b sin2g cos^2 2g: sin4b = -1, sin2g = 1/sqrt3
    g = 0.5 * math.asin(1 / math.sqrt(3))
    b = 3 * math.pi / 8
    cut = (1 - oracle.sv_zz(n, edges, [g], [b])) / 2
    assert np.allclose(cut, 0.5 + 1 / (3 * math.sqrt(3)), atol=1e-13)
    scale = 10 ** int(gold["decimals"])
    assert math.floor(float(cut.min()) * scale) / scale == gold["ratio"]
    # no angle on a grid does better than the optimum
    best = 0.0
    for gg in np.linspace(0, math.pi, 41):
        for bb in np.linspace(0, math.pi / 2, 41):
            best = max(best, float(((1 - oracle.sv_zz(n, edges, [gg], [bb])) / 2).mean()))
    assert best <= 0.5 + 1 / (3 * math.sqrt(3)) + 1e-12
    assert best >= gold["ratio"] - 0.01


@pytest.mark.parametrize("p", [1, 2, 3])
def test_invariants(p):
    n, edges = 12, synth.random_regular_graph(12, 77)
    m = edges.shape[0]
    zero = np.zeros(p)
    assert np.abs(oracle.sv_zz(n, edges, zero, zero)).max() < 1e-14
    assert abs(oracle.sv_energy(n, edges, zero, zero) - m / 2) < 1e-12
    g, b = synth.angles(p, 77)
    assert np.abs(oracle.sv_zz(n, edges, g, zero)).max() < 1e-13  # beta = 0: diagonal evolution only
    zz = oracle.sv_zz(n, edges, g, b)
    assert np.all(np.abs(zz) <= 1 + 1e-12)
    E = oracle.energy_from_zz(zz)
    assert -1e-12 <= E <= m + 1e-12
    np.testing.assert_allclose(oracle.sv_zz(n, edges, g + math.pi, b), zz, atol=1e-12)
    np.testing.assert_allclose(oracle.sv_zz(n, edges, g, b + math.pi), zz, atol=1e-12)


@pytest.mark.parametrize("name", ["petersen", "K4", "prism", "ring7", "rr10"])
@pytest.mark.parametrize("p", [1, 2])
def test_bucket_matches_brute_force(name, p):
    n, edges = SMALL_GRAPHS[name]
    g, b = synth.angles(p, 5)
    for e in range(min(edges.shape[0], 6)):
        nv, _, _ = oracle.edge_network_shape(n, edges, p, e)
        if nv > 24:
            continue
        ref = oracle.edge_brute(n, edges, g, b, e)
        val, _ = oracle.edge_bucket(n, edges, g, b, e, seed=e)
        assert abs(val - ref) < 1e-12


@pytest.mark.parametrize("n,seed,p", [(10, 1000, 1), (12, 21, 2), (14, 22, 3), (16, 23, 2)])
def test_bucket_matches_state_vector(n, seed, p):
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    vals, _ = oracle.bucket_zz(n, edges, g, b, seed=1)
    sv = oracle.sv_zz(n, edges, g, b)
    np.testing.assert_allclose(vals.real, sv, rtol=0, atol=1e-12)
    assert np.abs(vals.imag).max() < 1e-12


def test_bucket_order_independence():
    n, edges = 16, synth.random_regular_graph(16, 31)
    g, b = synth.angles(3, 31)
    a, wa = oracle.bucket_zz(n, edges, g, b, seed=1)
    c, wc = oracle.bucket_zz(n, edges, g, b, seed=12345)
    np.testing.assert_allclose(a, c, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n,seed,p", [(12, 21, 2), (14, 22, 3), (16, 23, 4)])
def test_min_fill_route_matches_state_vector_and_brute_force(n, seed, p):
    """The oracle's min-fill order (used for the N=1000 p=5 networks) gives the
    state vector's values, and brute force on a small network; its widths are
    no larger than the min-degree order's on these graphs' worst edge."""
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    sv = oracle.sv_zz(n, edges, g, b)
    for e in range(0, edges.shape[0], 3):
        val, w = oracle.edge_bucket_min_fill(n, edges, g, b, e, seed=e)
        assert abs(val.real - sv[e]) < 1e-12 and abs(val.imag) < 1e-12
    e = 0
    if p <= 2:
        assert abs(oracle.edge_bucket_min_fill(n, edges, g, b, e)[0] - oracle.edge_brute(n, edges, g, b, e)) < 1e-12


def test_min_fill_order_is_narrower_on_a_wide_network():
    """On an N=1000 p=5 lightcone the min-fill order stays within width 28
    where min-degree orders (three seeds) do not; the values agree with a
    second min-fill seed (order independence)."""
    n, p = 1000, 5
    edges = synth.random_regular_graph(n, 1000)
    g, b = synth.angles(p, 1000)
    e = 0  # a network of moderate width, cheap in every order
    v0, w0 = oracle.edge_bucket_min_fill(n, edges, g, b, e, seed=0)
    v1, w1 = oracle.edge_bucket_min_fill(n, edges, g, b, e, seed=7)
    vd, wd = oracle.edge_bucket(n, edges, g, b, e, seed=0, max_width=31)
    assert abs(v0 - v1) < 1e-12 and abs(v0 - vd) < 1e-12
    assert w0 <= wd


@pytest.mark.parametrize("p", [1, 2, 3])
def test_lightcone_shape(p):
    n, edges = 20, synth.random_regular_graph(20, 41)
    G = nx.Graph()
    G.add_edges_from(map(tuple, edges))
    for e in range(0, edges.shape[0], 5):
        j, k = map(int, edges[e])
        dj = nx.single_source_shortest_path_length(G, j)
        dk = nx.single_source_shortest_path_length(G, k)
        nv, nt, qv = oracle.edge_network_shape(n, edges, p, e)
        expect = np.zeros(n, dtype=int)
        for q in range(n):
            d = min(dj.get(q, 10 ** 9), dk.get(q, 10 ** 9))
            if d <= p:
                expect[q] = 2 * (p - d) + 1
        np.testing.assert_array_equal(qv, expect)
        assert nv == expect.sum()


def test_grad_param_shift_matches_finite_differences():
    n, edges = 8, synth.random_regular_graph(8, 3)
    g, b = synth.angles(2, 3)
    ps = oracle.grad_param_shift(n, edges, g, b)
    fd = oracle.grad_fd(lambda G, B: oracle.sv_energy(n, edges, G, B), g, b)
    np.testing.assert_allclose(ps[0], fd[0], atol=1e-7)
    np.testing.assert_allclose(ps[1], fd[1], atol=1e-7)


@pytest.mark.parametrize("name", ["petersen", "K4", "prism"])
def test_grad_param_shift_matches_closed_form_derivative(name):
    n, edges = SMALL_GRAPHS[name]
    for g, b in [(0.3, 0.7), (1.9, 0.2)]:
        ps = oracle.grad_param_shift(n, edges, [g], [b])
        cf = oracle.p1_closed_form_grad(n, edges, g, b)
        assert abs(ps[0][0] - cf[0]) < 1e-11
        assert abs(ps[1][0] - cf[1]) < 1e-11
        # the hand derivative against differences of the formula itself
        h = 1e-6
        Ecf = lambda gg, bb: oracle.energy_from_zz(oracle.p1_closed_form(n, edges, gg, bb))
        assert abs((Ecf(g + h, b) - Ecf(g - h, b)) / (2 * h) - cf[0]) < 1e-6
        assert abs((Ecf(g, b + h) - Ecf(g, b - h)) / (2 * h) - cf[1]) < 1e-6


def test_bucket_energy_finite_difference_matches_param_shift():
    n, edges = 10, synth.random_regular_graph(10, 8)
    g, b = synth.angles(2, 8)
    ps = oracle.grad_param_shift(n, edges, g, b)
    fd = oracle.grad_fd(lambda G, B: oracle.bucket_energy(n, edges, G, B), g, b)
    np.testing.assert_allclose(fd[0], ps[0], atol=1e-7)
    np.testing.assert_allclose(fd[1], ps[1], atol=1e-7)


# --- planted mistakes: each must break one of the pins above -------------------

def test_planted_wrong_mixer_sign_is_caught():
    n, edges = SMALL_GRAPHS["petersen"]
    g, b = 0.37, 0.91
    wrong = oracle.sv_zz(n, edges, [g], [-b])  # exp(+i b X) instead of exp(-i b X)
    assert np.abs(wrong - oracle.p1_closed_form(n, edges, g, b)).max() > 1e-3


def test_planted_wrong_gamma_scale_is_caught():
    n, edges = SMALL_GRAPHS["prism"]
    g, b = 0.37, 0.91
    wrong = oracle.sv_zz(n, edges, [g / 2], [b])  # exp(-i g/2 ZZ): the paper's C without rescaling
    assert np.abs(wrong - oracle.p1_closed_form(n, edges, g, b)).max() > 1e-3


def test_planted_dropped_zz_gate_is_caught():
    n, edges = 8, synth.random_regular_graph(8, 13)
    g, b = synth.angles(2, 13)
    za = np.repeat(g[:, None], edges.shape[0], axis=1)
    xa = np.repeat(b[:, None], n, axis=1)
    za[1, 3] = 0.0  # one ZZ gate of layer 2 missing
    wrong = oracle.sv_zz_gates(n, edges, za, xa)
    assert np.abs(wrong - _dense_zz(n, edges, g, b)).max() > 1e-4


# ---- contractions over binary indices (§II-E "tncontract") ------------------

@pytest.mark.parametrize("seed", range(6))
def test_contract_matches_brute_force_on_random_expressions(seed):
    """oracle.contract (one einsum) against the literal sum over every label
    assignment, on the paper's kind of random expression (4..7 indices)."""
    la, lb, lo = synth.tncontract_random(seed, n_lo=4, n_hi=7)
    A = synth.tensor_entries(len(la), 10 * seed)
    B = synth.tensor_entries(len(lb), 10 * seed + 1)
    np.testing.assert_allclose(oracle.contract([A, B], [la, lb], lo), oracle.contract_brute([A, B], [la, lb], lo),
                               rtol=0, atol=1e-12)


def test_contract_special_cases():
    """Closed forms: all-ones operands give 2^(summed labels) everywhere; a
    basis vector on one label selects a slice; a scalar output is the full
    sum; a permuted output is the transpose."""
    ones4, ones2 = np.ones((2,) * 4), np.ones((2,) * 2)
    # the paper's example shapes, dacb,ad->bcd: one label (a) summed
    out = oracle.contract([ones4, ones2], [[3, 0, 2, 1], [0, 3]], [1, 2, 3])
    assert out.shape == (2, 2, 2) and np.allclose(out, 2.0)
    out = oracle.contract([ones4, np.ones((2,) * 3)], [[2, 0, 4, 3], [4, 0, 3]], [2])  # three summed
    assert np.allclose(out, 8.0)
    A = synth.tensor_entries(4, 3)
    e1 = np.array([0.0, 1.0])
    np.testing.assert_allclose(oracle.contract([A, e1], [[0, 1, 2, 3], [1]], [0, 2, 3]), A[:, 1, :, :], atol=0)
    np.testing.assert_allclose(oracle.contract([A, np.ones(2)], [[0, 1, 2, 3], [0]], []), A.sum(), rtol=1e-14)
    np.testing.assert_allclose(oracle.contract([A, np.ones(2)], [[0, 1, 2, 3], [1]], [3, 0, 2]),
                               A.sum(axis=1).transpose(2, 0, 1), rtol=1e-14)


def test_planted_contraction_mistake_is_caught():
    """A planted mistake -- an output axis order swapped -- fails the brute force pin."""
    la, lb, lo = [0, 1, 2, 3], [1, 2], [0, 3]
    A, B = synth.tensor_entries(4, 8), synth.tensor_entries(2, 9)
    wrong = oracle.contract([A, B], [la, lb], lo[::-1])
    assert not np.allclose(wrong, oracle.contract_brute([A, B], [la, lb], lo), atol=1e-6)


def test_random_expressions_follow_the_paper_recipe():
    """synth.tncontract_random: 4..25 indices; the first tensor holds all of
    them, the second every contracted one, the result the rest; at least one
    index contracted and one kept."""
    for s in range(200):
        la, lb, lo = synth.tncontract_random(s)
        n = len(la)
        assert 4 <= n <= 25 and sorted(la) == list(range(n))
        summed = set(la) - set(lo)
        assert summed and lo and summed <= set(lb) and set(lb) <= set(la)
        assert len(set(lb)) == len(lb) and len(set(lo)) == len(lo)
