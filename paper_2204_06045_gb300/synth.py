"""Seeded synthetic inputs: random 3-regular graphs and QAOA angles.

This module only draws inputs. It holds none of the method's arithmetic, so the
CPU oracle (under ``oracle/``) and the CUDA path can both be fed from it without
sharing any computation.

The paper evaluates QAOA MaxCut on random 3-regular graphs (§II-E "Circuit
Simulation", §III-A: a 3-regular graph of 30 vertices at depth p=4). It does not
say how the graphs or angles are drawn, so the recipe is fixed here:

* Graph with seed ``s``: the configuration (pairing) model on ``numpy``'s
  ``Generator(PCG64(s))``. The 3·N vertex stubs are shuffled with one
  ``permutation`` call and paired consecutively; a draw with a self-loop or a
  repeated edge is rejected and the next permutation of the same generator is
  taken. Edges are returned as sorted ``(min, max)`` pairs in lexicographic
  order.
* Angles for a graph with seed ``s``: ``Generator(PCG64(s + 1))``; first
  ``gamma_1..gamma_p ~ U(0, pi)``, then ``beta_1..beta_p ~ U(0, pi/2)``.
* Batches of graphs: vertex counts drawn once from ``Generator(PCG64(7))``
  (even integers, uniform in ``[lo, hi]``); graph ``g`` then uses seed
  ``base_seed + g``.
* Random contraction expressions (the paper's "tncontract random", §II-E and
  §III-E: every index of size 2, 4 to 25 indices): ``Generator(PCG64(s))``
  draws the number of indices n, then the number m of contracted indices
  (1..n-1), then how many of the n - m result indices the second tensor also
  holds; the first tensor holds all n indices in a random order, the second
  the m contracted ones and those result indices in a random order, and the
  result the n - m uncontracted indices in a random order (e.g. the paper's
  ``dacb,ad->bcd``). Tensor entries are complex normal draws of a second
  generator.
"""
from __future__ import annotations

import numpy as np


def random_regular_graph(n: int, seed: int, degree: int = 3) -> np.ndarray:
    """Return an (m, 2) int32 array of edges of a simple random ``degree``-regular graph."""
    if n <= degree or (n * degree) % 2:
        raise ValueError(f"no simple {degree}-regular graph on {n} vertices")
    rng = np.random.Generator(np.random.PCG64(seed))
    stubs = np.repeat(np.arange(n, dtype=np.int64), degree)
    for _ in range(100000):
        perm = stubs[rng.permutation(stubs.size)]
        a, b = perm[0::2], perm[1::2]
        if np.any(a == b):
            continue
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        keys = lo * n + hi
        if np.unique(keys).size != keys.size:
            continue
        order = np.argsort(keys)
        return np.stack([lo[order], hi[order]], axis=1).astype(np.int32)
    raise RuntimeError("pairing model did not produce a simple graph")


def angles(p: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Return ``(gammas, betas)``, each float64 of length ``p``, for graph seed ``seed``."""
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    gammas = rng.uniform(0.0, np.pi, size=p)
    betas = rng.uniform(0.0, np.pi / 2, size=p)
    return gammas, betas


def batch_sizes(n_graphs: int, lo: int = 50, hi: int = 1000, seed: int = 7) -> np.ndarray:
    """Even vertex counts uniform in ``[lo, hi]`` for a batch of graphs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    half = rng.integers(lo // 2, hi // 2 + 1, size=n_graphs)
    return (2 * half).astype(np.int32)


def batch(n_graphs: int, p: int, lo: int = 50, hi: int = 1000, base_seed: int = 1000):
    """A batch of graphs with per-graph angles: list of ``(n, edges, gammas, betas)``."""
    out = []
    for g, n in enumerate(batch_sizes(n_graphs, lo, hi)):
        edges = random_regular_graph(int(n), base_seed + g)
        gam, bet = angles(p, base_seed + g)
        out.append((int(n), edges, gam, bet))
    return out


def ring_graph(n: int) -> np.ndarray:
    """Cycle C_n (2-regular), a hand-checkable small case."""
    return np.array([(min(i, (i + 1) % n), max(i, (i + 1) % n)) for i in range(n)], dtype=np.int32)


def petersen_graph() -> np.ndarray:
    """The Petersen graph: 3-regular, 10 vertices, girth 5 (triangle-free)."""
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    e = [(min(a, b), max(a, b)) for a, b in outer + spokes + inner]
    return np.array(sorted(e), dtype=np.int32)


def complete_graph(n: int) -> np.ndarray:
    """K_n; K_4 is the smallest 3-regular graph and is full of triangles."""
    return np.array([(a, b) for a in range(n) for b in range(a + 1, n)], dtype=np.int32)


def prism_graph() -> np.ndarray:
    """Triangular prism: 3-regular on 6 vertices with two triangles."""
    e = [(0, 1), (1, 2), (0, 2), (3, 4), (4, 5), (3, 5), (0, 3), (1, 4), (2, 5)]
    return np.array(sorted(e), dtype=np.int32)


def tncontract_random(seed: int, n_lo: int = 4, n_hi: int = 25):
    """One random contraction expression: ``(labels_a, labels_b, labels_out)``, each a list of
    int labels in C order (first label the slowest axis), labels ``0..n-1``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(rng.integers(n_lo, n_hi + 1))
    m = int(rng.integers(1, n))  # contracted indices, at least one result index left
    idx = rng.permutation(n)
    summed, result = idx[:m], idx[m:]
    k = int(rng.integers(0, result.size + 1))  # result indices the second tensor holds too
    b = np.concatenate([summed, rng.permutation(result)[:k]])
    return ([int(x) for x in rng.permutation(n)], [int(x) for x in rng.permutation(b)],
            [int(x) for x in rng.permutation(result)])


def tensor_entries(shape_rank: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """Complex normal entries for a tensor of ``shape_rank`` indices of size 2 (shape 2 x ... x 2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal((2, 1 << shape_rank))
    return (v[0] + 1j * v[1]).astype(dtype).reshape((2,) * shape_rank)
