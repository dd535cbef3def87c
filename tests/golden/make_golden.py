"""Write the stored expected values under tests/golden/ from the CPU oracle alone.

Usage: python tests/golden/make_golden.py [name ...]
Names: c2_sv (N=30 p=4 state vector, ~16 GiB of host memory, minutes),
       c5_grad (N=20 p=4 parameter-shift gradient), c5_bucket (N=50 p=4 bucket
       elimination at the seeded angles), c4_bucket (every edge of N=1000 p=5
       by bucket elimination in a min-fill order, ~minutes), c5_fd (central
       differences of 8 sampled N=50 p=4 edges' share of the energy, bucket
       elimination), dedup_fd (the same for every edge of an N=60 p=2 graph
       whose lightcones repeat).
Each file records the seeds and the oracle route that produced it. Inputs come
from the seeded generators in ``paper_2204_06045_gb300.synth``; every value is
computed by ``oracle`` and nothing else.
"""
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_2204_06045_gb300 import synth  # noqa: E402

OUT = Path(__file__).resolve().parent


def _write(name, header, rows):
    with open(OUT / name, "w") as f:
        for h in header:
            f.write(f"# {h}\n")
        for r in rows:
            f.write(" ".join(r) + "\n")


def c2_sv():
    n, seed, p = 30, 1000, 4
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    t = time.time()
    zz = oracle.sv_zz(n, edges, g, b)
    dt = time.time() - t
    rows = [["gamma"] + [repr(float(x)) for x in g], ["beta"] + [repr(float(x)) for x in b]]
    rows += [["edge", str(e), str(int(edges[e, 0])), str(int(edges[e, 1])), repr(float(zz[e]))]
             for e in range(edges.shape[0])]
    rows.append(["energy", repr(oracle.energy_from_zz(zz))])
    _write("c2_n30_p4_statevector.txt",
           [f"Per-edge <Z_jZ_k> on the seeded random 3-regular graph N={n} (seed {seed}), p={p},",
            "angles from synth.angles(p, seed). Route: oracle.sv_zz, a 2^30 complex128 state vector",
            f"({oracle.get_threads()} threads, {dt:.0f} s). Written by tests/golden/make_golden.py c2_sv."],
           rows)


def c5_grad():
    n, seed, p = 20, 1020, 4
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    t = time.time()
    dg, db = oracle.grad_param_shift(n, edges, g, b)
    E = oracle.sv_energy(n, edges, g, b)
    dt = time.time() - t
    rows = [["gamma"] + [repr(float(x)) for x in g], ["beta"] + [repr(float(x)) for x in b],
            ["energy", repr(E)], ["dE_dgamma"] + [repr(float(x)) for x in dg],
            ["dE_dbeta"] + [repr(float(x)) for x in db]]
    _write("c5_n20_p4_gradient.txt",
           [f"Energy and gradient on the seeded random 3-regular graph N={n} (seed {seed}), p={p}.",
            "Route: oracle.grad_param_shift (exact parameter shift per gate on a 2^20 state vector)",
            f"({oracle.get_threads()} threads, {dt:.0f} s). Written by tests/golden/make_golden.py c5_grad."],
           rows)


def c5_bucket():
    n, seed, p = 50, 1000, 4
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    t = time.time()
    vals, w = oracle.bucket_zz(n, edges, g, b, seed=1, max_width=31)
    dt = time.time() - t
    rows = [["gamma"] + [repr(float(x)) for x in g], ["beta"] + [repr(float(x)) for x in b]]
    rows += [["edge", str(e), str(int(edges[e, 0])), str(int(edges[e, 1])), repr(float(vals[e].real)),
              repr(float(vals[e].imag))] for e in range(edges.shape[0])]
    rows.append(["energy", repr(oracle.energy_from_zz(vals.real))])
    _write("c5_n50_p4_bucket.txt",
           [f"Per-edge network values on the seeded random 3-regular graph N={n} (seed {seed}), p={p}.",
            f"Route: oracle.bucket_zz (complex128 bucket elimination, min-degree order, max width {w})",
            f"({oracle.get_threads()} threads, {dt:.0f} s). Written by tests/golden/make_golden.py c5_bucket."],
           rows)


def c4_bucket():
    """Every edge of the N=1000 p=5 graph (the wide-bucket workload picks its
    networks among them): complex128 bucket elimination in the oracle's own
    greedy min-fill order, seed = edge index (next seeds if a bucket would be
    wider than 28)."""
    n, seed, p = 1000, 1000, 5
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    t = time.time()
    rows = [["gamma"] + [repr(float(x)) for x in g], ["beta"] + [repr(float(x)) for x in b]]
    vals = []
    for e in range(edges.shape[0]):
        for s in range(e, e + 5000, 1000):
            try:
                v, w = oracle.edge_bucket_min_fill(n, edges, g, b, e, seed=s, max_width=28)
                break
            except RuntimeError:
                continue
        else:
            raise RuntimeError(f"edge {e}: no min-fill order within width 28")
        vals.append(v.real)
        rows.append(["edge", str(e), str(int(edges[e, 0])), str(int(edges[e, 1])), repr(float(v.real)),
                     repr(float(v.imag)), str(w), str(s)])
    dt = time.time() - t
    rows.append(["energy", repr(oracle.energy_from_zz(np.array(vals)))])
    _write("c4_n1000_p5_bucket.txt",
           [f"Per-edge network values on the seeded random 3-regular graph N={n} (seed {seed}), p={p}.",
            "Route: oracle.edge_bucket_min_fill (complex128 bucket elimination, the oracle's greedy",
            "min-fill order with random ties); columns: edge, j, k, Re, Im, max width, order seed",
            f"({oracle.get_threads()} threads, {dt:.0f} s). Written by tests/golden/make_golden.py c4_bucket."],
           rows)


def _fd_share(n, edges, g, b, sel, h):
    """Energy share E_S = |S|/2 - 1/2 sum_{e in S} <Z_jZ_k> of the edges in S and its
    central differences (step h) in every angle; each <Z_jZ_k> by the oracle's
    bucket elimination in its own min-fill order (route 2, complex128)."""
    def E(gg, bb):
        s = 0.0
        for e in sel:
            v, _ = oracle.edge_bucket_min_fill(n, edges, gg, bb, int(e), seed=int(e), max_width=30)
            s += v.real
        return 0.5 * len(sel) - 0.5 * s
    dg, db = oracle.grad_fd(E, g, b, h=h)
    return E(g, b), dg, db


def _write_fd(name, header, n, edges, g, b, sel, h):
    t = time.time()
    E, dg, db = _fd_share(n, edges, g, b, sel, h)
    dt = time.time() - t
    rows = [["gamma"] + [repr(float(x)) for x in g], ["beta"] + [repr(float(x)) for x in b],
            ["edges"] + [str(int(e)) for e in sel], ["h", repr(h)], ["energy", repr(E)],
            ["dE_dgamma"] + [repr(float(x)) for x in dg], ["dE_dbeta"] + [repr(float(x)) for x in db]]
    _write(name, header + [f"({oracle.get_threads()} threads, {dt:.0f} s). Written by tests/golden/make_golden.py."],
           rows)


def c5_fd():
    """N=50 p=4 (seed 1000): 8 edges drawn by PCG64(5050) without replacement."""
    n, seed, p = 50, 1000, 4
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    sel = np.sort(np.random.default_rng(5050).choice(edges.shape[0], size=8, replace=False))
    _write_fd("c5_n50_p4_fd.txt",
              [f"Energy share of 8 sampled edges and its angle derivatives on the seeded random 3-regular graph",
               f"N={n} (seed {seed}), p={p}, angles synth.angles(p, seed); edges drawn by numpy PCG64(5050).",
               "E_S = |S|/2 - 1/2 sum_{e in S} <Z_jZ_k>; derivatives by central differences (step h) of E_S,",
               "every <Z_jZ_k> by oracle.edge_bucket_min_fill (complex128 bucket elimination, route 2)"],
              n, edges, g, b, sel, 1e-5)


def dedup_fd():
    """N=60 p=2 (seed 3), every edge: a graph whose lightcones repeat."""
    n, seed, p = 60, 3, 2
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    _write_fd("dedup_n60_p2_fd.txt",
              [f"Energy and angle derivatives on the seeded random 3-regular graph N={n} (seed {seed}), p={p},",
               "angles synth.angles(p, seed); many of its lightcones are isomorphic. Derivatives by central",
               "differences (step h) of E, every <Z_jZ_k> by oracle.edge_bucket_min_fill (route 2)"],
              n, edges, g, b, np.arange(edges.shape[0]), 1e-5)


JOBS = {"c2_sv": c2_sv, "c5_grad": c5_grad, "c5_bucket": c5_bucket, "c4_bucket": c4_bucket, "c5_fd": c5_fd,
        "dedup_fd": dedup_fd}

if __name__ == "__main__":
    names = sys.argv[1:] or list(JOBS)
    for nm in names:
        t = time.time()
        JOBS[nm]()
        print(f"{nm}: {time.time() - t:.1f} s", flush=True)
