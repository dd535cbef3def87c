"""Write the stored expected values under tests/golden/ from the CPU oracle alone.

Usage: python tests/golden/make_golden.py [name ...]
Names: c2_sv (N=30 p=4 state vector, ~16 GiB of host memory, minutes),
       c5_grad (N=20 p=4 parameter-shift gradient), c5_bucket (N=50 p=4 bucket
       elimination at the seeded angles), c4_bucket (every edge of N=1000 p=5
       by bucket elimination in a min-fill order, ~minutes).
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


JOBS = {"c2_sv": c2_sv, "c5_grad": c5_grad, "c5_bucket": c5_bucket, "c4_bucket": c4_bucket}

if __name__ == "__main__":
    names = sys.argv[1:] or list(JOBS)
    for nm in names:
        t = time.time()
        JOBS[nm]()
        print(f"{nm}: {time.time() - t:.1f} s", flush=True)
