"""CPU oracle for QAOA MaxCut edge expectations, complex128.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. Nothing here is imported
by the product package, and nothing here imports it.

Routes (each a plain implementation of the paper's definitions):

* ``sv_zz`` / ``sv_zz_gates`` -- state vector over 2^N amplitudes (Eq. 2).
* ``edge_bucket`` / ``bucket_zz`` -- bucket elimination of each edge's
  lightcone network (§II-B) with the C library's own network builder and a
  min-degree order with random ties.
* ``edge_brute`` -- the sum over every variable assignment of one network.
* ``p1_closed_form`` -- the published p=1 formula (Wang, Hadfield, Jiang and
  Rieffel, Phys. Rev. A 97, 022304 (2018)) rewritten in this gate convention.
* ``grad_param_shift`` / ``grad_fd`` -- gradients of the energy.
* ``contract`` / ``contract_brute`` -- a contraction of tensors over binary
  indices (the paper's "tncontract" expressions, §II-E): out[K] = the sum over
  the labels not in K of the product of the operands.

Gate convention: layer k applies ``exp(-i gamma_k s_a s_b)`` on every edge,
then ``exp(-i beta_k X)`` on every qubit, from |+>^N, with ``s(x) = 1 - 2x``.
The paper's Eq. 2 writes ``exp(-i gamma C)`` with ``C = 1/2 sum (1 - Z Z)``;
that is this convention with ``gamma_paper = -2 gamma`` (up to a global
phase).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_LIB_PATH = _HERE / "liboracle.so"
_lib = None

OR_OK, OR_EINVAL, OR_ENOMEM, OR_ETOOBIG = 0, -1, -2, -3


def build(force: bool = False) -> Path:
    """Compile ``liboracle.so`` with gcc (C11, OpenMP)."""
    src = _HERE / "oracle.c"
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < src.stat().st_mtime:
        tmp = _LIB_PATH.with_suffix(f".{os.getpid()}.tmp.so")
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall",
               "-o", str(tmp), str(src), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(str(_LIB_PATH))
        i32p = ctypes.POINTER(ctypes.c_int32)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        c_int, u64 = ctypes.c_int, ctypes.c_uint64
        lib.oracle_sv_zz.argtypes = [c_int, c_int, i32p, c_int, dp, dp, dp]
        lib.oracle_sv_zz_gates.argtypes = [c_int, c_int, i32p, c_int, dp, dp, dp]
        lib.oracle_edge_bucket.argtypes = [c_int, c_int, i32p, c_int, dp, dp, c_int, u64, c_int, dp, ip]
        lib.oracle_bucket_zz.argtypes = [c_int, c_int, i32p, c_int, dp, dp, u64, c_int, dp, ip]
        lib.oracle_edge_brute.argtypes = [c_int, c_int, i32p, c_int, dp, dp, c_int, dp]
        lib.oracle_edge_network_shape.argtypes = [c_int, c_int, i32p, c_int, c_int, ip, ip, ip]
        lib.oracle_edge_bucket_order.argtypes = [c_int, c_int, i32p, c_int, dp, dp, c_int, c_int, u64, c_int, dp, ip]
        lib.oracle_set_threads.argtypes = [c_int]
        lib.oracle_get_threads.restype = c_int
        for f in (lib.oracle_sv_zz, lib.oracle_sv_zz_gates, lib.oracle_edge_bucket,
                  lib.oracle_bucket_zz, lib.oracle_edge_brute, lib.oracle_edge_network_shape,
                  lib.oracle_edge_bucket_order):
            f.restype = c_int
        _lib = lib
    return _lib


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc: int, what: str):
    if rc != OR_OK:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


# --------------------------------------------------------------------------
# Route 1: state vector (Eq. 2)
# --------------------------------------------------------------------------

def sv_zz(n: int, edges, gammas, betas) -> np.ndarray:
    """Per-edge <Z_a Z_b> of the depth-p QAOA state, by state vector."""
    lib = _load()
    e, ep = _i32(edges)
    g, gp = _f64(gammas)
    b, bp = _f64(betas)
    out = np.zeros(e.shape[0], dtype=np.float64)
    _check(lib.oracle_sv_zz(n, e.shape[0], ep, g.size, gp, bp,
                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "sv_zz")
    return out


def sv_zz_gates(n: int, edges, zz_angles, x_angles) -> np.ndarray:
    """Per-edge <Z_a Z_b> with one angle per gate: ``zz_angles`` (p, m), ``x_angles`` (p, n)."""
    lib = _load()
    e, ep = _i32(edges)
    za, zap = _f64(zz_angles)
    xa, xap = _f64(x_angles)
    p = za.shape[0]
    assert za.shape == (p, e.shape[0]) and xa.shape == (p, n)
    out = np.zeros(e.shape[0], dtype=np.float64)
    _check(lib.oracle_sv_zz_gates(n, e.shape[0], ep, p, zap, xap,
                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "sv_zz_gates")
    return out


# --------------------------------------------------------------------------
# Routes 2 and 3: lightcone networks (§II-B)
# --------------------------------------------------------------------------

def edge_bucket(n: int, edges, gammas, betas, eidx: int, seed: int = 0, max_width: int = 30):
    """(value, max bucket width) of edge ``eidx``'s network by bucket elimination."""
    lib = _load()
    e, ep = _i32(edges)
    g, gp = _f64(gammas)
    b, bp = _f64(betas)
    out = np.zeros(2, dtype=np.float64)
    w = ctypes.c_int(0)
    _check(lib.oracle_edge_bucket(n, e.shape[0], ep, g.size, gp, bp, int(eidx), int(seed), int(max_width),
                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(w)),
           "edge_bucket")
    return complex(out[0], out[1]), int(w.value)


def edge_bucket_min_fill(n: int, edges, gammas, betas, eidx: int, seed: int = 0, max_width: int = 30):
    """(value, max bucket width) of edge ``eidx``'s network, eliminated in a greedy
    min-fill order with random ties (the oracle's own, for networks whose
    min-degree orders are too wide)."""
    lib = _load()
    e, ep = _i32(edges)
    g, gp = _f64(gammas)
    b, bp = _f64(betas)
    out = np.zeros(2, dtype=np.float64)
    w = ctypes.c_int(0)
    _check(lib.oracle_edge_bucket_order(n, e.shape[0], ep, g.size, gp, bp, int(eidx), 1, int(seed), int(max_width),
                                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(w)),
           "edge_bucket_min_fill")
    return complex(out[0], out[1]), int(w.value)


def bucket_zz(n: int, edges, gammas, betas, seed: int = 0, max_width: int = 30):
    """(complex values of every edge's network, max bucket width) by bucket elimination."""
    lib = _load()
    e, ep = _i32(edges)
    g, gp = _f64(gammas)
    b, bp = _f64(betas)
    out = np.zeros(2 * e.shape[0], dtype=np.float64)
    w = ctypes.c_int(0)
    _check(lib.oracle_bucket_zz(n, e.shape[0], ep, g.size, gp, bp, int(seed), int(max_width),
                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(w)),
           "bucket_zz")
    return out[0::2] + 1j * out[1::2], int(w.value)


def edge_brute(n: int, edges, gammas, betas, eidx: int) -> complex:
    """Value of edge ``eidx``'s network as the sum over every variable assignment."""
    lib = _load()
    e, ep = _i32(edges)
    g, gp = _f64(gammas)
    b, bp = _f64(betas)
    out = np.zeros(2, dtype=np.float64)
    _check(lib.oracle_edge_brute(n, e.shape[0], ep, g.size, gp, bp, int(eidx),
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "edge_brute")
    return complex(out[0], out[1])


def edge_network_shape(n: int, edges, p: int, eidx: int):
    """(variables, tensors, variables per qubit wire) of edge ``eidx``'s network."""
    lib = _load()
    e, ep = _i32(edges)
    nv, nt = ctypes.c_int(0), ctypes.c_int(0)
    qv = np.zeros(n, dtype=np.int32)
    _check(lib.oracle_edge_network_shape(n, e.shape[0], ep, int(p), int(eidx), ctypes.byref(nv),
                                         ctypes.byref(nt), qv.ctypes.data_as(ctypes.POINTER(ctypes.c_int))),
           "edge_network_shape")
    return int(nv.value), int(nt.value), qv


# --------------------------------------------------------------------------
# Energy (§II-B edge decomposition)
# --------------------------------------------------------------------------

def energy_from_zz(zz) -> float:
    """<C> = |E|/2 - 1/2 sum_jk e_jk, summed in edge order in float64."""
    zz = np.asarray(zz, dtype=np.float64)
    s = 0.0
    for v in zz:
        s += float(v)
    return 0.5 * zz.size - 0.5 * s


def sv_energy(n: int, edges, gammas, betas) -> float:
    return energy_from_zz(sv_zz(n, edges, gammas, betas))


def bucket_energy(n: int, edges, gammas, betas, seed: int = 0) -> float:
    vals, _ = bucket_zz(n, edges, gammas, betas, seed)
    return energy_from_zz(vals.real)


# --------------------------------------------------------------------------
# Route 4: closed form at p = 1
# --------------------------------------------------------------------------

def _p1_terms(n: int, edges):
    edges = np.asarray(edges)
    deg = np.zeros(n, dtype=np.int64)
    nbr = [set() for _ in range(n)]
    for a, b in edges:
        deg[a] += 1
        deg[b] += 1
        nbr[a].add(int(b))
        nbr[b].add(int(a))
    out = []
    for a, b in edges:
        out.append((int(deg[a] - 1), int(deg[b] - 1), len(nbr[a] & nbr[b])))
    return out


def p1_closed_form(n: int, edges, gamma: float, beta: float) -> np.ndarray:
    """Per-edge <Z_u Z_v> at p=1 from the published closed form.

    With g = gamma_paper = -2*gamma, d = deg(u)-1, e = deg(v)-1 and f the number
    of triangles on (u, v):
      <C_uv> = 1/2 + 1/4 sin(4b) sin(g) (cos^d g + cos^e g)
               - 1/4 sin^2(2b) cos^(d+e-2f)(g) (1 - cos^f(2g)),
    and <Z_u Z_v> = 1 - 2 <C_uv>.
    """
    g = -2.0 * gamma
    out = []
    for d, e, f in _p1_terms(n, edges):
        c = (0.5 + 0.25 * math.sin(4 * beta) * math.sin(g) * (math.cos(g) ** d + math.cos(g) ** e)
             - 0.25 * math.sin(2 * beta) ** 2 * math.cos(g) ** (d + e - 2 * f) * (1 - math.cos(2 * g) ** f))
        out.append(1.0 - 2.0 * c)
    return np.array(out)


def p1_closed_form_grad(n: int, edges, gamma: float, beta: float):
    """(dE/dgamma, dE/dbeta) of the p=1 energy, differentiating the closed form by hand.

    E = sum_uv <C_uv>; with g = -2 gamma, d/dgamma = -2 d/dg.
    """
    g = -2.0 * gamma
    sg, cg = math.sin(g), math.cos(g)
    s4, c4 = math.sin(4 * beta), math.cos(4 * beta)
    s2b = math.sin(2 * beta)
    c2g, s2g = math.cos(2 * g), math.sin(2 * g)

    def powd(x, k):  # d/dx x^k
        return k * x ** (k - 1) if k > 0 else 0.0

    dE_dg = 0.0
    dE_db = 0.0
    for d, e, f in _p1_terms(n, edges):
        A = cg ** d + cg ** e
        dA_dg = (powd(cg, d) + powd(cg, e)) * (-sg)
        r = d + e - 2 * f
        Bc = cg ** r
        dBc_dg = powd(cg, r) * (-sg)
        F = 1 - c2g ** f
        dF_dg = -powd(c2g, f) * (-2 * s2g)
        # <C> = 1/2 + 1/4 s4 sg A - 1/4 s2b^2 Bc F
        dE_dg += 0.25 * s4 * (cg * A + sg * dA_dg) - 0.25 * s2b ** 2 * (dBc_dg * F + Bc * dF_dg)
        dE_db += 0.25 * (4 * c4) * sg * A - 0.25 * (2 * s2b * 2 * math.cos(2 * beta)) * Bc * F
    return -2.0 * dE_dg, dE_db


# --------------------------------------------------------------------------
# Gradients
# --------------------------------------------------------------------------

def grad_param_shift(n: int, edges, gammas, betas):
    """(dE/dgamma, dE/dbeta) by the parameter-shift rule on the state vector.

    Every gate is exp(-i theta G) with G^2 = I, so the energy restricted to one
    gate's angle is a + b cos 2theta + c sin 2theta and its derivative is
    exactly E(theta + pi/4) - E(theta - pi/4). dE/dgamma_k sums this over the
    |E| ZZ gates of layer k, dE/dbeta_k over the N mixers of layer k.
    """
    edges = np.asarray(edges, dtype=np.int32)
    m = edges.shape[0]
    p = len(gammas)
    za = np.repeat(np.asarray(gammas, dtype=np.float64)[:, None], m, axis=1)
    xa = np.repeat(np.asarray(betas, dtype=np.float64)[:, None], n, axis=1)

    def E(z, x):
        return energy_from_zz(sv_zz_gates(n, edges, z, x))

    dg = np.zeros(p)
    db = np.zeros(p)
    s = math.pi / 4
    for k in range(p):
        for e in range(m):
            zp, zm = za.copy(), za.copy()
            zp[k, e] += s
            zm[k, e] -= s
            dg[k] += E(zp, xa) - E(zm, xa)
        for q in range(n):
            xp, xm = xa.copy(), xa.copy()
            xp[k, q] += s
            xm[k, q] -= s
            db[k] += E(za, xp) - E(za, xm)
    return dg, db


def grad_fd(energy_fn, gammas, betas, h: float = 1e-5):
    """Central finite differences of ``energy_fn(gammas, betas)``."""
    gammas = np.asarray(gammas, dtype=np.float64)
    betas = np.asarray(betas, dtype=np.float64)
    p = gammas.size
    dg, db = np.zeros(p), np.zeros(p)
    for k in range(p):
        gp, gm = gammas.copy(), gammas.copy()
        gp[k] += h
        gm[k] -= h
        dg[k] = (energy_fn(gp, betas) - energy_fn(gm, betas)) / (2 * h)
        bp, bm = betas.copy(), betas.copy()
        bp[k] += h
        bm[k] -= h
        db[k] = (energy_fn(gammas, bp) - energy_fn(gammas, bm)) / (2 * h)
    return dg, db


# --------------------------------------------------------------------------
# Contractions over binary indices (§II-E, "tncontract")
# --------------------------------------------------------------------------

_SUBSCRIPTS = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"


def contract(ops, labels, out_labels) -> np.ndarray:
    """out[K] = sum over the labels not in K of prod_t ops[t][L_t], in complex128.

    ``ops[t]`` has one axis of size 2 per label of ``labels[t]`` (C order);
    the result has one per label of ``out_labels``. numpy's einsum does the
    sum of products, the definition written as one expression."""
    names = {}
    for L in list(labels) + [out_labels]:
        for x in L:
            names.setdefault(int(x), _SUBSCRIPTS[len(names)])
    spec = ",".join("".join(names[int(x)] for x in L) for L in labels) + "->" + "".join(
        names[int(x)] for x in out_labels)
    return np.einsum(spec, *[np.asarray(o, dtype=np.complex128) for o in ops], optimize=False)


def contract_brute(ops, labels, out_labels) -> np.ndarray:
    """The same sum as ``contract`` by explicit loops over every assignment of
    the labels (small expressions only): the literal definition."""
    alls = sorted({int(x) for L in labels for x in L})
    out = np.zeros((2,) * len(out_labels), dtype=np.complex128)
    for a in range(1 << len(alls)):
        val = {lab: (a >> i) & 1 for i, lab in enumerate(alls)}
        prod = 1.0 + 0.0j
        for o, L in zip(ops, labels):
            prod *= complex(np.asarray(o)[tuple(val[int(x)] for x in L)])
        out[tuple(val[int(x)] for x in out_labels)] += prod
    return out
