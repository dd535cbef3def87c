"""Test-side numpy emulation of the device data flow of a plan.

From the arrays the kernels read (qt_plan_export_device): the arena's gate
table is written here from the gates' definitions (Eq. 2, as plan_eval does),
every bucket is contracted from arena offsets in plan order with the kernels'
documented indexing, and the epilogue is formed from the factor lists. Tiles,
staging, gate-table folding and fused units are left out: those are how the
kernels compute the same values. This checks, without a GPU, the layout the
kernels consume: operand offsets (slices included), masks over the tile
outputs (merged buckets included), operands without the summed variable, the
merged pair sums, the factor lists and the energy's owned halves.
"""
import numpy as np

from plan_eval import leaf_tensor, pext

FIRST = np.uint64(1) << np.uint64(63)


def _slot_kind(slot):
    """(kind, layer) of leaf slot `slot`: 0 |+>, 1 Z, then per layer ZZ, ZZ*, mixer, mixer*."""
    if slot < 2:
        return slot, -1
    return 2 + (slot - 2) % 4, (slot - 2) // 4


def emulate(pl, gammas, betas, p):
    """(per-network complex values, per-graph energies) of plan `pl`."""
    B, O, nff, F, GO = pl.export_device()
    G = len(GO)
    gam = np.atleast_2d(np.asarray(gammas, dtype=np.float64))
    bet = np.atleast_2d(np.asarray(betas, dtype=np.float64))
    L = 2 + 4 * p
    res_end = [int(b["out_off"]) + (1 << (int(b["n_out"]) + 1 - int(b["n_sum"]))) for b in B]
    size = max([G * L * 4] + res_end) + 4
    arena = np.zeros(size, dtype=complex)
    for g in range(G):
        for slot in range(L):
            kind, layer = _slot_kind(slot)
            arena[(g * L + slot) * 4:(g * L + slot) * 4 + 4] = leaf_tensor(kind, layer, gam[g], bet[g])
    for b in B:
        n = int(b["n_out"])
        o = np.arange(1 << n, dtype=np.int64)
        acc = np.zeros(1 << n, dtype=complex)
        for x in (0, 1):
            prod = np.ones(1 << n, dtype=complex)
            for t in range(int(b["op_begin"]), int(b["op_begin"]) + int(b["n_ops"])):
                op = O[t]
                j = pext(o, int(op["mask"]))
                idx = int(op["off"]) + (2 * j + x if op["pairs_x"] else j)
                prod = prod * arena[idx]
            acc += prod
        m = int(b["n_sum"]) - 1
        if m:  # outputs (o, s2, s1), s1 as bit 0 and s2 as bit 1: add the groups of 2^m
            acc = acc.reshape(-1, 1 << m).sum(axis=1)
        arena[int(b["out_off"]):int(b["out_off"]) + acc.size] = acc
    n_nets = nff.size - 1
    vals = np.zeros(n_nets, dtype=complex)
    for net in range(n_nets):
        total, prod = 0.0 + 0j, None
        for f in F[nff[net]:nff[net + 1]]:
            if (f & FIRST) and prod is not None:
                total += prod
                prod = None
            v = arena[int(f & ~FIRST)]
            prod = v if prod is None else prod * v
        vals[net] = total + (prod if prod is not None else 1.0)
    sizes = pl.n_edges
    first = np.concatenate([[0], np.cumsum(sizes)])
    energies = np.array([0.5 * GO[g] - 0.5 * vals[first[g]:first[g + 1]].real.sum() for g in range(G)])
    return vals, energies
