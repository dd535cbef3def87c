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


STEP = 1 << 18  # a unit step record runs several buckets at once


def _pext_int(o: int, mask: int) -> int:
    r, k = 0, 0
    while mask:
        low = mask & -mask
        if o & low:
            r |= 1 << k
        k += 1
        mask ^= low
    return r


def run_unit_program(recs, first, n_buckets, arena, root_off, scratch_elems):
    """Interpret one fused unit's program as the persistent kernel runs it:
    steps of one bucket (outputs over the whole warp) or of several
    independent buckets (one output per lane, the lane map in the step record).
    Results live in a scratch array until the root's goes to the arena. Every
    member of a step reads before any writes; the step's scratch writes must
    not touch what any of its members reads (the planner's placement), which
    is asserted here, as is the shift form of one-run masks. `recs` is a list
    of (a, b, off) integer tuples."""
    scr = [complex("nan")] * scratch_elems

    def output(ops, o):
        vals = [1 + 0j, 1 + 0j]
        reads = []
        for a, b, off in ops:
            j = _pext_int(o, a)
            if b & 2:
                assert ((o & a) >> (b >> 8)) == j, "shift extract disagrees with the bit extract"
            src = scr if b & 1 else arena
            if b & 1:
                reads += [off + 2 * j, off + 2 * j + 1]
            vals[0] *= src[off + 2 * j]
            vals[1] *= src[off + 2 * j + 1]
        return vals[0] + vals[1], reads

    pos, k = first, 0
    while k < n_buckets:
        ha, hb, hoff = recs[pos]
        writes, reads = [], set()
        if ha & STEP:
            n_recs, n_items, used = ha & 0x3F, (ha >> 20) & 7, (ha >> 24) & 0x3F
            for lane in range(used):
                q = (hoff >> (2 * lane)) & 3
                at = 1 if q == 0 else (hb >> (8 * (q - 1))) & 0xFF
                qa, qb, qoff = recs[pos + at]
                n_ops = (qa >> 8) & 0xFF
                assert not (qa >> 16) & 1, "the unit's root in a step of several buckets"
                o = lane - qoff
                assert 0 <= o < (1 << (qa & 0xFF))
                v, r = output(recs[pos + at + 1:pos + at + 1 + n_ops], o)
                reads.update(r)
                writes.append((qb + o, v))
            pos += n_recs
            k += n_items
            assert not reads & {w for w, _ in writes}, "a step writes scratch that one of its members reads"
        else:
            n_out, n_ops, root = ha & 0xFF, (ha >> 8) & 0xFF, (ha >> 16) & 1
            ops = recs[pos + 1:pos + 1 + n_ops]
            for o in range(1 << n_out):
                v, _ = output(ops, o)
                writes.append(((root_off if root else hb) + o, v))
            pos += 1 + n_ops
            k += 1
            if root:
                for w, v in writes:
                    arena[w] = v
                continue
        for w, v in writes:
            scr[w] = v


def emulate(pl, gammas, betas, p, with_units=False, scratch_elems=1024):
    """(per-network complex values, per-graph energies) of plan `pl`. With
    `with_units`, fused units run their programs (interpreted here) instead of
    contracting their members one by one."""
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
    role = None
    if with_units:
        Bi, _ = pl.export()
        role = Bi["unit_role"]
        units, recs_arr = pl.export_units()
        recs = [(int(r["a"]), int(r["b"]), int(r["off"])) for r in recs_arr]
        unit_of = {int(u["root"]): u for u in units}
    for bi, b in enumerate(B):
        if role is not None and role[bi] == 1:
            continue  # a unit member: its unit's program computes it in scratch
        if role is not None and role[bi] == 2:
            u = unit_of[bi]
            run_unit_program(recs, int(u["first_rec"]), int(u["n_buckets"]), arena, int(b["out_off"]), scratch_elems)
            continue
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
