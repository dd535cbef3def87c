"""Host-side tests of the planner behind qt_plan (no GPU: host_only plans).

* the exported schedule, contracted with numpy, equals the oracle's values;
* each network eliminates every one of its variables exactly once;
* the bucket graph is an in-forest with one root per network;
* operand masks and ranks agree with the producing bucket's width;
* lightcone wires carry 2(p - d) + 1 variables at distance d <= p (§II-B);
* statistics and byte accounting agree with the exported schedule;
* malformed graphs and width caps are rejected with the documented codes.
"""
import re
from pathlib import Path

import networkx as nx
import numpy as np
import pytest

import oracle
from paper_2204_06045_gb300 import qtgb, synth
from plan_eval import evaluate

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2204_06045_gb300 import build
    build.build()


def host_plan(n, edges, p, **kw):
    """A host-only plan; unsliced unless the test asks for slicing."""
    kw.setdefault("slice_width", -1)
    return qtgb.plan(n, edges, p, host_only=True, **kw)


@pytest.mark.parametrize("n,seed,p", [(10, 1000, 1), (12, 21, 2), (14, 22, 3), (16, 5, 2)])
def test_schedule_matches_oracle(n, seed, p):
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    with host_plan(n, edges, p) as pl:
        B, O = pl.export()
        vals = evaluate(B, O, g, b)
    np.testing.assert_allclose(vals.real, oracle.sv_zz(n, edges, g, b), rtol=0, atol=1e-12)
    assert np.abs(vals.imag).max() < 1e-12


@pytest.mark.parametrize("name,n,edges", [("K4", 4, synth.complete_graph(4)), ("prism", 6, synth.prism_graph()),
                                          ("petersen", 10, synth.petersen_graph()), ("ring", 8, synth.ring_graph(8))])
def test_schedule_matches_oracle_small_graphs(name, n, edges):
    for p in (1, 2):
        g, b = synth.angles(p, 3)
        with host_plan(n, edges, p, restarts=3, seed=7) as pl:
            B, O = pl.export()
            vals = evaluate(B, O, g, b)
        np.testing.assert_allclose(vals.real, oracle.sv_zz(n, edges, g, b), rtol=0, atol=1e-12)


def test_batch_schedule_matches_oracle():
    graphs = [(10, synth.random_regular_graph(10, 1)), (12, synth.random_regular_graph(12, 2)),
              (8, synth.random_regular_graph(8, 3))]
    p = 2
    G = np.array([synth.angles(p, s)[0] for s in (1, 2, 3)])
    Bt = np.array([synth.angles(p, s)[1] for s in (1, 2, 3)])
    with qtgb.plan_batch(graphs, p, host_only=True, slice_width=-1) as pl:
        B, O = pl.export()
        gon = np.repeat(np.arange(3), [e.shape[0] for _, e in graphs])
        vals = evaluate(B, O, G, Bt, gon)
    ref = np.concatenate([oracle.sv_zz(n, e, G[i], Bt[i]) for i, (n, e) in enumerate(graphs)])
    np.testing.assert_allclose(vals.real, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n,seed,p", [(30, 1000, 4), (50, 1000, 3)])
def test_structure(n, seed, p):
    edges = synth.random_regular_graph(n, seed)
    with host_plan(n, edges, p) as pl:
        B, O = pl.export()
        st = pl.stats()
        assert st["n_networks"] == edges.shape[0]
        for net in range(edges.shape[0]):
            idx = np.nonzero(B["network"] == net)[0]
            assert np.all(np.diff(idx) == 1), "buckets of a network are contiguous"
            wires = pl.network_wires(net, n)
            V = int(wires.sum())
            ns = B["n_sum"][idx]
            assert (ns <= 3).all()
            assert ((B["var2"][idx] >= 0) == (ns >= 2)).all() and ((B["var3"][idx] >= 0) == (ns >= 3)).all()
            allv = B["var"][idx].tolist() + B["var2"][idx][ns >= 2].tolist() + B["var3"][idx][ns >= 3].tolist()
            assert sorted(allv) == list(range(V)), "each variable eliminated once"
            roots = idx[B["parent"][idx] < 0]
            assert len(roots) == 1, "one connected network, one scalar result"
            assert B["width"][roots[0]] == 1
            for b in idx:
                par = B["parent"][b]
                if par >= 0:
                    assert idx[0] <= par < idx[-1] + 1 and par > b
            # children counts
            for b in idx:
                ops = O[B["op_begin"][b]:B["op_begin"][b] + B["n_ops"][b]]
                kids = ops["src"][ops["src"] >= 0]
                assert len(kids) == B["n_deps"][b]
                for k in kids:
                    assert B["parent"][k] == b
                n_res = B["width"][b] - B["n_sum"][b]  # the result's index bits
                alls = 0
                for op in ops:
                    assert bin(int(op["mask"])).count("1") + bin(int(op["smask"])).count("1") == op["rank"]
                    assert int(op["mask"]) >> n_res == 0
                    assert 1 <= int(op["smask"]) < (1 << B["n_sum"][b])
                    alls |= int(op["smask"])
                    if op["src"] >= 0:
                        assert op["rank"] == B["width"][op["src"]] - B["n_sum"][op["src"]]
                        assert B["level"][b] > B["level"][op["src"]]
                    else:
                        assert op["rank"] in (1, 2)
                assert alls == (1 << B["n_sum"][b]) - 1, "every summed variable is carried"
                # the union of operand bits is the whole output index
                allm = 0
                for op in ops:
                    allm |= int(op["mask"])
                assert allm == (1 << n_res) - 1
        # statistics agree with the exported schedule
        assert st["n_buckets"] == B.shape[0]
        assert st["max_width"] == B["width"].max()
        assert st["width_hist"].sum() == B.shape[0]
        assert st["sum_2w"] == float(np.sum(2.0 ** B["width"]))
        opbytes = sum(float(np.sum(2.0 ** O["rank"][B["op_begin"][b]:B["op_begin"][b] + B["n_ops"][b]]))
                      for b in range(B.shape[0]))
        outbytes = np.sum(2.0 ** (B["width"] - B["n_sum"]))
        assert np.isclose(st["alg_bytes"], 8 * (opbytes + outbytes))


@pytest.mark.parametrize("p", [1, 2, 3])
def test_lightcone_wires(p):
    n, edges = 24, synth.random_regular_graph(24, 9)
    G = nx.Graph()
    G.add_edges_from(map(tuple, edges))
    with host_plan(n, edges, p) as pl:
        for e in range(0, edges.shape[0], 4):
            j, k = map(int, edges[e])
            dj = nx.single_source_shortest_path_length(G, j)
            dk = nx.single_source_shortest_path_length(G, k)
            expect = [2 * (p - min(dj[q], dk[q])) + 1 if min(dj[q], dk[q]) <= p else 0 for q in range(n)]
            np.testing.assert_array_equal(pl.network_wires(e, n), expect)
            # the same shape as the oracle's own network builder
            np.testing.assert_array_equal(pl.network_wires(e, n), oracle.edge_network_shape(n, edges, p, e)[2])


def test_restarts_never_worse():
    n, edges = 30, synth.random_regular_graph(30, 1000)
    with host_plan(n, edges, 4, restarts=-1) as a, host_plan(n, edges, 4, restarts=4, seed=11) as b, \
            host_plan(n, edges, 4) as c:
        assert b.stats()["sum_2w"] <= a.stats()["sum_2w"]
        assert c.stats()["sum_2w"] <= a.stats()["sum_2w"]  # the default restarts the wide networks


def test_width27_bytes_convention():
    # a width-w bucket writes 2^(w-1) entries; a 27-index tensor of complex128 is ~2 GB (§III-C)
    gold = dict(l.split() for l in (ROOT / "tests/golden/width27_c128_bytes.txt").read_text().splitlines()
                if l.strip() and not l.startswith("#"))
    w = int(gold["width"])
    assert abs((2 ** w) * 16 - float(gold["bytes_approx"])) / float(gold["bytes_approx"]) < 0.08


@pytest.mark.parametrize("edges,n,p", [
    ([(0, 0), (0, 1)], 3, 1),          # self-loop
    ([(0, 1), (1, 0)], 3, 1),          # duplicate edge
    ([(0, 1), (1, 5)], 3, 1),          # vertex out of range
    ([(0, 1), (1, 2)], 3, 0),          # p < 1
])
def test_invalid_graphs(edges, n, p):
    with pytest.raises(qtgb.QTError) as ei:
        host_plan(n, np.array(edges), p)
    assert ei.value.code == qtgb.QT_EINVAL


def test_width_cap():
    n, edges = 30, synth.random_regular_graph(30, 1000)
    with pytest.raises(qtgb.QTError) as ei:
        host_plan(n, edges, 4, max_width=8)
    assert ei.value.code == qtgb.QT_EWIDTH


def test_arena_cap():
    n, edges = 30, synth.random_regular_graph(30, 1000)
    with pytest.raises(qtgb.QTError) as ei:
        host_plan(n, edges, 4, arena_bytes=1 << 20)
    assert ei.value.code == qtgb.QT_ENOMEM


def test_host_only_plan_refuses_evaluation():
    n, edges = 10, synth.random_regular_graph(10, 1)
    with host_plan(n, edges, 1) as pl:
        with pytest.raises(qtgb.QTError) as ei:
            pl.energy([0.1], [0.2])
        assert ei.value.code == qtgb.QT_ESTATE


def test_library_exports_every_declared_symbol():
    header = (ROOT / "include/qt.h").read_text()
    declared = set(re.findall(r"^\s*(?:int|void|const char \*)\s*(qt_\w+)\s*\(", header, flags=re.M))
    assert declared, "no declarations parsed"
    assert declared == set(qtgb.EXPORTS)
    L = qtgb.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert "sm_103a" in qtgb.version()


# ---- the persistent kernel's tile arithmetic, replayed on the host ----------

def _pext(x, m):
    r, k = 0, 0
    while m:
        low = m & -m
        if x & low:
            r |= 1 << k
        m ^= low
        k += 1
    return r


def _pext_arr(x, m):
    out = np.zeros_like(x)
    k = 0
    while m:
        low = m & -m
        out |= ((x & low) != 0).astype(x.dtype) << k
        m ^= low
        k += 1
    return out


def _check_tiles(B, O, b, max_tiles=24):
    """Replays the persistent kernel's staging of one bucket: for a claim group
    of consecutive tiles (the compressed base index advanced from tile to tile
    as the kernel does) and a few other tiles, every staged entry the tile loop
    reads for output o and summed value x is the entry 2 pext(o, M) + x of the
    operand, copies stay inside the operand, and footprints fit the stage."""
    n_out = int(B["width"][b]) - 1
    cb = int(B["tile_log2"][b])
    low = (1 << cb) - 1
    assert int(B["tile_bits"][b]) == low and cb <= n_out
    n_tiles = 1 << (n_out - cb)
    j = np.arange(1 << cb, dtype=np.int64)
    rng = np.random.default_rng(b)
    tiles = list(range(min(n_tiles, 16))) + [int(t) for t in rng.integers(0, n_tiles, size=max_tiles - 16)]
    ob, no = int(B["op_begin"][b]), int(B["n_ops"][b])
    folded = int(B["folded"][b])
    total = 0
    for t in range(no):
        M = int(O["mask"][ob + t])
        if (folded >> t) & 1:
            # a folded tensor has at most one output bit; one above the tile
            # is selected by bit (bit - cb) of the tile index
            assert bin(M).count("1") <= 1
            if M & ~low:
                pos = M.bit_length() - 1 - cb
                assert all(((c << cb) & M != 0) == bool((c >> pos) & 1) for c in tiles)
            continue
        rank = int(O["rank"][ob + t])
        plow = bin(M & low).count("1")
        mh = M >> cb
        total += 2 << plow
        cbase, prev = None, None
        for c in tiles:
            if prev is not None and c == prev + 1:  # the kernel's update within a group
                tb = (c & -c).bit_length() - 1
                r = bin(mh & ((1 << tb) - 1)).count("1")
                cbase = cbase - ((1 << r) - 1) + (((mh >> tb) & 1) << r)
            else:
                cbase = _pext(c, mh)
            prev = c
            stage = 2 * (cbase << plow) + np.arange(2 << plow)  # one bulk copy
            assert stage.max() < (1 << rank)
            o = (c << cb) + j
            assert o.max() < (1 << n_out)
            for x in (0, 1):
                np.testing.assert_array_equal(stage[2 * _pext_arr(j, M & low) + x], 2 * _pext_arr(o, M) + x)
    return total


@pytest.mark.parametrize("dtype,stage_elems", [("c64", 1024), ("c128", 512)])
def test_tile_copy_arithmetic(dtype, stage_elems):
    n, p = 30, 4
    edges = synth.random_regular_graph(n, 1000)
    with host_plan(n, edges, p, dtype=dtype) as pl:
        B, O = pl.export()
    rng = np.random.default_rng(0)
    wide = [b for b in range(len(B)) if B["width"][b] >= 12]
    for b in wide[:40] + [int(x) for x in rng.choice(len(B), size=60, replace=False)]:
        assert _check_tiles(B, O, b) <= stage_elems


def test_fused_units_are_closed_small_subtrees():
    """Fused units: every member has at most 2^8 outputs; a member's consumer is
    in its unit (a member or the root); a root's consumer is outside; every
    operand of a member or root that is an earlier result comes from the same
    unit. Gradient plans and the per-bucket schedule form no units."""
    graphs = [(n, e) for n, e, _, _ in synth.batch(4, 3, lo=50, hi=200, base_seed=1000)]
    with qtgb.plan_batch(graphs, 3, host_only=True) as pl:
        B, O = pl.export()
        st = pl.stats()
    role = B["unit_role"]
    assert st["n_units"] == int((role == 2).sum()) > 0
    assert st["n_fused"] == int((role > 0).sum())
    # unit of each bucket: walk up through members to the root
    unit = np.full(len(B), -1)
    for b in range(len(B)):
        if role[b] == 0:
            continue
        r = b
        while role[r] == 1:
            r = B["parent"][r]
            assert r >= 0 and role[r] > 0
        unit[b] = r
    for b in np.nonzero(role > 0)[0]:
        assert B["width"][b] - 1 <= 8
        ob, no = B["op_begin"][b], B["n_ops"][b]
        for src in O["src"][ob:ob + no]:
            if src >= 0:
                assert unit[src] == unit[b] and role[src] == 1
    for b in np.nonzero(role == 2)[0]:
        par = B["parent"][b]
        assert par < 0 or unit[par] != unit[b]
    with qtgb.plan_batch(graphs, 3, host_only=True, with_grad=True) as pl:
        assert pl.stats()["n_units"] == 0
    with qtgb.plan_batch(graphs, 3, host_only=True, sched="per_bucket") as pl:
        assert pl.stats()["n_units"] == 0
    with qtgb.plan_batch(graphs, 3, host_only=True, fuse=False) as pl:
        assert pl.stats()["n_units"] == 0


def _check_claim_order(B, O, G):
    """Every tile of every bucket scheduled on its own appears in exactly one
    group; a fused unit's root appears once; no bucket inside a unit appears;
    every group comes after every group of each of its bucket's producers
    (for a unit: after the producers outside it, of which there are none)."""
    nb = len(B)
    role = B["unit_role"]
    covered = [[] for _ in range(nb)]
    pos_last = np.full(nb, -1)
    pos_first = np.full(nb, -1)
    for i, gr in enumerate(G):
        b = int(gr["bucket"])
        assert role[b] != 1, "a bucket inside a unit was scheduled on its own"
        if pos_first[b] < 0:
            pos_first[b] = i
        pos_last[b] = i
        covered[b].append((int(gr["first_tile"]), int(gr["n_tiles"])))
        assert (gr["unit_buckets"] > 0) == (role[b] == 2)
    for b in range(nb):
        if role[b] == 1:
            assert not covered[b]
            continue
        n_tiles = 1 << (int(B["width"][b]) - 1 - int(B["tile_log2"][b]))
        if role[b] == 2:
            assert covered[b] == [(0, 1)]
            continue
        tiles = sorted(covered[b])
        assert tiles[0][0] == 0 and sum(t[1] for t in tiles) == n_tiles
        for (a, na), (c, _) in zip(tiles, tiles[1:]):
            assert a + na == c
        assert all(1 <= t[1] <= 16 for t in tiles)
    for b in range(nb):
        if role[b] != 0:
            continue
        ob, no = B["op_begin"][b], B["n_ops"][b]
        for src in O["src"][ob:ob + no]:
            if src >= 0:
                assert pos_last[src] < pos_first[b], "a group precedes one of its producers"


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_claim_order_covers_every_tile_and_respects_dependencies(dtype):
    n, p = 30, 4
    edges = synth.random_regular_graph(n, 1000)
    with host_plan(n, edges, p, dtype=dtype) as pl:
        B, O = pl.export()
        G = pl.export_groups()
        assert len(G) == pl.stats()["n_items"]
    _check_claim_order(B, O, G)


def test_claim_order_with_fused_units():
    graphs = [(n, e) for n, e, _, _ in synth.batch(6, 3, lo=50, hi=300, base_seed=1000)]
    with qtgb.plan_batch(graphs, 3, host_only=True) as pl:
        B, O = pl.export()
        G = pl.export_groups()
        assert pl.stats()["n_units"] > 0
    _check_claim_order(B, O, G)


def test_graph_without_edges_plans_no_networks():
    """C = 0 on a graph without edges: no networks, no buckets; in a batch such
    a graph contributes nothing but keeps its place."""
    empty = np.zeros((0, 2), dtype=np.int32)
    with host_plan(5, empty, 2) as pl:
        st = pl.stats()
        assert st["n_networks"] == 0 and st["n_buckets"] == 0
        assert len(pl.export_groups()) == 0
    graphs = [(5, empty), (10, synth.random_regular_graph(10, 1)), (1, empty)]
    with qtgb.plan_batch(graphs, 2, host_only=True) as pl:
        st = pl.stats()
        assert st["n_graphs"] == 3 and st["n_networks"] == 15
    with pytest.raises(qtgb.QTError):
        host_plan(0, empty, 2)


def test_tile_caps_per_width_class():
    """opts.tile_cap bounds the tile of each bucket-width class (output bits
    <= 6, 7..10, 11..14, 15..19, >= 20); 0 keeps the default (9)."""
    n, p = 30, 4
    edges = synth.random_regular_graph(n, 1000)
    cls = lambda n_out: 0 if n_out <= 6 else 1 if n_out <= 10 else 2 if n_out <= 14 else 3 if n_out <= 19 else 4
    with host_plan(n, edges, p, tile_cap=[0, 7, 8, 0, 6]) as pl:
        B, O = pl.export()
        st = pl.stats()
    assert st["tile_cap"] == [9, 7, 8, 9, 6]
    caps = [9, 7, 8, 9, 6]
    for b in range(len(B)):
        n_out = int(B["width"][b]) - 1
        assert B["tile_log2"][b] <= min(n_out, caps[cls(n_out)])
    assert (B["tile_log2"][B["width"] - 1 >= 20] == 6).all()
    for b in np.nonzero(B["width"] >= 12)[0][:30]:
        _check_tiles(B, O, int(b))
    with pytest.raises(qtgb.QTError):
        host_plan(n, edges, p, tile_cap=[12, 0, 0, 0, 0])


def test_adjoint_budget_splits_networks_into_passes():
    """A gradient plan over opts.adjoint_budget_bytes runs its networks in
    passes that fit; a budget below the largest network is refused."""
    n, p = 30, 4
    edges = synth.random_regular_graph(n, 1000)
    with host_plan(n, edges, p, with_grad=True) as full:
        need = full.stats()["arena_bytes"]
        assert full.stats()["n_passes"] == 1
    with host_plan(n, edges, p, with_grad=True, adjoint_budget_bytes=need // 3) as pl:
        assert pl.stats()["n_passes"] >= 3
    with pytest.raises(qtgb.QTError) as ei:
        host_plan(n, edges, p, with_grad=True, adjoint_budget_bytes=1 << 20)
    assert ei.value.code == qtgb.QT_ENOMEM


@pytest.mark.parametrize("n,seed,p", [(16, 23, 3), (20, 1020, 4), (30, 1000, 4)])
def test_merged_eliminations_give_the_same_values(n, seed, p):
    """Merged eliminations (the default; opts.no_merge turns them off): chains
    of eliminations merged (buckets summing two or three variables) contract,
    in the numpy evaluator of the exported schedule, to the same network
    values as the unmerged schedule and the oracle."""
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    with host_plan(n, edges, p, merge=True) as pl:
        Bm, Om = pl.export()
        stm = pl.stats()
    with host_plan(n, edges, p, merge=False) as pl:
        B1, _ = pl.export()
        st1 = pl.stats()
    merged = Bm["n_sum"] > 1
    assert merged.any() and (Bm["n_sum"] <= 3).all()
    assert len(Bm) == len(B1) - int((Bm["n_sum"] - 1).sum())
    assert stm["alg_bytes"] < st1["alg_bytes"]
    # every operand's index bits: its output bits plus its summed variables
    for k in np.nonzero(merged)[0]:
        for t in range(Bm["op_begin"][k], Bm["op_begin"][k] + Bm["n_ops"][k]):
            assert bin(int(Om["mask"][t])).count("1") + bin(int(Om["smask"][t])).count("1") == Om["rank"][t]
    if n <= 20:
        vals = evaluate(Bm, Om, g, b)
        np.testing.assert_allclose(vals.real, oracle.sv_zz(n, edges, g, b), rtol=0, atol=1e-12)
        assert np.abs(vals.imag).max() < 1e-12


def test_merge_applies_to_persistent_plans_only():
    """The per-bucket kernel sums one variable per bucket: its plans are never
    merged. Persistent energy plans merge by default; gradient plans when asked
    (the reverse sweep takes merged buckets)."""
    n, seed, p = 18, 5, 4
    edges = synth.random_regular_graph(n, seed)
    with host_plan(n, edges, p, merge=True, sched="per_bucket") as pl:
        B, _ = pl.export()
    with host_plan(n, edges, p, merge=True) as pl:
        Bm, _ = pl.export()
    with host_plan(n, edges, p, merge=True, with_grad=True) as pl:
        Bg, _ = pl.export()
    with host_plan(n, edges, p, with_grad=True) as pl:  # gradient plans merge only when asked
        Bd, _ = pl.export()
    assert (B["n_sum"] == 1).all() and (Bm["n_sum"] > 1).any() and (Bg["n_sum"] > 1).any()
    assert (Bd["n_sum"] == 1).all()


@pytest.mark.parametrize("n,seed,p,width", [(12, 21, 2, 5), (14, 22, 3, 8), (16, 23, 3, 9), (18, 5, 4, 17)])
def test_sliced_networks_sum_to_the_same_values(n, seed, p, width):
    """opts.slice_width: every network wider than the target gets variables
    fixed; its slices (2^s networks over the other variables, one per
    assignment of the fixed ones) contract, in the numpy evaluator, to values
    whose sum per network is the state vector's <Z_jZ_k>."""
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    with host_plan(n, edges, p, slice_width=width) as pl:
        B, O = pl.export()
        F = pl.export_fixed()
        st = pl.stats()
    with host_plan(n, edges, p) as pl:
        st0 = pl.stats()
    assert st0["max_width"] > width and st["slice_bits"] >= 1
    assert st["n_slices"] > edges.shape[0] and st["max_width"] <= max(width, st0["max_width"] - st["slice_bits"])
    for net in range(edges.shape[0]):
        idx = np.nonzero(B["network"] == net)[0]
        slices = np.unique(B["slice"][idx])
        assert slices.tolist() == list(range(len(slices))) and len(slices) & (len(slices) - 1) == 0
        # every slice is the same schedule: widths, operand counts and masks agree
        per = [idx[B["slice"][idx] == s] for s in slices]
        for q in per[1:]:
            assert (B["width"][q] == B["width"][per[0]]).all() and (B["n_ops"][q] == B["n_ops"][per[0]]).all()
            assert (B["var"][q] == B["var"][per[0]]).all()
        # fixed gate entries: the same gates in every slice, entries in range
        f = F[F["network"] == net]
        if len(slices) > 1:
            assert len(f) % len(slices) == 0
    assert ((O["leaf_sub"] == 0) | (O["leaf_sub"] == 2)).all()
    assert (O["leaf_sub"][O["src"] >= 0] == 0).all()
    assert ((F["entry"] >= 0) & (F["entry"] < 4)).all()
    vals = evaluate(B, O, g, b, fixed=F)
    np.testing.assert_allclose(vals.real, oracle.sv_zz(n, edges, g, b), rtol=0, atol=1e-12)
    assert np.abs(vals.imag).max() < 1e-12


def test_slicing_options():
    n, seed, p = 16, 23, 3
    edges = synth.random_regular_graph(n, seed)
    for bad in (dict(slice_width=1), dict(slice_width=32), dict(slice_width=-2), dict(max_slice_bits=17)):
        with pytest.raises(qtgb.QTError):
            host_plan(n, edges, p, **bad)
    with host_plan(n, edges, p, slice_width=6, max_slice_bits=2) as pl:
        st = pl.stats()
    assert st["slice_bits"] == 2 and st["max_width"] > 6  # the bit budget ran out first
    with host_plan(n, edges, p, slice_width=6, with_grad=True) as pl:  # gradient plans are sliced too
        st = pl.stats()
    assert st["slice_bits"] > 0 and st["n_slices"] > edges.shape[0]
    with host_plan(n, edges, p, slice_width=30) as pl:  # nothing that wide: no slices
        assert pl.stats()["n_slices"] == edges.shape[0] and len(pl.export_fixed()) == 0
    # the default target: 22 for complex64, 20 for complex128 (N=30 p=4 reaches width 26)
    e30 = synth.random_regular_graph(30, 1000)
    for dtype, target in (("c64", 22), ("c128", 20)):
        with qtgb.plan(30, e30, 4, host_only=True, dtype=dtype) as pl:
            st = pl.stats()
        assert st["slice_bits"] > 0 and st["max_width"] <= target


@pytest.mark.parametrize("n,seed,p", [(20, 3, 1), (60, 3, 2), (100, 7, 3)])
def test_deduplicated_networks_take_their_representatives_values(n, seed, p):
    """opts.dedup: networks whose lightcones are isomorphic are
    contracted once. Every network's value (its representative's) equals its
    own contraction in the full plan; representatives come first and are
    contracted; duplicates have no buckets."""
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    with host_plan(n, edges, p, dedup=True) as pl:
        B, O = pl.export()
        F = pl.export_fixed()
        R = pl.export_reps()
        st = pl.stats()
    with host_plan(n, edges, p) as pl:
        B0, O0 = pl.export()
        st0 = pl.stats()
    assert st["n_unique"] < st["n_networks"] == edges.shape[0] and st0["n_unique"] == st0["n_networks"]
    assert st["n_buckets"] < st0["n_buckets"]
    reps = np.unique(R)
    assert (R <= np.arange(R.size)).all() and (R[reps] == reps).all() and reps.size == st["n_unique"]
    assert set(np.unique(B["network"]).tolist()) == set(reps.tolist())
    vals = evaluate(B, O, g, b, fixed=F)
    mine = np.array([vals[R[i]] for i in range(R.size)])
    full = evaluate(B0, O0, g, b)
    np.testing.assert_allclose(mine, full, rtol=0, atol=1e-12)
    if n <= 20:
        np.testing.assert_allclose(mine.real, oracle.sv_zz(n, edges, g, b), rtol=0, atol=1e-12)


def test_dedup_stays_within_a_graph_and_off_for_passes():
    graphs = [(40, synth.random_regular_graph(40, 1)), (40, synth.random_regular_graph(40, 2))]
    with qtgb.plan_batch(graphs, 2, host_only=True, dedup=True, slice_width=-1) as pl:
        R = pl.export_reps()
    m0 = graphs[0][1].shape[0]
    assert (R[:m0] < m0).all() and (R[m0:] >= m0).all()  # no sharing across graphs (their angles differ)
    assert len(np.unique(R[:m0])) < m0 and len(np.unique(R[m0:])) < R.size - m0
    with host_plan(40, graphs[0][1], 2, dedup=True, with_grad=True) as pl:  # the sweep seeds a class once
        assert pl.stats()["n_unique"] < pl.stats()["n_networks"]
    with host_plan(40, graphs[0][1], 2, dedup=True, with_grad=True, adjoint_budget_bytes=1 << 16) as pl:
        assert pl.stats()["n_unique"] == pl.stats()["n_networks"]  # plans in passes contract every network


@pytest.mark.parametrize("grad", [False, True])
def test_dedup_kept_under_a_budget_the_deduplicated_plan_fits(grad):
    """A budget set but not exceeded by the deduplicated plan keeps deduplication
    (no passes); one below it runs every network in passes."""
    n, seed, p = 60, 3, 2
    edges = synth.random_regular_graph(n, seed)
    key = "adjoint_budget_bytes" if grad else "energy_budget_bytes"
    with host_plan(n, edges, p, dedup=True, with_grad=grad, slice_width=-1) as pl:
        st = pl.stats()
    assert st["n_unique"] < st["n_networks"]
    with host_plan(n, edges, p, dedup=True, with_grad=grad, slice_width=-1, **{key: st["arena_bytes"]}) as pl:
        s2 = pl.stats()
        assert s2["n_unique"] == st["n_unique"] and s2["n_passes"] == 1 and s2["pass_arena_bytes"] == 0
    with host_plan(n, edges, p, dedup=True, with_grad=grad, slice_width=-1, **{key: st["arena_bytes"] // 2}) as pl:
        s3 = pl.stats()
        assert s3["n_passes"] >= 2 and s3["n_unique"] == s3["n_networks"]
        assert 0 < s3["pass_arena_bytes"] <= st["arena_bytes"] // 2


def test_energy_budget_runs_in_passes_that_fit():
    """opts.energy_budget_bytes: an energy plan over the budget is cut into
    passes over its networks' slices, each pass's arena within the budget; a
    slice that alone exceeds it gives QT_ENOMEM."""
    n, p = 30, 4
    edges = synth.random_regular_graph(n, 1000)
    with qtgb.plan(n, edges, p, host_only=True) as pl:
        full = pl.stats()["arena_bytes"]
    last = 1
    for budget in (full // 2, full // 5, full // 12):
        with qtgb.plan(n, edges, p, host_only=True, energy_budget_bytes=budget) as pl:
            st = pl.stats()
        assert st["n_passes"] > last and 0 < st["pass_arena_bytes"] <= budget
        last = st["n_passes"]
    with qtgb.plan(n, edges, p, host_only=True, energy_budget_bytes=full * 2) as pl:
        assert pl.stats()["n_passes"] == 1 and pl.stats()["pass_arena_bytes"] == 0
    with pytest.raises(qtgb.QTError) as ei:
        qtgb.plan(n, edges, p, host_only=True, energy_budget_bytes=1 << 20)
    assert ei.value.code == qtgb.QT_ENOMEM


@pytest.mark.parametrize("n,seed,p", [(200, 5, 2), (400, 9, 3), (60, 11, 3), (90, 4, 3)])
def test_dedup_contracts_one_network_per_lightcone_class(n, seed, p):
    """opts.dedup contracts exactly one network per isomorphism class of
    lightcones (qubits within distance p of the edge, labelled by distance;
    the graph edges with an endpoint within p - 1): the classes are counted
    here with networkx's isomorphism test, independently of the planner's
    keys (AHU codes for trees, a canonical search for lightcones with cycles)."""
    edges = synth.random_regular_graph(n, seed)
    G = nx.Graph()
    G.add_edges_from(map(tuple, edges))
    classes = {}
    for j, k in edges:
        d = nx.multi_source_dijkstra_path_length(G, [int(j), int(k)], cutoff=p)
        H = nx.Graph()
        H.add_nodes_from((v, {"d": d[v]}) for v in d)
        H.add_edges_from((a, c) for a, c in G.subgraph(d).edges() if min(d[a], d[c]) <= p - 1)
        sig = (H.number_of_nodes(), H.number_of_edges(), tuple(sorted(d.values())))
        reps = classes.setdefault(sig, [])
        if not any(nx.is_isomorphic(R, H, node_match=lambda a, c: a["d"] == c["d"]) for R in reps):
            reps.append(H)
    n_classes = sum(len(r) for r in classes.values())
    with host_plan(n, edges, p, dedup=True) as pl:
        st = pl.stats()
    assert n_classes < edges.shape[0]
    assert st["n_unique"] == n_classes


# ---- contraction plans (the paper's "tncontract" expressions, §II-E) --------

def test_contraction_plans_follow_bucket_elimination():
    """Host-only contraction plans: the paper's two printed expressions give one
    bucket (dacb,ad->bcd: width 4) and two (caedb,eab->cde: widths 5, 4); two
    summed labels over 2^10 or more outputs merge into one bucket; the bytes
    are the buckets' operands read once and results written once."""
    with qtgb.contraction([[3, 0, 2, 1], [0, 3]], [1, 2, 3], host_only=True) as c:
        st = c.stats()
    assert st["n_buckets"] == 1 and st["widths"] == [4] and st["n_summed"] == 1
    assert st["alg_bytes"] == 8 * (16 + 4 + 8)
    with qtgb.contraction([[2, 0, 4, 3, 1], [4, 0, 1]], [2, 3, 4], host_only=True) as c:
        st = c.stats()
    assert st["n_buckets"] == 2 and st["widths"] == [5, 4] and st["n_merged"] == 0
    assert st["alg_bytes"] == 8 * ((32 + 8 + 16) + (16 + 8))
    with qtgb.contraction([list(range(15)), [3, 9]], [x for x in range(15) if x not in (3, 9)], dtype="c128",
                          host_only=True) as c:
        st = c.stats()
    assert st["n_buckets"] == 1 and st["n_merged"] == 1 and st["widths"] == [15]
    assert st["alg_bytes"] == 16 * (2 ** 15 + 4 + 2 ** 13)
    assert st["copy_bytes"] == 16 * 2 * (2 ** 15 + 4 + 2 ** 13)


@pytest.mark.parametrize("seed", range(40))
def test_random_contraction_plans_are_accepted(seed):
    """Every expression of the paper's recipe (4..25 indices) plans, the widest
    bucket holding every index."""
    la, lb, lo = synth.tncontract_random(seed)
    with qtgb.contraction([la, lb], lo, host_only=True) as c:
        st = c.stats()
    assert st["max_width"] == len(la) and st["n_summed"] == len(la) - len(lo)


def test_invalid_contractions_are_refused_on_the_host():
    for labels, lo in (([[0, 1], [2, 3]], [0, 1, 2, 3]), ([[0, 0]], [0]), ([[0, 1]], [5]), ([[0, 1], [2, 3]], [1, 3]),
                       ([[0, 1, 2], [1]], [1, 2]), ([list(range(31))], [0])):
        with pytest.raises(qtgb.QTError) as ei:
            qtgb.contraction(labels, lo, host_only=True)
        assert ei.value.code == qtgb.QT_EINVAL, labels
