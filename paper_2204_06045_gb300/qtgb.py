"""Python binding of libqtgb (include/qt.h): argument marshalling only.

Every step of the energy evaluation runs in the CUDA kernels behind the C ABI.
There is no fallback: if ``libqtgb.so`` is missing or a call fails, this module
raises. PyTorch is used only to pass device tensors and CUDA streams.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
LIB_PATH = _HERE / "libqtgb.so"

QT_OK, QT_EINVAL, QT_EWIDTH, QT_ENOMEM, QT_ECUDA, QT_ETIMEOUT, QT_EBOUNDS, QT_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
QT_C64, QT_C128 = 0, 1
QT_SCHED_PERSISTENT, QT_SCHED_PER_BUCKET = 0, 1
LEAF_KINDS = ("plus", "zobs", "zz", "zz_conj", "rx", "rx_conj")

# every symbol include/qt.h declares
EXPORTS = ("qt_plan", "qt_plan_subset", "qt_plan_batch", "qt_plan_stats_get", "qt_plan_export", "qt_plan_network_wires",
           "qt_energy", "qt_energy_batch", "qt_energy_grad", "qt_last_imag", "qt_sync", "qt_kernel_time",
           "qt_bucket_time", "qt_trace_counters", "qt_trace_bucket_times", "qt_debug_stall_bucket", "qt_plan_free", "qt_error_string", "qt_version", "qt_last_error_detail",
           "qt_energy_noalloc", "qt_fma_peak", "qt_plan_export_groups", "qt_plan_shard", "qt_plan_export_fixed",
           "qt_plan_export_reps", "qt_plan_export_device", "qt_plan_pass", "qt_contract_plan", "qt_contract_run",
           "qt_contract_sync", "qt_contract_stats_get", "qt_contract_free", "qt_plan_export_units")


class QTError(RuntimeError):
    def __init__(self, code: int, what: str):
        detail = ""
        if code in (QT_ECUDA, QT_ENOMEM):
            detail = lib().qt_last_error_detail().decode()
        super().__init__(f"{what}: {error_string(code)} ({code})" + (f" [{detail}]" if detail else ""))
        self.code = code


class PlanOpts(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("sched", ctypes.c_int), ("order_restarts", ctypes.c_int32),
                ("order_seed", ctypes.c_uint64), ("max_width", ctypes.c_int32), ("arena_bytes", ctypes.c_size_t),
                ("with_grad", ctypes.c_int32), ("spin_limit", ctypes.c_uint64), ("chunk_log2", ctypes.c_int32),
                ("host_only", ctypes.c_int32), ("run_tiles", ctypes.c_int32), ("trace", ctypes.c_int32),
                ("order", ctypes.c_int32), ("no_fuse", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("tile_cap", ctypes.c_int8 * 8), ("no_merge", ctypes.c_int32), ("adjoint_budget_bytes", ctypes.c_size_t),
                ("slice_width", ctypes.c_int32), ("max_slice_bits", ctypes.c_int32), ("dedup", ctypes.c_int32),
                ("energy_budget_bytes", ctypes.c_size_t)]


class PlanStats(ctypes.Structure):
    _fields_ = [("n_graphs", ctypes.c_int32), ("n_networks", ctypes.c_int32), ("n_buckets", ctypes.c_int64),
                ("n_operands", ctypes.c_int64), ("max_width", ctypes.c_int32), ("p", ctypes.c_int32),
                ("sum_2w", ctypes.c_double), ("alg_bytes", ctypes.c_double), ("flops", ctypes.c_double),
                ("arena_bytes", ctypes.c_int64), ("n_tasks", ctypes.c_int64), ("n_items", ctypes.c_int64),
                ("n_levels", ctypes.c_int32), ("dtype", ctypes.c_int32), ("width_hist", ctypes.c_int64 * 64),
                ("plan_seconds", ctypes.c_double), ("sim_seconds", ctypes.c_double),
                ("n_units", ctypes.c_int64), ("n_fused", ctypes.c_int64), ("tile_cap", ctypes.c_int32 * 8),
                ("run_tiles", ctypes.c_int32), ("tune_seconds", ctypes.c_double), ("tune_candidates", ctypes.c_int32),
                ("n_passes", ctypes.c_int32), ("slice_bits", ctypes.c_int32), ("n_slices", ctypes.c_int64),
                ("n_unique", ctypes.c_int64), ("pass_arena_bytes", ctypes.c_int64)]


BUCKET_DTYPE = np.dtype([("network", np.int32), ("width", np.int32), ("n_ops", np.int32), ("op_begin", np.int32),
                         ("parent", np.int32), ("n_deps", np.int32), ("level", np.int32), ("var", np.int32),
                         ("tile_log2", np.int32), ("tile_bits", np.uint32), ("folded", np.uint32),
                         ("unit_role", np.uint32), ("n_sum", np.int32), ("var2", np.int32),
                         ("var3", np.int32), ("slice", np.int32)])
GROUP_DTYPE = np.dtype([("bucket", np.int32), ("first_tile", np.int32), ("n_tiles", np.int32),
                        ("unit_buckets", np.int32)])
OPERAND_DTYPE = np.dtype([("src", np.int32), ("leaf_kind", np.int32), ("leaf_layer", np.int32),
                          ("mask", np.uint32), ("rank", np.int32), ("smask", np.uint32), ("leaf_sub", np.int32),
                          ("pad", np.int32)])
DEV_BUCKET_DTYPE = np.dtype([("out_off", np.uint64), ("op_begin", np.int32), ("n_ops", np.int32),
                             ("n_out", np.int32), ("n_sum", np.int32)])
DEV_OPERAND_DTYPE = np.dtype([("off", np.uint64), ("mask", np.uint32), ("pairs_x", np.int32), ("leaf", np.int32),
                              ("pad", np.int32)])
class ContractStats(ctypes.Structure):
    _fields_ = [("n_buckets", ctypes.c_int32), ("max_width", ctypes.c_int32), ("n_summed", ctypes.c_int32),
                ("n_merged", ctypes.c_int32), ("alg_bytes", ctypes.c_double), ("copy_bytes", ctypes.c_double),
                ("arena_bytes", ctypes.c_int64), ("widths", ctypes.c_int32 * 32)]


UNIT_DTYPE = np.dtype([("root", np.int32), ("n_buckets", np.int32), ("first_rec", np.int64)])
UNIT_REC_DTYPE = np.dtype([("a", np.uint32), ("b", np.uint32), ("off", np.uint64)])
FIXED_DTYPE = np.dtype([("network", np.int32), ("slice", np.int32), ("leaf_kind", np.int32), ("leaf_layer", np.int32),
                        ("entry", np.int32), ("pad", np.int32)])

_lib = None


def use_library(path) -> None:
    """Load the library from ``path`` instead (a tuning variant); before first use."""
    global LIB_PATH, _lib
    if _lib is not None:
        raise RuntimeError("libqtgb is already loaded")
    LIB_PATH = Path(path)


def lib():
    """Load libqtgb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2204_06045_gb300.build.build()")
        L = ctypes.CDLL(str(LIB_PATH))
        vp, dp, i32, i64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_int64
        i32p = ctypes.POINTER(ctypes.c_int32)
        L.qt_plan.argtypes = [i32, i32, i32p, i32, ctypes.POINTER(PlanOpts), ctypes.POINTER(vp)]
        L.qt_plan_batch.argtypes = [i32, i32p, i32p, i32p, i32, ctypes.POINTER(PlanOpts), ctypes.POINTER(vp)]
        L.qt_plan_subset.argtypes = [i32, i32, i32p, i32, i32, i32p, ctypes.POINTER(PlanOpts), ctypes.POINTER(vp)]
        L.qt_plan_stats_get.argtypes = [vp, ctypes.POINTER(PlanStats)]
        L.qt_plan_export.argtypes = [vp, vp, vp]
        L.qt_plan_network_wires.argtypes = [vp, i32, i32p]
        L.qt_energy.argtypes = [vp, vp, vp, vp, vp, vp]
        L.qt_energy_batch.argtypes = [vp, vp, vp, vp, vp, vp]
        L.qt_energy_grad.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.qt_energy_noalloc.argtypes = [vp, vp, vp, vp, vp, vp]
        L.qt_fma_peak.argtypes = [i32, dp]
        L.qt_plan_export_groups.argtypes = [vp, vp, ctypes.POINTER(i64)]
        L.qt_plan_export_units.argtypes = [vp, vp, vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.qt_plan_export_fixed.argtypes = [vp, vp, ctypes.POINTER(i64)]
        L.qt_plan_export_reps.argtypes = [vp, i32p]
        L.qt_plan_export_device.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.POINTER(i64)]
        L.qt_plan_pass.argtypes = [vp, i32, ctypes.POINTER(vp), i32p, i32p]
        L.qt_plan_shard.argtypes = [i32, i32, i32p, i32, i32, i32, ctypes.POINTER(PlanOpts), ctypes.POINTER(vp), i32p,
                                    i32p]
        L.qt_last_imag.argtypes = [vp, dp]
        L.qt_sync.argtypes = [vp, vp]
        L.qt_kernel_time.argtypes = [vp, dp, ctypes.POINTER(i64), i32]
        L.qt_debug_stall_bucket.argtypes = [vp, i64]
        L.qt_trace_counters.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(i64)]
        L.qt_bucket_time.argtypes = [vp, i64, i32, dp, dp]
        L.qt_trace_bucket_times.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
        L.qt_plan_free.argtypes = [vp]
        L.qt_plan_free.restype = None
        L.qt_contract_plan.argtypes = [i32, i32p, i32p, i32, i32p, ctypes.c_int, i32, ctypes.POINTER(vp)]
        L.qt_contract_run.argtypes = [vp, ctypes.POINTER(vp), vp, vp]
        L.qt_contract_sync.argtypes = [vp, vp]
        L.qt_contract_stats_get.argtypes = [vp, ctypes.POINTER(ContractStats)]
        L.qt_contract_free.argtypes = [vp]
        L.qt_contract_free.restype = None
        L.qt_error_string.argtypes = [ctypes.c_int]
        L.qt_error_string.restype = ctypes.c_char_p
        L.qt_version.restype = ctypes.c_char_p
        L.qt_last_error_detail.restype = ctypes.c_char_p
        for name in ("qt_plan", "qt_plan_subset", "qt_plan_batch", "qt_plan_stats_get", "qt_plan_export", "qt_plan_network_wires",
                     "qt_energy", "qt_energy_batch", "qt_energy_grad", "qt_last_imag", "qt_sync", "qt_kernel_time",
                     "qt_debug_stall_bucket", "qt_trace_counters", "qt_bucket_time", "qt_trace_bucket_times",
                     "qt_energy_noalloc", "qt_fma_peak", "qt_plan_export_groups", "qt_plan_shard",
                     "qt_plan_export_fixed", "qt_plan_export_reps", "qt_plan_export_device", "qt_plan_pass",
                     "qt_contract_plan", "qt_contract_run", "qt_contract_sync", "qt_contract_stats_get",
                     "qt_plan_export_units"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def fma_peak(dtype: str = "c128") -> float:
    """Measured FMA throughput (TFLOP/s) of the current device: FP64 for c128, FP32 for c64."""
    out = ctypes.c_double(0.0)
    _check(lib().qt_fma_peak({"c64": QT_C64, "c128": QT_C128}[dtype], ctypes.byref(out)), "qt_fma_peak")
    return out.value


def error_string(code: int) -> str:
    return lib().qt_error_string(int(code)).decode()


def version() -> str:
    return lib().qt_version().decode()


def _check(rc: int, what: str):
    if rc != QT_OK:
        raise QTError(rc, what)


def _ptr(x):
    """Address of a numpy array or a torch tensor (host or CUDA); None -> NULL."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"unsupported buffer {type(x)}")


def _f64_in(x):
    if hasattr(x, "data_ptr"):
        import torch
        assert x.dtype == torch.float64 and x.is_contiguous(), "angle tensors must be contiguous float64"
        return x
    return np.ascontiguousarray(x, dtype=np.float64)


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


class Plan:
    """A planned QAOA MaxCut energy evaluation on one graph or a batch of graphs."""

    def __init__(self, handle, n_edges_per_graph, p, dtype, n_vertices, owned=True):
        self._h = ctypes.c_void_p(handle)
        self._owned = owned  # False: a pass of another plan, which frees it
        self.n_edges = list(n_edges_per_graph)
        self.n_vertices = list(n_vertices)
        self.p = p
        self.dtype = dtype

    # -- construction -------------------------------------------------------------
    @staticmethod
    def _opts(dtype="c64", sched="persistent", restarts=0, seed=0, max_width=31, arena_bytes=0,
              with_grad=False, spin_limit=0, chunk_log2=0, host_only=False, run_tiles=0, trace=False,
              order="simulated", fuse=True, autotune=0, tile_cap=None, adjoint_budget_bytes=0, merge=None,
              slice_width=0, max_slice_bits=0, dedup=False, energy_budget_bytes=0):
        # slice_width: 0 the library's default target, -1 no slicing
        o = PlanOpts()
        o.dtype = {"c64": QT_C64, "c128": QT_C128}[dtype]
        o.sched = {"persistent": QT_SCHED_PERSISTENT, "per_bucket": QT_SCHED_PER_BUCKET}[sched]
        o.order_restarts = int(restarts)
        o.order_seed = int(seed)
        o.max_width = int(max_width)
        o.arena_bytes = int(arena_bytes)
        o.with_grad = int(bool(with_grad))
        o.spin_limit = int(spin_limit)
        o.chunk_log2 = int(chunk_log2)
        o.host_only = int(bool(host_only))
        o.run_tiles = int(run_tiles)
        o.trace = int(bool(trace))
        o.order = {"simulated": 0, "ready_queue": 1}[order]
        o.no_fuse = 0 if fuse else 1
        o.autotune = int(autotune)
        o.adjoint_budget_bytes = int(adjoint_budget_bytes)
        # merge: None the library's default (energy plans merge, gradient plans do not),
        # True every persistent plan, gradient plans included; False none
        o.no_merge = 0 if merge is None else (-1 if merge else 1)
        o.slice_width = int(slice_width)
        o.max_slice_bits = int(max_slice_bits)
        o.dedup = 1 if dedup else 0
        o.energy_budget_bytes = int(energy_budget_bytes)
        for i, c in enumerate(tile_cap or []):
            o.tile_cap[i] = int(c)
        return o

    @classmethod
    def create(cls, n: int, edges, p: int, **opts) -> "Plan":
        e = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
        o = cls._opts(**opts)
        h = ctypes.c_void_p()
        _check(lib().qt_plan(int(n), int(e.shape[0]), e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(p),
                             ctypes.byref(o), ctypes.byref(h)), "qt_plan")
        return cls(h.value, [e.shape[0]], p, opts.get("dtype", "c64"), [n])

    @classmethod
    def create_subset(cls, n: int, edges, p: int, sel, **opts) -> "Plan":
        """Plan only the lightcone networks of the edges listed in ``sel``."""
        e = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
        sv = np.ascontiguousarray(sel, dtype=np.int32).ravel()
        o = cls._opts(**opts)
        h = ctypes.c_void_p()
        ip = ctypes.POINTER(ctypes.c_int32)
        _check(lib().qt_plan_subset(int(n), int(e.shape[0]), e.ctypes.data_as(ip), int(p), int(sv.size),
                                    sv.ctypes.data_as(ip), ctypes.byref(o), ctypes.byref(h)), "qt_plan_subset")
        return cls(h.value, [sv.size], p, opts.get("dtype", "c64"), [n])

    @classmethod
    def create_shard(cls, n: int, edges, p: int, world: int, rank: int, **opts) -> "Plan":
        """Rank ``rank``'s share (by LPT on network cost) of the graph's networks;
        ``plan.shard_edges`` lists its edges."""
        e = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
        mine = np.zeros(max(1, e.shape[0]), dtype=np.int32)
        cnt = ctypes.c_int32(0)
        o = cls._opts(**opts)
        h = ctypes.c_void_p()
        ip = ctypes.POINTER(ctypes.c_int32)
        _check(lib().qt_plan_shard(int(n), int(e.shape[0]), e.ctypes.data_as(ip), int(p), int(world), int(rank),
                                   ctypes.byref(o), ctypes.byref(h), mine.ctypes.data_as(ip), ctypes.byref(cnt)),
               "qt_plan_shard")
        pl = cls(h.value, [int(cnt.value)], p, opts.get("dtype", "c64"), [n])
        pl.shard_edges = mine[:cnt.value].copy()
        return pl

    @classmethod
    def create_batch(cls, graphs, p: int, **opts) -> "Plan":
        """``graphs``: sequence of ``(n_vertices, edges)``."""
        ns = np.array([g[0] for g in graphs], dtype=np.int32)
        es = [np.ascontiguousarray(g[1], dtype=np.int32).reshape(-1, 2) for g in graphs]
        ms = np.array([e.shape[0] for e in es], dtype=np.int32)
        allv = np.ascontiguousarray(np.concatenate(es, axis=0))
        o = cls._opts(**opts)
        h = ctypes.c_void_p()
        ip = ctypes.POINTER(ctypes.c_int32)
        _check(lib().qt_plan_batch(len(graphs), ns.ctypes.data_as(ip), ms.ctypes.data_as(ip), allv.ctypes.data_as(ip),
                                   int(p), ctypes.byref(o), ctypes.byref(h)), "qt_plan_batch")
        return cls(h.value, ms.tolist(), p, opts.get("dtype", "c64"), ns.tolist())

    def close(self):
        if self._h is not None and self._h.value and self._owned:
            lib().qt_plan_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- inspection ---------------------------------------------------------------
    def stats(self) -> dict:
        s = PlanStats()
        _check(lib().qt_plan_stats_get(self._h, ctypes.byref(s)), "qt_plan_stats_get")
        d = {k: getattr(s, k) for k, _ in PlanStats._fields_ if k not in ("width_hist", "tile_cap")}
        d["width_hist"] = np.array(list(s.width_hist), dtype=np.int64)
        d["tile_cap"] = [int(x) for x in s.tile_cap[:5]]
        return d

    def export(self):
        st = self.stats()
        b = np.zeros(st["n_buckets"], dtype=BUCKET_DTYPE)
        o = np.zeros(st["n_operands"], dtype=OPERAND_DTYPE)
        _check(lib().qt_plan_export(self._h, b.ctypes.data, o.ctypes.data), "qt_plan_export")
        return b, o

    def network_wires(self, network: int, n_vertices: int) -> np.ndarray:
        out = np.zeros(n_vertices, dtype=np.int32)
        _check(lib().qt_plan_network_wires(self._h, int(network), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
               "qt_plan_network_wires")
        return out

    # -- evaluation ---------------------------------------------------------------
    @property
    def n_networks(self) -> int:
        return int(sum(self.n_edges))

    def export_groups(self) -> np.ndarray:
        """The static work-group queue in claim order (bucket, first_tile, n_tiles, unit_buckets)."""
        n = max(1, self.stats()["n_items"])
        out = np.zeros(n, dtype=GROUP_DTYPE)
        cnt = ctypes.c_int64(0)
        _check(lib().qt_plan_export_groups(self._h, out.ctypes.data, ctypes.byref(cnt)), "qt_plan_export_groups")
        return out[:cnt.value]

    def export_units(self):
        """The fused units (root, n_buckets, first_rec) and the unit program's records (a, b, off)."""
        nu, nr = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(lib().qt_plan_export_units(self._h, None, None, ctypes.byref(nu), ctypes.byref(nr)), "qt_plan_export_units")
        units = np.zeros(max(1, nu.value), dtype=UNIT_DTYPE)
        recs = np.zeros(max(1, nr.value), dtype=UNIT_REC_DTYPE)
        _check(lib().qt_plan_export_units(self._h, units.ctypes.data, recs.ctypes.data, ctypes.byref(nu), ctypes.byref(nr)),
               "qt_plan_export_units")
        return units[:nu.value], recs[:nr.value]

    def export_device(self):
        """The arrays the kernels read: (buckets, operands, net_first_factor, factor, graph_owned)."""
        st = self.stats()
        nf = ctypes.c_int64(0)
        _check(lib().qt_plan_export_device(self._h, None, None, None, None, None, ctypes.byref(nf)),
               "qt_plan_export_device")
        b = np.zeros(max(1, st["n_buckets"]), dtype=DEV_BUCKET_DTYPE)
        o = np.zeros(max(1, st["n_operands"]), dtype=DEV_OPERAND_DTYPE)
        nff = np.zeros(st["n_networks"] + 1, dtype=np.uint32)
        f = np.zeros(max(1, nf.value), dtype=np.uint64)
        go = np.zeros(max(1, st["n_graphs"]), dtype=np.int32)
        _check(lib().qt_plan_export_device(self._h, b.ctypes.data, o.ctypes.data, nff.ctypes.data, f.ctypes.data,
                                           go.ctypes.data, ctypes.byref(nf)), "qt_plan_export_device")
        return b[:st["n_buckets"]], o[:st["n_operands"]], nff, f[:nf.value], go[:st["n_graphs"]]

    def passes(self):
        """The passes of a plan that runs in passes: (pass plan, its graph edges) pairs. The pass
        plans belong to this plan (valid while it is open)."""
        out = []
        for k in range(self.stats()["n_passes"] if self.stats()["pass_arena_bytes"] else 0):
            h = ctypes.c_void_p()
            edges = np.zeros(max(1, sum(self.n_edges)), dtype=np.int32)
            cnt = ctypes.c_int32(0)
            _check(lib().qt_plan_pass(self._h, k, ctypes.byref(h), edges.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      ctypes.byref(cnt)), "qt_plan_pass")
            out.append((Plan(h.value, [cnt.value], self.p, self.dtype, self.n_vertices, owned=False),
                        edges[:cnt.value].copy()))
        return out

    def export_reps(self) -> np.ndarray:
        """Per network, the network whose value it takes (itself when contracted)."""
        out = np.zeros(max(1, self.stats()["n_networks"]), dtype=np.int32)
        _check(lib().qt_plan_export_reps(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
               "qt_plan_export_reps")
        return out[:self.stats()["n_networks"]]

    def export_fixed(self) -> np.ndarray:
        """Fixed gate entries of every slice (network, slice, leaf_kind, leaf_layer, entry)."""
        cnt = ctypes.c_int64(0)
        _check(lib().qt_plan_export_fixed(self._h, None, ctypes.byref(cnt)), "qt_plan_export_fixed")
        out = np.zeros(max(1, cnt.value), dtype=FIXED_DTYPE)
        _check(lib().qt_plan_export_fixed(self._h, out.ctypes.data, ctypes.byref(cnt)), "qt_plan_export_fixed")
        return out[:cnt.value]

    def energy(self, gammas, betas, edge_zz=None, energy=None, stream=None):
        """One graph. With no output buffers given, returns ``(edge_zz, E)`` as host numpy/float.
        Output buffers may be numpy arrays or torch tensors (CUDA or pinned host)."""
        g, b = _f64_in(gammas), _f64_in(betas)
        own = edge_zz is None and energy is None
        if own:
            edge_zz = np.zeros(self.n_networks, dtype=np.float64)
            energy = np.zeros(1, dtype=np.float64)
        _check(lib().qt_energy(self._h, _ptr(g), _ptr(b), _ptr(edge_zz), _ptr(energy), _stream_ptr(stream)),
               "qt_energy")
        if own:
            return edge_zz, float(energy[0])
        return edge_zz, energy

    def energy_batch(self, gammas, betas, energies=None, edge_zz=None, stream=None):
        """Every graph of a batch plan: ``gammas``/``betas`` are (n_graphs, p)."""
        g, b = _f64_in(gammas), _f64_in(betas)
        own = energies is None and edge_zz is None
        if own:
            energies = np.zeros(len(self.n_edges), dtype=np.float64)
            edge_zz = np.zeros(self.n_networks, dtype=np.float64)
        _check(lib().qt_energy_batch(self._h, _ptr(g), _ptr(b), _ptr(energies), _ptr(edge_zz), _stream_ptr(stream)),
               "qt_energy_batch")
        return energies, edge_zz

    def energy_noalloc(self, gammas, betas, energies=None, edge_zz=None, stream=None):
        """Energies through ``qt_energy_noalloc``: the persistent kernel run in the
        library's static device scratch, with no device allocation by the call.
        Works on host-only plans. Returns ``(energies, edge_zz)``; synchronous."""
        g, b = _f64_in(gammas), _f64_in(betas)
        if energies is None and edge_zz is None:
            energies = np.zeros(len(self.n_edges), dtype=np.float64)
            edge_zz = np.zeros(self.n_networks, dtype=np.float64)
        _check(lib().qt_energy_noalloc(self._h, _ptr(g), _ptr(b), _ptr(energies), _ptr(edge_zz),
                                       _stream_ptr(stream)), "qt_energy_noalloc")
        return energies, edge_zz

    def energy_grad(self, gammas, betas, energy=None, dgamma=None, dbeta=None, stream=None):
        g, b = _f64_in(gammas), _f64_in(betas)
        G = len(self.n_edges)
        own = energy is None
        if own:
            energy = np.zeros(G, dtype=np.float64)
            dgamma = np.zeros(G * self.p, dtype=np.float64)
            dbeta = np.zeros(G * self.p, dtype=np.float64)
        _check(lib().qt_energy_grad(self._h, _ptr(g), _ptr(b), _ptr(energy), _ptr(dgamma), _ptr(dbeta),
                                    _stream_ptr(stream)), "qt_energy_grad")
        return energy, dgamma, dbeta

    def last_imag(self) -> np.ndarray:
        out = np.zeros(self.n_networks, dtype=np.float64)
        _check(lib().qt_last_imag(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "qt_last_imag")
        return out

    def sync(self, stream=None):
        _check(lib().qt_sync(self._h, _stream_ptr(stream)), "qt_sync")

    def kernel_time(self, reset: bool = False):
        """(average ms per launch of the main kernel, number of launches timed)."""
        ms = ctypes.c_double(0)
        n = ctypes.c_int64(0)
        _check(lib().qt_kernel_time(self._h, ctypes.byref(ms), ctypes.byref(n), int(reset)), "qt_kernel_time")
        return ms.value, n.value

    def bucket_time(self, bucket: int, reps: int = 5):
        """(mean ms, algorithmic bytes) of the persistent kernel on one bucket alone."""
        ms = ctypes.c_double(0)
        by = ctypes.c_double(0)
        _check(lib().qt_bucket_time(self._h, int(bucket), int(reps), ctypes.byref(ms), ctypes.byref(by)),
               "qt_bucket_time")
        return ms.value, by.value

    def trace_bucket_times(self) -> np.ndarray:
        """(n_buckets, 2) array of start and end times (ns) of the last traced run."""
        nb = self.stats()["n_buckets"]
        out = np.zeros(2 * nb, dtype=np.uint64)
        _check(lib().qt_trace_bucket_times(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))),
               "qt_trace_bucket_times")
        return out.reshape(nb, 2)

    TRACE_PHASES = ("claim", "prep", "deps", "issue", "wait", "compute", "finish", "gate")

    def trace_counters(self) -> dict:
        """Per-phase cycles summed over warps, tile and run counts, warps launched."""
        buf = (ctypes.c_uint64 * 10)()
        nw = ctypes.c_int64(0)
        _check(lib().qt_trace_counters(self._h, buf, ctypes.byref(nw)), "qt_trace_counters")
        d = {k: int(buf[i]) for i, k in enumerate(self.TRACE_PHASES[:7])}
        d["gate"] = int(buf[9])
        d.update(tiles=int(buf[7]), runs=int(buf[8]), warps=int(nw.value))
        return d

    def debug_stall_bucket(self, bucket: int):
        _check(lib().qt_debug_stall_bucket(self._h, int(bucket)), "qt_debug_stall_bucket")


class Contraction:
    """A planned contraction of complex tensors over binary (size-2) indices:
    out[K] = sum over the labels not in K of prod_t T_t[L_t] (qt_contract_*).
    ``labels``: one sequence of non-negative int labels per operand, in C
    order; ``out_labels``: the output's, in C order. Runs on device tensors."""

    def __init__(self, labels, out_labels, dtype="c64", host_only=False):
        self.labels = [list(map(int, L)) for L in labels]
        self.out_labels = list(map(int, out_labels))
        self.dtype = dtype
        ranks = np.array([len(L) for L in self.labels], dtype=np.int32)
        flat = np.array([x for L in self.labels for x in L], dtype=np.int32)
        outl = np.array(self.out_labels if self.out_labels else [0], dtype=np.int32)
        ip = ctypes.POINTER(ctypes.c_int32)
        h = ctypes.c_void_p()
        _check(lib().qt_contract_plan(len(self.labels), ranks.ctypes.data_as(ip), flat.ctypes.data_as(ip),
                                      len(self.out_labels), outl.ctypes.data_as(ip),
                                      {"c64": QT_C64, "c128": QT_C128}[dtype], int(bool(host_only)),
                                      ctypes.byref(h)), "qt_contract_plan")
        self._h = h

    def stats(self) -> dict:
        s = ContractStats()
        _check(lib().qt_contract_stats_get(self._h, ctypes.byref(s)), "qt_contract_stats_get")
        d = {k: getattr(s, k) for k, _ in ContractStats._fields_ if k != "widths"}
        d["widths"] = [int(x) for x in s.widths[:min(32, s.n_buckets)]]
        return d

    def run(self, ops, out, stream=None):
        """ops: contiguous complex CUDA tensors (shapes 2 x ... x 2 of each operand's rank); out: the
        output tensor, written. With a stream the call only enqueues (see ``sync``)."""
        ptrs = (ctypes.c_void_p * len(ops))(*[o.data_ptr() for o in ops])
        _check(lib().qt_contract_run(self._h, ptrs, out.data_ptr(), _stream_ptr(stream)), "qt_contract_run")
        return out

    def sync(self, stream=None):
        _check(lib().qt_contract_sync(self._h, _stream_ptr(stream)), "qt_contract_sync")

    def close(self):
        if self._h is not None and self._h.value:
            lib().qt_contract_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def contraction(labels, out_labels, dtype="c64", host_only=False) -> Contraction:
    return Contraction(labels, out_labels, dtype, host_only)


def plan(n: int, edges, p: int, **opts) -> Plan:
    return Plan.create(n, edges, p, **opts)


def plan_subset(n: int, edges, p: int, sel, **opts) -> Plan:
    return Plan.create_subset(n, edges, p, sel, **opts)


def plan_shard(n: int, edges, p: int, world: int, rank: int, **opts) -> Plan:
    return Plan.create_shard(n, edges, p, world, rank, **opts)


def plan_batch(graphs, p: int, **opts) -> Plan:
    return Plan.create_batch(graphs, p, **opts)


def _autograd_function():
    import torch

    class QAOAEnergy(torch.autograd.Function):
        """E(gamma, beta) of a single-graph gradient plan as a differentiable torch op.

        forward runs qt_energy_grad (the energy and its adjoint in one call) and
        keeps the gradient; backward scales it by the incoming gradient.
        ``gammas`` and ``betas`` are float64 tensors of length p (CPU or CUDA).
        CUDA tensors stay on the device: their pointers and the current stream
        go to the call, which enqueues its work without waiting for it, and the
        energy and gradient are written to CUDA tensors (a kernel-side error
        surfaces at the plan's next synchronous call or ``plan.sync()``).
        """

        @staticmethod
        def forward(ctx, plan, gammas, betas):
            g = gammas.detach().to(torch.float64).contiguous()
            b = betas.detach().to(torch.float64).contiguous()
            if g.is_cuda:
                b = b.to(g.device)
                E = torch.empty(1, dtype=torch.float64, device=g.device)
                dg = torch.empty(plan.p, dtype=torch.float64, device=g.device)
                db = torch.empty(plan.p, dtype=torch.float64, device=g.device)
                plan.energy_grad(g, b, energy=E, dgamma=dg, dbeta=db, stream=torch.cuda.current_stream(g.device))
                ctx.save_for_backward(dg, db.to(betas.device))
                return E[0]
            E, dg, db = plan.energy_grad(g.numpy(), b.cpu().numpy())
            ctx.save_for_backward(torch.as_tensor(dg, dtype=torch.float64, device=gammas.device),
                                  torch.as_tensor(db, dtype=torch.float64, device=betas.device))
            return torch.as_tensor(E[0], dtype=torch.float64, device=gammas.device)

        @staticmethod
        def backward(ctx, grad_out):
            dg, db = ctx.saved_tensors
            return None, grad_out * dg, grad_out * db

    return QAOAEnergy


def qaoa_energy(plan: "Plan", gammas, betas):
    """Differentiable energy: ``qaoa_energy(plan, gammas, betas).backward()`` fills the angle gradients."""
    return _autograd_function().apply(plan, gammas, betas)
