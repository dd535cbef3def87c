#!/usr/bin/env python3
"""QAOA MaxCut energy evaluations per second, one JSON line on rank 0.

Workload (default): the seeded random 3-regular graph N=30 (seed 1000, 45
edges), depth p=4, angles from the seeded generator; one step = one full
energy evaluation E = |E|/2 - 1/2 sum_jk <Z_jZ_k> over all 45 lightcone
networks by bucket elimination, complex64 with FP32 arithmetic (the precision
form). The plain complex128 form is measured beside it under "c128".

* value: device-resident angles and outputs, K steps timed with CUDA events on
  the launch stream (barrier + synchronize on both sides, max over ranks).
  Each step's tensors total several GB, far above the 129 MB L2.
* e2e: the same evaluation through the public API with host angles in and
  host results out, the copies inside the timed region.
* roofline: algorithmic bytes of one evaluation (every operand read once,
  every result written once) over the average duration of the persistent
  bucket kernel, from CUDA events recorded around it on its stream.
* cpu_baseline: one whole evaluation of the same workload (all 45 networks)
  by the CPU oracle's bucket elimination in its own greedy min-fill order, on
  all host cores (rank 0, one GPU only), plus a one-thread estimate.
* summary (the line's last key): the headline figures of every configuration
  in one short object -- complex64 and complex128 evaluations/s, the roofline
  fractions, accuracy, the wide-bucket GB/s, the 64-graph batch against the
  plain per-bucket complex128 form, the N=50 p=4 gradient rate.

``--impl reference`` times the CPU oracle alone (there is no reference code
base; the oracle stands in for it) and prints its line with "impl": "reference".
Multi-GPU (torchrun): the graph's networks (their slices) are split over the
ranks by longest-processing-time on their cost and each step ends with one
all-reduce of the partial energy (strong scaling); ``--replicas`` runs an
independent copy per rank instead (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

PAPER_SECONDS_PER_EVAL = 1.4  # best mixed merged backend, N=30 p=4, V100 (Table II)
REF_TIMED_BUDGET_S = 150.0    # the reference arm's timed steps together, about (cost-weighted groups per step)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["c2", "c3", "c5", "tncontract"], default="c2",
                    help="c2: the headline line (N=30 p=4 evals/s, plus wide-bucket GB/s on N=1000 p=5, the "
                         "batch, gradient and random-contraction legs); c3: 64-graph batch; c5: gradients on "
                         "N=50 p=4; tncontract: the paper's random contraction expressions against torch.einsum")
    ap.add_argument("--c3-skip-plain", action="store_true",
                    help="--workload c3: skip the plain per-bucket complex128 form (profiler captures)")
    ap.add_argument("--c5-n", type=int, default=50,
                    help="--workload c5: vertices of the random 3-regular graph (50; smaller for profiler captures)")
    ap.add_argument("--no-buckets", action="store_true", help="skip the wide-bucket GB/s measurement")
    ap.add_argument("--no-autotune", action="store_true", help="skip the plan-time autotuner's line")
    ap.add_argument("--no-alt", action="store_true", help="skip the alternative plan (the plain greedy order)")
    ap.add_argument("--replicas", action="store_true",
                    help="with N GPUs: every rank evaluates its own copy of the workload (weak scaling); default: "
                         "the graph's networks split over the ranks by LPT on cost, one all-reduce per step")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the 64-graph batch and gradient legs of the summary")
    return ap.parse_args()


WORKLOAD = dict(n=30, seed=1000, p=4)


def workload_inputs():
    from paper_2204_06045_gb300 import synth
    n, seed, p = WORKLOAD["n"], WORKLOAD["seed"], WORKLOAD["p"]
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    return n, p, edges, g, b


def config_dict(dtype_note: str):
    n, seed, p = WORKLOAD["n"], WORKLOAD["seed"], WORKLOAD["p"]
    return {"workload": f"QAOA MaxCut energy, random 3-regular N={n} (seed {seed}, 45 edges), p={p}, "
                        f"all 45 lightcone networks by bucket elimination, {dtype_note}",
            "graph_seed": seed, "n_vertices": n, "p": p, "angles": "synth.angles(p, seed)",
            "l2": "no flush: each evaluation reads and writes several GB of tensors (L2 is 129 MB)"}


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ----------------------------------------------------------------------------- CPU oracle

def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in Path("/proc/cpuinfo").read_text().splitlines():
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_networks(nets):
    """Seconds the oracle takes for each network in `nets` of the workload (complex128 bucket
    elimination in the oracle's own greedy min-fill order), on its current thread count."""
    import oracle
    n, p, edges, g, b = workload_inputs()
    out = []
    for e in nets:
        t0 = time.perf_counter()
        oracle.edge_bucket_min_fill(n, edges, g, b, int(e), seed=int(e), max_width=31)
        out.append(time.perf_counter() - t0)
    return np.array(out)


def cpu_baseline(one_thread_budget_s: float = 4.0):
    """One whole evaluation (every network) on all host cores, timed; and a one-thread figure
    estimated from the cheapest networks, weighted by their share of the all-core time."""
    import oracle
    oracle.build()
    cores = oracle.get_threads()
    n, p, edges, g, b = workload_inputs()
    m = edges.shape[0]
    t = oracle_networks(range(m))
    total = float(t.sum())
    order = np.argsort(t)
    picked, acc = [], 0.0
    for e in order:  # cheapest first, within the budget at ~cores times the all-core time
        if picked and acc + t[e] * cores > one_thread_budget_s:
            break
        picked.append(int(e))
        acc += t[e] * cores
    oracle.set_threads(1)
    try:
        t1 = float(oracle_networks(picked).sum())
    finally:
        oracle.set_threads(cores)
    share = float(t[picked].sum()) / total
    return {"value": 1.0 / total, "unit": "evals/s", "cores": cores, "kind": "oracle",
            "sample": f"one whole evaluation: all {m} lightcone networks, complex128 bucket elimination "
                      f"(oracle, its greedy min-fill order) on {cores} threads in {total:.2f} s",
            "nproc": os.cpu_count(), "cpu_model": cpu_model(),
            "one_thread": {"value": share / t1 if t1 > 0 else None, "unit": "evals/s",
                           "sample": f"{len(picked)} cheapest networks ({100 * share:.2f}% of the all-core time) on "
                                     f"1 thread in {t1:.2f} s, scaled by that share (an estimate)"}}


def run_reference(args, rank, world):
    """The CPU oracle on the same workload. The first warm-up step is one whole
    evaluation whose per-network times split the networks into G groups of
    about equal cost (longest first); each further step evaluates the next
    group, and a step counts as its group's share of the whole evaluation, so
    the K timed steps stay within about REF_TIMED_BUDGET_S."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    n, p, edges, g, b = workload_inputs()
    m = edges.shape[0]
    calib = oracle_networks(range(m))  # warm-up step 1: a whole evaluation
    total = float(calib.sum())
    G = max(1, min(m, int(np.ceil(args.steps * total / REF_TIMED_BUDGET_S))))
    groups = [[] for _ in range(G)]
    load = np.zeros(G)
    for e in np.argsort(-calib):
        k = int(np.argmin(load))
        groups[k].append(int(e))
        load[k] += calib[e]
    share = load / total
    for w in range(1, args.warmup):
        oracle_networks(groups[w % G])
    times, done = [], 0.0
    for s in range(args.steps):
        times.append(float(oracle_networks(groups[s % G]).sum()))
        done += share[s % G]
    total_t = sum(times)
    value = done / total_t
    cores = oracle.get_threads()
    sample = (f"{m} networks split into {G} groups of about equal oracle time (from a whole evaluation in the first "
              f"warm-up step, {total:.2f} s on {cores} threads); step k evaluates group k mod {G} and counts as its "
              f"share of an evaluation; evals/s = sum of shares / time")
    line = {"impl": "reference", "metric": "QAOA energy evals/s (3-reg N=30 p=4)", "value": value, "unit": "evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": value * PAPER_SECONDS_PER_EVAL, "dtype": "c128", "data": "synthetic",
            "config": config_dict("complex128 CPU oracle, bucket elimination in its greedy min-fill order"),
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle", "sample": sample,
                             "nproc": os.cpu_count(), "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU

def measured_peaks():
    f = ROOT / "MEASURED_PEAKS.json"
    if f.exists():
        d = json.loads(f.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


FORWARD_SOURCES = ("kernels.cu", "device_common.cuh", "kernels.hpp", "qt_internal.hpp")


def forward_source_sha() -> str:
    """Hash of the sources the forward kernels are built from (a profile summary
    records it; its DRAM figures are used only while the sources match)."""
    h = hashlib.sha256()
    for name in FORWARD_SOURCES:
        h.update((ROOT / "paper_2204_06045_gb300" / "csrc" / name).read_bytes())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_tag: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the current kernel source."""
    f = ROOT / "profiles" / f"{kernel_tag}.txt"
    if not f.exists():
        return None
    sha = forward_source_sha()
    vals = {}
    for line in f.read_text().splitlines():
        parts = line.split()
        if len(parts) == 2 and not line.startswith("#"):
            vals[parts[0]] = parts[1]
    if vals.get("forward_src_sha256_16") != sha:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def golden_c4():
    """Per-edge <Z_jZ_k> of the N=1000 p=5 graph from the stored oracle values (dict edge -> value)."""
    f = ROOT / "tests" / "golden" / "c4_n1000_p5_bucket.txt"
    if not f.exists():
        return None
    ref = {}
    for line in f.read_text().splitlines():
        parts = line.split()
        if parts and parts[0] == "edge":
            ref[int(parts[1])] = float(parts[4])
    return ref


def golden_c2():
    """Per-edge <Z_jZ_k> and E of the default workload from the stored 2^30 state-vector values."""
    f = ROOT / "tests" / "golden" / "c2_n30_p4_statevector.txt"
    if not f.exists():
        return None, None
    zz, E = [], None
    for line in f.read_text().splitlines():
        parts = line.split()
        if parts and parts[0] == "edge":
            zz.append(float(parts[4]))
        elif parts and parts[0] == "energy":
            E = float(parts[1])
    return np.array(zz), E


def accuracy(zz, E, ref_zz, ref_E):
    """Errors against the stored state vector. `max_scaled_err_zz` is |d e| / max(|e|, 1e-2), the
    survey's measure; the tests bound the relative error of each edge's energy (1 - e)/2 and the
    absolute error of e (the adopted reading); both are printed."""
    if ref_zz is None:
        return {"reference": "unavailable"}
    d = np.abs(np.asarray(zz) - ref_zz)
    return {"reference": "2^30 complex128 state vector (oracle, stored)",
            "max_abs_err_zz": float(d.max()),
            "max_rel_err_zz": float(np.max(d / np.abs(ref_zz))),
            "max_scaled_err_zz": float(np.max(d / np.maximum(np.abs(ref_zz), 1e-2))),
            "max_rel_err_edge_energy": float(np.max(d / np.abs(1.0 - ref_zz))),
            "rel_err_energy": float(abs(E - ref_E) / abs(ref_E))}


def roofline(dtype, st, kms, launches, achieved_gbs, peak_gbs, peak_kind, fma_tflops, traffic):
    """complex64: HBM-bound (FP32 arithmetic is ~1-3 flop/byte, far below the ridge). complex128:
    FP64 arithmetic bound on GB300 (its FP64 rate is below 1 flop per byte of HBM bandwidth), so the
    line reports flops against the measured FP64 FMA rate and keeps the HBM figures beside it."""
    tflops = st["flops"] / (kms * 1e-3) / 1e12 if kms > 0 else None
    common = {"kernel": "k_persistent", "kernel_ms": kms, "kernel_launches": launches,
              "alg_bytes_per_launch": st["alg_bytes"], "flops_per_launch": st["flops"]}
    hbm = {"achieved": achieved_gbs, "peak": peak_gbs, "unit": "GB/s",
           "frac": achieved_gbs / peak_gbs if achieved_gbs else None, "peak_source": peak_kind}
    alu = {"achieved": tflops, "peak": fma_tflops, "unit": "TFLOP/s",
           "frac": tflops / fma_tflops if tflops else None,
           "peak_source": f"measured {'FP64' if dtype == 'c128' else 'FP32'} FMA rate (qt_fma_peak)"}
    if dtype == "c128":
        return {"bound": "alu", **alu, "traffic": traffic, "hbm": hbm, **common}
    return {"bound": "hbm", **hbm, "traffic": traffic, "alu": alu, **common}


def wide_buckets(peak, torch):
    """HBM GB/s of the persistent kernel on every bucket of width >= 24, each run alone.

    Workload: random 3-regular N=1000 (seed 1000), p=5; the lightcone networks
    of the edges whose plain greedy order reaches a maximum bucket width of
    26..28 (chosen on a host-only plan of every edge). The per-bucket and
    per-network bandwidths are those of plain buckets (one summed variable
    each, no merging, no slicing): a merged bucket moves fewer bytes for the
    same work. The times of the same networks with merged eliminations, and
    with the default plan (merged and sliced), are reported beside them."""
    from paper_2204_06045_gb300 import qtgb, synth
    n, p, seed = 1000, 5, 1000
    edges = synth.random_regular_graph(n, seed)
    g, b = synth.angles(p, seed)
    with qtgb.plan(n, edges, p, host_only=True, slice_width=-1, restarts=-1) as hp:
        B, _ = hp.export()
    mw = np.zeros(edges.shape[0], dtype=np.int64)
    np.maximum.at(mw, B["network"], B["width"])
    sel = np.nonzero((mw >= 26) & (mw <= 28))[0]
    out = {"workload": f"3-regular N={n} seed {seed}, p={p}: {sel.size} lightcone networks with greedy max width "
                       f"26..28; every bucket of width >= 24, timed alone (mean of 3 launches after 1)",
           "edges": sel.tolist()}
    ref = golden_c4()
    for dtype in ("c64", "c128"):
        with qtgb.plan_subset(n, edges, p, sel, dtype=dtype, merge=False, slice_width=-1, restarts=-1) as pl:
            zz, _ = pl.energy(g, b)  # also leaves real data in every operand
            if ref is not None:
                want = np.array([ref[int(e)] for e in sel])
                d = np.abs(zz - want)
                out.setdefault("check", {})[dtype] = {
                    "reference": "oracle complex128 bucket elimination, min-fill order (stored)",
                    "max_abs_err_zz": float(d.max()), "max_rel_err_zz": float((d / np.abs(want)).max()),
                    "max_rel_err_edge_energy": float((d / np.abs(1.0 - want)).max())}
            Bs, _ = pl.export()
            tot_b = tot_ms = 0.0
            per = []
            for bk in np.nonzero(Bs["width"] >= 24)[0]:
                ms, by = pl.bucket_time(int(bk), reps=3)
                tot_b += by
                tot_ms += ms
                per.append(by / ms / 1e6)
        agg = tot_b / tot_ms / 1e6
        out[dtype] = {"buckets": len(per), "agg_gbs": agg, "median_gbs": float(np.median(per)),
                      "max_gbs": float(np.max(per)), "min_gbs": float(np.min(per)), "frac_of_peak": agg / peak,
                      "bytes": tot_b, "ms": tot_ms}
        # single-edge contraction: each network alone in its own plan, every bucket of it in one
        # persistent launch; algorithmic bytes of the network over the kernel's time
        tot = {}
        variants = {"plain": dict(merge=False, slice_width=-1, restarts=-1), "merged": dict(slice_width=-1, restarts=-1),
                    "default": {}}
        for key, kw in variants.items():
            nb = nm = 0.0
            for e in sel:
                with qtgb.plan_subset(n, edges, p, [int(e)], dtype=dtype, **kw) as one:
                    for _ in range(2):
                        one.energy(g, b)
                    one.kernel_time(reset=True)
                    for _ in range(3):
                        one.energy(g, b)
                    ms, _ = one.kernel_time(reset=True)
                    nb += one.stats()["alg_bytes"]
                    nm += ms
            tot[key] = (nb, nm)
        nb, nm = tot["plain"]
        out[dtype]["networks"] = {"count": int(sel.size), "agg_gbs": nb / nm / 1e6, "frac_of_peak": nb / nm / 1e6 / peak,
                                  "bytes": nb, "ms": nm,
                                  "note": "each network alone, plain buckets: all its buckets in one persistent launch "
                                          "(mean of 3 after 2)"}
        mb, mm = tot["merged"]
        out[dtype]["networks_merged"] = {"ms": mm, "bytes": mb, "agg_gbs": mb / mm / 1e6, "speedup_vs_plain": nm / mm,
                                         "note": "the same networks with merged eliminations"}
        db, dm = tot["default"]
        out[dtype]["networks_default"] = {"ms": dm, "bytes": db, "agg_gbs": db / dm / 1e6, "speedup_vs_plain": nm / dm,
                                          "note": "the same networks with the default plan: merged eliminations and "
                                                  "index slicing"}
    return out


_LETTERS = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"


def tncontract_leg(torch, n_expr=24, reps=5):
    """The paper's "tncontract random" benchmark (§II-E; Table III, Tensor Network
    Random Contraction): seeded random expressions of 4..25 indices of size 2
    (synth.tncontract_random, seeds 0..n_expr-1), complex64, each run through
    qt_contract (permuting copies in, the bucket-elimination kernel, the copy out)
    and through torch.einsum on the same GPU, both from device tensors to a device
    tensor; CUDA events on one stream, mean of `reps` after 2. FLOP rate in the
    paper's convention: 8 x 2^(distinct indices) per contraction / time."""
    from paper_2204_06045_gb300 import qtgb, synth
    rows = []
    s = torch.cuda.current_stream()
    for k in range(n_expr):
        la, lb, lo = synth.tncontract_random(k)
        n = len(la)
        gen = torch.Generator(device="cuda").manual_seed(k)
        A = torch.randn((2,) * n, dtype=torch.complex64, device="cuda", generator=gen)
        B = torch.randn((2,) * len(lb), dtype=torch.complex64, device="cuda", generator=gen)
        spec = "".join(_LETTERS[x] for x in la) + "," + "".join(_LETTERS[x] for x in lb) + "->" + \
            "".join(_LETTERS[x] for x in lo)
        out = torch.empty((2,) * len(lo), dtype=torch.complex64, device="cuda")
        with qtgb.contraction([la, lb], lo, dtype="c64") as c:
            st = c.stats()
            for _ in range(2):
                c.run([A, B], out, stream=s)
            c.sync(s)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                c.run([A, B], out, stream=s)
            e1.record(s)
            c.sync(s)
            ms = e0.elapsed_time(e1) / reps
        for _ in range(2):
            ref = torch.einsum(spec, A, B)
        e0.record(s)
        for _ in range(reps):
            ref = torch.einsum(spec, A, B)
        e1.record(s)
        torch.cuda.synchronize()
        ms_lib = e0.elapsed_time(e1) / reps
        diff = float((out - ref).abs().max() / ref.abs().max().clamp_min(1.0))
        rows.append({"indices": n, "summed": n - len(lo), "b_rank": len(lb), "ms": ms, "einsum_ms": ms_lib,
                     "buckets": st["n_buckets"], "gbs": (st["alg_bytes"] + st["copy_bytes"]) / ms / 1e6,
                     "paper_gflops": 8.0 * 2.0 ** n / ms / 1e6, "max_rel_diff_vs_einsum": diff})
    big = [r for r in rows if r["indices"] >= 20]
    ours, lib = sum(r["ms"] for r in big), sum(r["einsum_ms"] for r in big)
    top = max(rows, key=lambda r: r["indices"])
    return {"workload": f"{n_expr} random expressions (synth.tncontract_random seeds 0..{n_expr - 1}: 4..25 indices, "
                        "the first tensor holding all, the second the contracted ones and some result indices), "
                        "complex64, device tensors in and out",
            "einsum_time_over_ours_20plus": lib / ours if ours > 0 else None, "expressions_20plus": len(big),
            "ms_20plus": ours, "einsum_ms_20plus": lib,
            "largest": {k: top[k] for k in ("indices", "ms", "einsum_ms", "paper_gflops", "gbs")},
            "max_rel_diff_vs_einsum": max(r["max_rel_diff_vs_einsum"] for r in rows), "rows": rows}


def run_tncontract(args, world, local_rank):
    """--workload tncontract: the random-expression comparison as its own line."""
    import torch
    from paper_2204_06045_gb300 import build
    torch.cuda.set_device(local_rank)
    build.build()
    res = tncontract_leg(torch, n_expr=24, reps=max(1, min(args.steps, 20)))
    line = {"metric": "tncontract random (paper §II-E): torch.einsum time / this library's time, expressions of "
                      ">= 20 indices",
            "value": res["einsum_time_over_ours_20plus"], "unit": "x", "n_gpus": 1, "steps": args.steps,
            "warmup": 2, "higher_is_better": True, "dtype": "c64", "data": "synthetic",
            "config": {"workload": res["workload"]}, "tncontract": res}
    print(json.dumps(line), flush=True)


def alt_plans(n, p, edges, g, b, ref_zz, default, torch):
    """Beside the headline (which it does not change): the same workload planned
    with the plain greedy min-fill order (no restarts; the default plan restarts
    the order 64 times for every network whose greedy order reaches width 18).
    Each entry records its kernel time, bytes and agreement, or the error it met."""
    from paper_2204_06045_gb300 import qtgb
    m = edges.shape[0]
    out = {}
    for dtype, steps in (("c64", 100), ("c128", 20)):
        try:
            with qtgb.plan(n, edges, p, dtype=dtype, restarts=-1) as pl:
                st = pl.stats()
                gd = torch.tensor(g, dtype=torch.float64, device="cuda")
                bd = torch.tensor(b, dtype=torch.float64, device="cuda")
                zz = torch.zeros(m, dtype=torch.float64, device="cuda")
                E = torch.zeros(1, dtype=torch.float64, device="cuda")
                ms, kms, _ = time_device(pl, gd, bd, zz, E, steps, 3, None, torch)
                err = float(np.max(np.abs(zz.cpu().numpy() - ref_zz))) if ref_zz is not None else None
            out[f"plain_greedy_{dtype}"] = {
                "ms_per_step": ms / steps, "kernel_ms": kms, "alg_bytes": st["alg_bytes"],
                "plan_seconds": st["plan_seconds"],
                "default_kernel_ms": default[dtype]["roofline"]["kernel_ms"],
                "default_alg_bytes": default[dtype]["roofline"]["alg_bytes_per_launch"],
                "default_plan_seconds": default[dtype]["plan"]["plan_seconds"], "max_abs_err_zz": err}
        except Exception as ex:  # recorded, not fatal: the headline stands without it
            out[f"plain_greedy_{dtype}"] = {"error": repr(ex)}
    return out


def time_device(pl, gd, bd, zz, E, steps, warmup, dist, torch):
    s = torch.cuda.current_stream()
    for _ in range(warmup):
        pl.energy(gd, bd, edge_zz=zz, energy=E, stream=s)
    pl.sync(s)
    pl.kernel_time(reset=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(s)
    for _ in range(steps):
        pl.energy(gd, bd, edge_zz=zz, energy=E, stream=s)
    ev1.record(s)
    torch.cuda.synchronize()
    pl.sync(s)
    ms = ev0.elapsed_time(ev1)
    kms, launches = pl.kernel_time(reset=True)
    return ms, kms, launches


def time_e2e(pl, g, b, steps, dist, torch):
    for _ in range(2):
        pl.energy(g, b)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        zz, E = pl.energy(g, b)  # host arrays in, host results out; the call waits for its copies
    return time.perf_counter() - t0


def max_over_ranks(x, dist, torch):
    """The slowest rank's value (the whole job's time): an all-reduce MAX over
    the process group (NCCL on GPUs, gloo on CPU)."""
    if dist is None:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, seconds):
    """Weak scaling: every rank processes its own units; the job's rate is all
    ranks' units over the slowest rank's time."""
    return world * units_per_rank / seconds


def c3_leg(torch, steps):
    """The 64-graph batch (random 3-regular, N even in [50, 1000], p=3, per-graph angles):
    every network in one persistent complex64 launch, with and without lightcone
    deduplication; beside it the plain form -- complex128, one launch per bucket -- on every
    eighth graph, with the batched complex64 form timed on the same eight graphs."""
    from paper_2204_06045_gb300 import qtgb, synth
    graphs = synth.batch(64, 3, lo=50, hi=1000, base_seed=1000)
    spec = [(nn, e) for nn, e, _, _ in graphs]
    G = np.array([gg for _, _, gg, _ in graphs])
    Bt = np.array([bb for _, _, _, bb in graphs])

    def timed(sel, reps, warm, **kw):
        with qtgb.plan_batch([spec[i] for i in sel], 3, **kw) as pl:
            st = pl.stats()
            gd = torch.tensor(G[sel].ravel(), dtype=torch.float64, device="cuda")
            bd = torch.tensor(Bt[sel].ravel(), dtype=torch.float64, device="cuda")
            en = torch.zeros(len(sel), dtype=torch.float64, device="cuda")
            s = torch.cuda.current_stream()
            for _ in range(warm):
                pl.energy_batch(gd, bd, energies=en, stream=s)
            pl.sync(s)
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
            ev[0].record(s)
            for i in range(reps):
                pl.energy_batch(gd, bd, energies=en, stream=s)
                ev[i + 1].record(s)
            torch.cuda.synchronize()
            pl.sync(s)
            steps_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(reps)]
            st = dict(st, max_step_ms=max(steps_ms))
            return ev[0].elapsed_time(ev[reps]) / reps, en.cpu().numpy(), st

    every = list(range(64))
    sub = list(range(0, 64, 8))
    with ClockSampler(torch.cuda.current_device()) as clk:
        ms, en, st = timed(every, steps, 3, dtype="c64")
    ms_d, en_d, st_d = timed(every, steps, 3, dtype="c64", dedup=True)
    ms_p, en_p, st_p = timed(sub, 1, 1, dtype="c128", sched="per_bucket")
    ms_s, en_s, _ = timed(sub, steps, 3, dtype="c64")
    return {"workload": "64 random 3-regular graphs, N even in [50,1000] (synth.batch, seed 1000+g), p=3",
            "c64_graph_evals_per_s": 64e3 / ms, "c64_ms_per_batch": ms, "c64_max_step_ms": st["max_step_ms"],
            "c64_clocks": clk.summary(), "buckets": int(st["n_buckets"]),
            "c64_dedup_graph_evals_per_s": 64e3 / ms_d, "dedup_networks_contracted": int(st_d["n_unique"]),
            "dedup_max_rel_energy_diff": float(np.max(np.abs(en_d - en) / np.abs(en))),
            "plain_subset": "graphs 0, 8, ..., 56",
            "plain_c128_per_bucket_graph_evals_per_s": 8e3 / ms_p, "plain_launches": int(st_p["n_buckets"]),
            "c64_batched_same_subset_graph_evals_per_s": 8e3 / ms_s,
            "speedup_batched_c64_vs_plain_c128": ms_p / ms_s,
            "max_rel_energy_diff_c64_vs_c128": float(np.max(np.abs(en_s - en_p) / np.abs(en_p)))}


def c5_leg():
    """Energy and its 2p angle derivatives on random 3-regular N=50 (seed 1000), p=4, by the
    adjoint of the bucket elimination (host arrays in and out), complex64 and complex128; and
    the gradient of 8 sampled edges' energy share against the oracle's central differences."""
    from paper_2204_06045_gb300 import qtgb, synth
    n, p = 50, 4
    edges = synth.random_regular_graph(n, 1000)
    g, b = synth.angles(p, 1000)
    out = {"workload": "random 3-regular N=50 seed 1000, p=4: energy + dE/dgamma_k, dE/dbeta_k"}
    grads = {}
    for dtype, steps in (("c64", 10), ("c128", 3)):
        with qtgb.plan(n, edges, p, dtype=dtype, with_grad=True) as pl:
            for _ in range(2):
                pl.energy_grad(g, b)
            t0 = time.perf_counter()
            for _ in range(steps):
                E, dg, db = pl.energy_grad(g, b)
            dt = (time.perf_counter() - t0) / steps
        out[f"{dtype}_grad_evals_per_s"] = 1.0 / dt
        grads[dtype] = np.concatenate([dg, db])
    out["c64_vs_c128_max_abs_diff"] = float(np.max(np.abs(grads["c64"] - grads["c128"])))
    f = ROOT / "tests" / "golden" / "c5_n50_p4_fd.txt"
    if f.exists():
        rows = {}
        for line in f.read_text().splitlines():
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                rows[k] = np.array([float(x) for x in v])
        ref = np.concatenate([rows["dE_dgamma"], rows["dE_dbeta"]])
        for dtype in ("c64", "c128"):
            with qtgb.plan_subset(n, edges, p, rows["edges"].astype(np.int32), dtype=dtype, with_grad=True) as pl:
                _, dg, db = pl.energy_grad(g, b)
            out[f"{dtype}_subset_vs_oracle_fd_max_abs"] = float(np.max(np.abs(np.concatenate([dg, db]) - ref)))
    return out


def summarize(line):
    """The headline figures of every configuration, short enough to read at the end of the line."""
    r, c = line["roofline"], line["c128"]
    s = {"c2_c64_evals_per_s": line["value"], "c2_c64_kernel_ms": r["kernel_ms"], "c2_c64_hbm_frac": r["frac"],
         "c2_c64_e2e_evals_per_s": line["e2e"]["value"],
         "c2_c128_evals_per_s": c["value"], "c2_c128_kernel_ms": c["roofline"]["kernel_ms"],
         "c2_c128_fp64_frac": c["roofline"]["frac"]}
    for dt, chk in (("c64", line["check"]), ("c128", c["check"])):
        s[f"c2_{dt}_max_abs_err_zz"] = chk.get("max_abs_err_zz")
        s[f"c2_{dt}_max_scaled_err_zz"] = chk.get("max_scaled_err_zz")
        s[f"c2_{dt}_max_rel_err_edge_energy"] = chk.get("max_rel_err_edge_energy")
    wb = line.get("bucket_gbs")
    if wb and "c64" in wb:
        s["wide_buckets_c64"] = {k: wb["c64"][k] for k in ("buckets", "agg_gbs", "frac_of_peak", "median_gbs", "min_gbs")}
        s["wide_buckets_c128_agg_gbs"] = wb["c128"]["agg_gbs"]
    if "c3" in line:
        s["c3"] = {k: line["c3"][k] for k in ("c64_graph_evals_per_s", "c64_dedup_graph_evals_per_s",
                                              "plain_c128_per_bucket_graph_evals_per_s",
                                              "c64_batched_same_subset_graph_evals_per_s",
                                              "speedup_batched_c64_vs_plain_c128")}
    if "c5" in line:
        s["c5"] = {k: v for k, v in line["c5"].items() if k != "workload"}
    if "tncontract" in line:
        s["tncontract"] = {k: line["tncontract"][k] for k in ("einsum_time_over_ours_20plus", "expressions_20plus",
                                                             "largest", "max_rel_diff_vs_einsum")}
    alt = line.get("alt_plans", {}).get("plain_greedy_c64", {})
    if "kernel_ms" in alt:
        s["plain_greedy_order_c64_kernel_ms"] = alt["kernel_ms"]
        s["plain_greedy_order_c64_alg_gb"] = alt["alg_bytes"] / 1e9
    if "cpu_baseline" in line:
        s["cpu_oracle_evals_per_s"] = line["cpu_baseline"]["value"]
    return s


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2204_06045_gb300 import build, qtgb

    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        dist = tdist
    torch.cuda.set_device(local_rank)
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    build.build()

    n, p, edges, g, b = workload_inputs()
    m = edges.shape[0]
    peak, peak_kind = measured_peaks()
    ref_zz, ref_E = golden_c2()
    fma_tflops = {"c64": qtgb.fma_peak("c64"), "c128": qtgb.fma_peak("c128")}
    results = {}
    for dtype in ("c64", "c128"):
        pl = qtgb.plan(n, edges, p, dtype=dtype)
        st = pl.stats()
        gd = torch.tensor(g, dtype=torch.float64, device="cuda")
        bd = torch.tensor(b, dtype=torch.float64, device="cuda")
        zz = torch.zeros(m, dtype=torch.float64, device="cuda")
        E = torch.zeros(1, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        with ClockSampler(local_rank) as clk:
            ms, kms, launches = time_device(pl, gd, bd, zz, E, args.steps, args.warmup, dist, torch)
        ms = max_over_ranks(ms, dist, torch)
        e2e_s = max_over_ranks(time_e2e(pl, g, b, args.steps, dist, torch), dist, torch)
        achieved = st["alg_bytes"] / (kms * 1e-3) / 1e9 if kms > 0 else None
        tag = f"k_persistent_{dtype}_n30_p4"
        results[dtype] = {
            "value": job_throughput(world, args.steps, ms * 1e-3),
            "ms_per_step": ms / args.steps,
            "e2e": {"value": job_throughput(world, args.steps, e2e_s), "unit": "evals/s",
                    "h2d_bytes_per_step": 2 * p * 8, "d2h_bytes_per_step": (m + 1) * 8},
            "roofline": roofline(dtype, st, kms, launches, achieved, peak, peak_kind, fma_tflops[dtype],
                                 ncu_traffic(tag)),
            "clocks": clk.summary(),
            "plan": {"buckets": st["n_buckets"], "merged_buckets": int((pl.export()[0]["n_sum"] > 1).sum()),
                     "slices": st["n_slices"], "slice_bits": st["slice_bits"], "fused_units": st["n_units"],
                     "max_width": st["max_width"], "sum_2w": st["sum_2w"],
                     "tasks": st["n_tasks"], "plan_seconds": st["plan_seconds"]},
            "check": dict(energy=float(E.item()), **accuracy(zz.cpu().numpy(), float(E.item()), ref_zz, ref_E)),
        }
        pl.close()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    main = results["c64"]
    line = {
        "metric": "QAOA energy evals/s (3-reg N=30 p=4)",
        "value": main["value"], "unit": "evals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": main["value"] * PAPER_SECONDS_PER_EVAL, "dtype": "c64", "data": "synthetic",
        "config": config_dict("complex64 with FP32 arithmetic, persistent dependency-queue kernel, "
                              "merged eliminations, index slicing to width 22 (complex128: 20)"),
        "e2e": main["e2e"], "roofline": main["roofline"], "clocks": main["clocks"],
        "gpu_launches": 3 * args.steps,
        "plan": main["plan"], "check": main["check"],
        "c128": {k: results["c128"][k] for k in ("value", "ms_per_step", "e2e", "roofline", "clocks", "plan", "check")},
    }
    if world == 1 and not args.no_autotune:
        # the plan-time autotuner on the same workload: what it chooses and the kernel time it gets
        t = time.perf_counter()
        with qtgb.plan(n, edges, p, dtype="c64", autotune=3) as tp:
            st = tp.stats()
            tg = torch.tensor(g, dtype=torch.float64, device="cuda")
            tb = torch.tensor(b, dtype=torch.float64, device="cuda")
            _, kms_t, _ = time_device(tp, tg, tb, torch.zeros(m, dtype=torch.float64, device="cuda"),
                                      torch.zeros(1, dtype=torch.float64, device="cuda"), 50, 3, None, torch)
        line["autotune_c64"] = {"tile_cap_by_width_class": st["tile_cap"], "run_tiles": st["run_tiles"],
                                "candidates": st["tune_candidates"], "plan_seconds": time.perf_counter() - t,
                                "kernel_ms": kms_t, "default_kernel_ms": main["roofline"]["kernel_ms"]}
    if world == 1 and not args.no_alt:
        line["alt_plans"] = alt_plans(n, p, edges, g, b, ref_zz, {"c64": main, "c128": results["c128"]}, torch)
    if world == 1 and not args.no_buckets:
        line["bucket_gbs"] = wide_buckets(peak, torch)
    if world == 1 and not args.no_extra:
        line["c3"] = c3_leg(torch, min(args.steps, 20))
        line["c5"] = c5_leg()
        line["tncontract"] = tncontract_leg(torch)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    line["summary"] = summarize(line)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_c3(args, world, local_rank):
    """64 seeded graphs, N ~ U{50..1000} even, p=3, per-graph angles: one persistent launch per batch."""
    import torch
    from paper_2204_06045_gb300 import build, qtgb, synth
    torch.cuda.set_device(local_rank)
    build.build()
    graphs = synth.batch(64, 3, lo=50, hi=1000, base_seed=1000)
    G = np.array([g for _, _, g, _ in graphs])
    Bt = np.array([b for _, _, _, b in graphs])
    res = {}
    legs = [("c64", "persistent", args.steps, False), ("c128", "persistent", args.steps, False),
            ("c128", "per_bucket", 1, False), ("c64", "persistent", args.steps, True)]
    if args.c3_skip_plain:
        legs = [leg for leg in legs if leg[1] != "per_bucket"]
    for dtype, sched, steps, dedup in legs:
        with qtgb.plan_batch([(n, e) for n, e, _, _ in graphs], 3, dtype=dtype, sched=sched, dedup=dedup) as pl:
            st = pl.stats()
            gd = torch.tensor(G.ravel(), dtype=torch.float64, device="cuda")
            bd = torch.tensor(Bt.ravel(), dtype=torch.float64, device="cuda")
            en = torch.zeros(64, dtype=torch.float64, device="cuda")
            s = torch.cuda.current_stream()
            for _ in range(1 if sched == "per_bucket" else args.warmup):
                pl.energy_batch(gd, bd, energies=en, stream=s)
            pl.sync(s)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(steps):
                pl.energy_batch(gd, bd, energies=en, stream=s)
            e1.record(s)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            res[f"{dtype}_{sched}" + ("_dedup" if dedup else "")] = {
                "ms_per_step": ms, "graph_evals_per_s": 64 / (ms * 1e-3), "steps": steps,
                "buckets": st["n_buckets"], "alg_bytes": st["alg_bytes"], "networks_contracted": st["n_unique"]}
    # accuracy: 64 seeded sample edges against the oracle's bucket elimination of their networks
    import oracle
    rng = np.random.default_rng(7)
    first = np.cumsum([0] + [e.shape[0] for _, e, _, _ in graphs])
    flat = np.sort(rng.choice(first[-1], size=64, replace=False))
    with qtgb.plan_batch([(n_, e) for n_, e, _, _ in graphs], 3, dtype="c64") as pl:
        _, zz = pl.energy_batch(G, Bt)
    errs = []
    for f in flat:
        gi = int(np.searchsorted(first, f, side="right") - 1)
        n_, e_, gg, bb = graphs[gi]
        ref, _ = oracle.edge_bucket(n_, e_, gg, bb, int(f - first[gi]), seed=int(f))
        errs.append(abs(zz[f] - ref.real))
    check = {"reference": "oracle complex128 bucket elimination of 64 sampled networks",
             "max_abs_err_zz": float(max(errs))}
    main = res["c64_persistent"]
    line = {"metric": "batched QAOA graph-evaluations/s (64 graphs, N in [50,1000], p=3)",
            "value": main["graph_evals_per_s"], "unit": "graph-evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": "64 seeded random 3-regular graphs, N uniform even in [50,1000] (synth.batch), "
                                   "p=3, per-graph angles; every edge's lightcone network in one persistent launch"},
            "plain_c128_per_bucket": res.get("c128_per_bucket"), "c128_persistent": res["c128_persistent"],
            "speedup_vs_plain_c128": (res["c128_per_bucket"]["ms_per_step"] / main["ms_per_step"]
                                      if "c128_per_bucket" in res else None), "check": check,
            "c64_dedup": dict(res["c64_persistent_dedup"],
                              note="opts.dedup: one network per isomorphism class of lightcones per graph "
                                   "(off in the main line)")}
    print(json.dumps(line), flush=True)


def run_c5(args, world, local_rank):
    """dE/dgamma_k, dE/dbeta_k on the seeded random 3-regular N=50 (seed 1000; --c5-n), p=4."""
    import torch
    from paper_2204_06045_gb300 import build, qtgb, synth
    torch.cuda.set_device(local_rank)
    build.build()
    n, p = args.c5_n, 4
    edges = synth.random_regular_graph(n, 1000)
    g, b = synth.angles(p, 1000)
    res = {}
    for dtype in ("c64", "c128"):
        with qtgb.plan(n, edges, p, dtype=dtype, with_grad=True) as pl:
            for _ in range(args.warmup):
                pl.energy_grad(g, b)
            steps = max(1, min(args.steps, 20))
            t0 = time.perf_counter()
            for _ in range(steps):
                E, dg, db = pl.energy_grad(g, b)
            dt = (time.perf_counter() - t0) / steps
            res[dtype] = {"ms_per_step": dt * 1e3, "grad_evals_per_s": 1 / dt, "steps": steps,
                          "dE_dgamma": dg.tolist(), "dE_dbeta": db.tolist(), "energy": float(E[0])}
    line = {"metric": f"QAOA energy+gradient evals/s (3-reg N={n} p=4)", "value": res["c64"]["grad_evals_per_s"],
            "unit": "grad-evals/s", "n_gpus": world, "steps": res["c64"]["steps"], "warmup": args.warmup,
            "ms_per_step": res["c64"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": f"random 3-regular N={n} seed 1000, p=4: energy and its 2p angle derivatives by "
                                   "the adjoint of the bucket elimination (host arrays in and out)"},
            "c128": res["c128"],
            "c64_vs_c128_max_abs_diff": float(np.max(np.abs(np.array(res["c64"]["dE_dgamma"] + res["c64"]["dE_dbeta"])
                                                          - np.array(res["c128"]["dE_dgamma"] + res["c128"]["dE_dbeta"]))))}
    print(json.dumps(line), flush=True)


def shard_step(pl, gd, bd, zz, E, s, dist):
    """One step of the sharded energy: this rank's networks, then one all-reduce (SUM) of the
    partial energy -- the one exchange the method has (E = |E|/2 - 1/2 sum of the edges' values)."""
    pl.energy(gd, bd, edge_zz=zz, energy=E, stream=s)
    if dist is not None:
        dist.all_reduce(E, op=dist.ReduceOp.SUM)


def run_shard(args, rank, world, local_rank):
    """One graph's energy split over the ranks: each contracts its share of the networks'
    slices (qt_plan_shard, longest processing time first on their cost), then one all-reduce of
    the partial energy per step (strong scaling: the job is one evaluation per step)."""
    import torch
    import torch.distributed as tdist
    from paper_2204_06045_gb300 import build, qtgb
    dist = None
    if world > 1:
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        dist = tdist
    torch.cuda.set_device(local_rank)
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    build.build()
    n, p, edges, g, b = workload_inputs()
    peak, peak_kind = measured_peaks()
    fma = qtgb.fma_peak("c64")
    with qtgb.plan_shard(n, edges, p, world, rank, dtype="c64") as pl:
        st = pl.stats()
        gd = torch.tensor(g, dtype=torch.float64, device="cuda")
        bd = torch.tensor(b, dtype=torch.float64, device="cuda")
        mine = pl.shard_edges
        zz = torch.zeros(max(1, mine.size), dtype=torch.float64, device="cuda") if mine.size else None
        E = torch.zeros(1, dtype=torch.float64, device="cuda")
        s = torch.cuda.current_stream()
        for _ in range(args.warmup):
            shard_step(pl, gd, bd, zz, E, s, dist)
        pl.sync(s)
        pl.kernel_time(reset=True)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local_rank) as clk:
            ev0.record(s)
            for _ in range(args.steps):
                shard_step(pl, gd, bd, zz, E, s, dist)
            ev1.record(s)
            torch.cuda.synchronize()
        pl.sync(s)
        ms = max_over_ranks(ev0.elapsed_time(ev1), dist, torch)
        kms, launches = pl.kernel_time(reset=True)
        energy = float(E.item())
        # end to end: host angles in, this rank's host results out, the partial energy reduced
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            _, e_part = pl.energy(g, b)
            et = torch.tensor([e_part], dtype=torch.float64, device="cuda")
            if dist is not None:
                dist.all_reduce(et, op=dist.ReduceOp.SUM)
            float(et.item())
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist, torch)
    _, ref_E = golden_c2()
    if rank == 0:
        achieved = st["alg_bytes"] / (kms * 1e-3) / 1e9 if kms > 0 else None
        line = {"metric": "QAOA energy evals/s (3-reg N=30 p=4)", "value": args.steps / (ms * 1e-3),
                "unit": "evals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
                "vs_baseline": args.steps / (ms * 1e-3) * PAPER_SECONDS_PER_EVAL, "dtype": "c64",
                "data": "synthetic",
                "config": config_dict("complex64; the networks' slices split over the ranks by LPT on cost, "
                                      "one all-reduce of the partial energy per step"),
                "e2e": {"value": args.steps / e2e_s, "unit": "evals/s", "h2d_bytes_per_step": 2 * p * 8,
                        "d2h_bytes_per_step": (int(mine.size) + 1) * 8},
                "roofline": dict(roofline("c64", st, kms, launches, achieved, peak, peak_kind, fma, None),
                                 note="rank 0's kernel and its share of the networks"),
                "clocks": clk.summary(), "gpu_launches": 3 * args.steps, "rank0_networks": int(mine.size),
                "check": {"energy": energy, "reference_energy": ref_E,
                          "rel_err_energy": abs(energy - ref_E) / abs(ref_E) if ref_E else None}}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "c3":
        if rank == 0:
            run_c3(args, world, local_rank)
    elif args.workload == "c5":
        if rank == 0:
            run_c5(args, world, local_rank)
    elif args.workload == "tncontract":
        if rank == 0:
            run_tncontract(args, world, local_rank)
    elif world > 1 and not args.replicas:
        run_shard(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
