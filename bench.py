#!/usr/bin/env python3
"""Throughput of the colour-coding DP on GB300 (one JSON line on stdout).

Workload: Chung-Lu power-law graph, n = 1,000,000, mean degree 16, degree
exponent 2.1 (seeded, synthetic; the paper's SNAP graphs are not available),
queries C6 and "glasses" (two triangles joined by a 2-edge path, k = 7),
plain form: one colouring per query per launch sequence.  A step counts both
queries under one fresh colouring each.  The graph is resident in HBM before
the timed region; the timed region covers K steps, each bracketed by CUDA
events on the library's stream, with a 256 MB L2 flush between steps outside
the events.

value: G edge-subset updates/s over all ranks, where the updates of a step
are the structural work the library reports (cc_work_units, independent of
the colouring).  Under torchrun each rank counts its own colourings on its
own copy of the graph (colourings are independent; no data-path
collective), so scaling is weak.

Roofline: the dominant stage is the C6 root-cycle closure; its algorithmic
bytes are 4 per data edge scanned by the DB procedure's path extensions
(both halves, every level), read from the library's structural counter
(cc_work_detail).  The leaf joins and triangle blocks of "glasses" get
their own lines (8 bytes per gathered table entry, 4 per neighbour id or
wedge, 8 per output entry).

--impl reference times the CPU oracle on all host cores: whole colourings
(one C6 and one glasses colouring per step) on a Chung-Lu graph of the same
shape and smaller size, one step per core in parallel, and prints the same
line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "colorful-count DP G edge·subset updates/s + colorings/s, batched vs plain; p99"
UNIT = "G edge-subset updates/s"
WORKLOAD = {"graph": "chung_lu", "n": 1_000_000, "mean_deg": 16, "gamma": 2.1, "seed": 2,
            "queries": ["C6", "glasses"], "form": "plain", "colourings_per_query_per_step": 1}
COLOR_SEED = 1
BATCH_QUERIES = ["C5", "chord_pendant", "glasses"]
# DRAM bytes (read + written) per algorithmic byte of each kernel family,
# from an ncu capture of every launch of those kernels on a small case of the
# benchmark's shape (Chung-Lu n = 2e5, mean 16, gamma 2.1; one C6 and one
# glasses colouring): the closure 24.48 GB / 13.01 GB, the leaf joins
# (lanes on the output slots) 88.6 MB / 978 MB, the triangle list 104.2 MB /
# 494 MB.  The bench multiplies them by the full workload's algorithmic
# bytes.  The small case's tables fit in L2, so the leaf-join and triangle
# ratios are lower bounds.
TRAFFIC_PER_ALG_BYTE = {"cycle_closure": 24.48 / 13.01, "leaf_join": 88.6 / 978.0, "triangle": 104.2 / 493.6}
FLUSH_BYTES = 256 << 20
# CPU baseline: whole colourings on a smaller graph of the benchmark's shape
CPU_GRAPH = {"graph": "chung_lu", "n": 2_000, "mean_deg": 16, "gamma": 2.1, "seed": 2}


def rank_trials(rank: int, count: int, offset: int = 0):
    """Colourings a rank counts: ranks never share one (colourings are
    independent, so the ranks need no data exchange)."""
    return [rank * 1_000_000 + offset + i for i in range(count)]


def max_over_ranks(value: float, dist, device=None) -> float:
    """The slowest rank's time (the job's time)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_name():
    w = WORKLOAD
    return (f"chung_lu n={w['n']} mean_deg={w['mean_deg']} gamma={w['gamma']} seed={w['seed']}; "
            f"queries C6 + glasses; plain form, 1 colouring per query per step")


def make_graph():
    import graphgen as gg
    w = WORKLOAD
    return gg.chung_lu(w["n"], w["mean_deg"], w["gamma"], w["seed"])


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ----------------------------------- CPU oracle -----------------------------------
def glasses_units(g):
    """Structural work of one "glasses" colouring (the library's plan: a
    triangle block, two leaf joins over tables of 15 and 20 signature slots,
    the root triangle), from the graph alone: 35 * nnz for the leaf joins
    plus twice the wedges the triangle blocks scan, where a source u scans,
    for each lower neighbour v but the lowest, v's lower neighbours (degree
    order: degree, then id)."""
    import numpy as np
    deg = np.diff(g.row_ptr)
    rank = np.lexsort((np.arange(g.n), deg)).argsort()
    src = np.repeat(np.arange(g.n), deg)
    lower = rank[g.col] < rank[src]
    lo_cnt = np.bincount(src[lower], minlength=g.n)
    # per source u: sum of lo_cnt over its lower neighbours, minus the lowest one's
    s_all = np.bincount(src[lower], weights=lo_cnt[g.col[lower]], minlength=g.n)
    lowest = np.full(g.n, -1, dtype=np.int64)
    lsrc, lnb = src[lower], g.col[lower]
    order = np.lexsort((rank[lnb], lsrc))
    first = np.ones(order.size, bool)
    first[1:] = lsrc[order][1:] != lsrc[order][:-1]
    lowest[lsrc[order][first]] = lnb[order][first]
    has = lowest >= 0
    wedges = s_all.sum() - lo_cnt[lowest[has]].sum()
    return 35.0 * g.nnz + 2.0 * float(wedges)


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def _cpu_step(trial):
    """One step of the oracle (one C6 and one glasses colouring) on the CPU
    baseline graph; returns the DP seconds.  Runs in a worker process."""
    import graphgen as gg
    import oracle as O
    g = gg.chung_lu(CPU_GRAPH["n"], CPU_GRAPH["mean_deg"], CPU_GRAPH["gamma"], CPU_GRAPH["seed"])
    secs = 0.0
    for name in WORKLOAD["queries"]:
        k, e = gg.query(name)
        t = {}
        O.dp_count(g, k, e, O.colors(COLOR_SEED, trial, g.n, k), timing=t)
        secs += t["dp_seconds"]
    return secs


def _cpu_warm(_):
    """Worker start-up outside the timed region: imports and the oracle library."""
    import graphgen as gg
    import oracle as O
    O.colors(1, 0, 1, 2)
    gg.chung_lu(CPU_GRAPH["n"], CPU_GRAPH["mean_deg"], CPU_GRAPH["gamma"], CPU_GRAPH["seed"])
    return 0


def oracle_baseline(rounds: int = 1):
    """The oracle as it stands on the host: one step alone (1 core), then one
    step per core in parallel (spawned worker processes, distinct colourings),
    `rounds` times.  Returns a cpu_baseline dict in the benchmark's units."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    import graphgen as gg
    import oracle as O
    g = gg.chung_lu(CPU_GRAPH["n"], CPU_GRAPH["mean_deg"], CPU_GRAPH["gamma"], CPU_GRAPH["seed"])
    units_step = O.cycle_units(g, 6, 6) + glasses_units(g)
    cores = os.cpu_count() or 1
    one = _cpu_step(0)
    with ProcessPoolExecutor(cores, mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_cpu_warm, range(cores)))  # warm-up: imports, oracle library
        t0 = time.perf_counter()
        list(ex.map(_cpu_step, range(100, 100 + rounds * cores)))
        wall = time.perf_counter() - t0
    steps = rounds * cores
    value = units_step * steps / wall / 1e9
    w = CPU_GRAPH
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "value_1core": units_step / one / 1e9, "colorings_per_s": 2 * steps / wall,
            "cpu_model": cpu_model(), "nproc": cores,
            "sample": (f"whole colourings (C6 + glasses per step, {steps} steps, one per core in spawned "
                       f"processes, {wall:.1f} s wall) on chung_lu n={w['n']} mean_deg={w['mean_deg']} "
                       f"gamma={w['gamma']} seed={w['seed']}, the benchmark graph's shape at 1/500 of its size; "
                       f"{units_step:.4g} updates per step")}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cb = oracle_baseline(rounds=max(1, args.steps // 4))
    ms = 1e3 / (cb["colorings_per_s"] / 2)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": workload_name(), **WORKLOAD},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------ GPU arm ------------------------------------
def serve_workload(requests, small_pool, workers, budget_gib, loads=(0.7, 1.0), progress=True):
    """Serving workload: Chung-Lu graphs n in {1e4, 1e5, 1e6}, mean degree
    8-16, exponent 2.1-2.5 resident on the device; a Poisson stream of
    requests for treewidth-2 queries with k = 4..8 and 1-32 colourings each,
    served by the library's continuous-batching loop (cc_server_*).  Arrival
    rate: the given fractions of the capacity measured by a closed-loop
    burst.  Returns p50/p99 arrival-to-result latency and throughput."""
    import numpy as np

    import graphgen as gg
    import paper_1602_04478_gb300 as P

    rng = np.random.default_rng(5)
    sizes = [10_000, 100_000, 1_000_000]
    graphs = []
    for n in sizes:
        for d in (8, 12, 16):
            for gm in (2.1, 2.3, 2.5):
                if n == 1_000_000 and (d, gm) != (16, 2.5) and small_pool:
                    continue
                graphs.append(gg.chung_lu(n, d, gm, int(rng.integers(1 << 30))))
    srv = P.Server(0, workers=workers, memory_budget=budget_gib << 30)
    gids = [srv.load_graph(g) for g in graphs]
    qnames = ["C4", "diamond", "C5", "chord_pendant", "C6", "glasses", "C6_2pendants"]
    qids = [srv.set_query(*gg.query(q)) for q in qnames]
    srv.set_seed(COLOR_SEED)

    small = {gid for gid, g in zip(gids, graphs) if g.n <= 10_000}

    def make_req():
        gid = gids[int(rng.integers(len(gids)))]
        # the doubly annotated 8-node query runs on the generic closure path,
        # seconds per colouring from n = 1e5 up: it is served on the n = 1e4 graphs
        pool = qids if gid in small else qids[:-1]
        return (gid, pool[int(rng.integers(len(pool)))], int(rng.integers(0, 1000)), int(rng.integers(1, 33)))

    def drain(expected):
        got, lat, bad = 0, [], 0
        while got < expected:
            for r in srv.poll(timeout_ms=500):
                got += 1
                lat.append(r["done_s"] - r["submit_s"])
                bad += r["status"] not in (0, -6)
        return lat, bad

    # capacity: closed-loop burst of requests
    burst = [make_req() for _ in range(requests // 4 or 1)]
    t0 = time.perf_counter()
    for rq in burst:
        srv.submit(*rq)
    drain(len(burst))
    cap = len(burst) / (time.perf_counter() - t0)
    out = {"graphs": len(graphs), "graph_sizes": sorted({g.n for g in graphs}), "queries": qnames,
           "workers": workers, "capacity_req_per_s": cap, "requests_per_rate": requests, "rates": []}
    if progress:
        # progress lines (a cut-off run still leaves its measurements); the last line is the summary
        print(json.dumps({"impl": "ours", "mode": "serve", **out, "partial": True}), flush=True)
    for frac in loads:
        lam = frac * cap
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=requests))
        reqs = [make_req() for _ in range(requests)]
        t0 = time.perf_counter()
        for at, rq in zip(arrivals, reqs):
            dt = at - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            srv.submit(*rq)
        lat, bad = drain(len(reqs))
        wall = time.perf_counter() - t0
        colourings = sum(r[3] for r in reqs)
        out["rates"].append({"load": frac, "lambda_req_per_s": lam, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                             "p99_ms": 1e3 * float(np.percentile(lat, 99)), "req_per_s": len(reqs) / wall,
                             "colorings_per_s": colourings / wall, "failed_requests": bad})
        if progress:
            print(json.dumps({"impl": "ours", "mode": "serve", **out, "partial": True}), flush=True)
    srv.close()
    return out


def run_serve(args):
    out = serve_workload(args.serve_requests, args.serve_small, args.workers, args.serve_budget)
    print(json.dumps({"impl": "ours", "mode": "serve", **out}), flush=True)
    return 0


def run_rmat_pendants(args):
    """R-MAT graph (a=0.57, b=0.19, c=0.19, edge factor 16, symmetrised and
    deduplicated) and the 8-node query (6-cycle with two pendants on opposite
    nodes): `--rmat-trials` colourings in one batched call.  Reports the time
    per colouring and the per-colouring status (overflow is reported, never
    wrapped)."""
    import numpy as np

    import graphgen as gg
    import paper_1602_04478_gb300 as P

    g = gg.rmat(args.rmat_scale, 16, 0.57, 0.19, 0.19, 1)
    ctx = P.Context(0)
    gid = ctx.load_graph(g)
    P.cc_set_coloring_seed(ctx.h, COLOR_SEED)
    q = ctx.set_query(*gg.query("C6_2pendants"))
    T = args.rmat_trials
    P.cc_set_graph_capture(ctx.h, False)  # one call: no replay to amortise a capture
    t0 = time.perf_counter()
    res, st = P.cc_count_batch(ctx.h, [(gid, q, 0, T)])
    dt = time.perf_counter() - t0
    over = [int(x) == (1 << 64) - 1 for x in res[0]]
    print(json.dumps({"impl": "ours", "mode": "rmat_pendants", "rmat_scale": args.rmat_scale, "n": g.n,
                      "nnz": int(g.nnz), "max_degree": int(np.diff(g.row_ptr).max()), "query": "C6_2pendants",
                      "trials": T, "s_per_coloring": dt / T, "status": P.ERRORS.get(st[0], st[0]),
                      "overflow_per_coloring": over,
                      "colorful": [int(x) for x in res[0]]}), flush=True)
    ctx.close()


PRECISION_GRAPHS = {
    "chung_lu n=1e4 d=8 g=2.1": ("chung_lu", 10_000, 8, 2.1, 11),
    "chung_lu n=1e4 d=16 g=2.5": ("chung_lu", 10_000, 16, 2.5, 12),
    "chung_lu n=1e5 d=8 g=2.3": ("chung_lu", 100_000, 8, 2.3, 13),
    "erdos_renyi n=1e4 m=5e4": ("erdos_renyi", 10_000, 50_000, 14),
    "rmat scale=12 ef=8": ("rmat", 12, 8, 0.57, 0.19, 0.19, 15),
}
PRECISION_QUERIES = ["C4", "diamond", "C5", "chord_pendant", "C6", "glasses", "C5_pendant_path", "C6_2pendants"]


def precision_stats(est, trials):
    """Coefficient of variation (sample std / mean, the paper reports
    variance / mean) of the first `trials` per-colouring estimates, and of
    their mean (std / mean / sqrt(trials)); None when the mean is 0."""
    import numpy as np
    x = np.asarray(est[:trials], dtype=np.float64)
    mu = float(x.mean())
    if mu == 0.0 or x.size < 2:
        return None, None
    cv = float(x.std(ddof=1)) / mu
    return cv, cv / math.sqrt(x.size)


def run_precision(args):
    """Precision of colour coding (the paper's Section "Precision of Color
    Coding"): for every (graph, query) pair of a synthetic test set, T fresh
    colourings in one batched call; the coefficient of variation of the
    per-colouring estimate n_colorful * k^k / k! / aut(Q) over the first 3,
    10 and T colourings, and the share of pairs at or below 0.1."""
    import graphgen as gg
    import paper_1602_04478_gb300 as P

    ctx = P.Context(0)
    P.cc_set_coloring_seed(ctx.h, 7)
    T = args.precision_trials
    pairs = []
    t0 = time.perf_counter()
    for gname, spec in PRECISION_GRAPHS.items():
        g = getattr(gg, spec[0])(*spec[1:])
        gid = ctx.load_graph(g)
        qids = {q: ctx.set_query(*gg.query(q)) for q in PRECISION_QUERIES}
        res, st = P.cc_count_batch(ctx.h, [(gid, qids[q], 0, T) for q in PRECISION_QUERIES])
        for (q, qid), cnt, code in zip(qids.items(), res, st):
            info = P.cc_query_info(ctx.h, qid)
            k = info["k"]
            scale = k ** k / math.factorial(k) / info["aut"]
            est = [float(c) * scale for c in cnt]
            row = {"graph": gname, "query": q, "status": P.ERRORS.get(code, "ok") if code else "ok",
                   "mean_estimate": sum(est) / len(est)}
            for t in (3, 10, T):
                cv, cvm = precision_stats(est, t)
                row[f"cov_{t}"] = cv
                row[f"cov_of_mean_{t}"] = cvm
            pairs.append(row)
        ctx.free_graph(gid)
    wall = time.perf_counter() - t0
    ok = [r for r in pairs if r["status"] == "ok" and r["cov_3"] is not None]
    summary = {}
    for t in (3, 10, T):
        summary[f"share_cov_le_0.1_{t}_trials"] = sum(r[f"cov_{t}"] <= 0.1 for r in ok) / max(1, len(ok))
        summary[f"share_cov_of_mean_le_0.1_{t}_trials"] = sum(r[f"cov_of_mean_{t}"] <= 0.1 for r in ok) / max(1, len(ok))
    print(json.dumps({"impl": "ours", "mode": "precision", "trials": T, "pairs": len(pairs),
                      "pairs_counted": len(ok), "colorings": T * len(pairs), "wall_s": wall, **summary,
                      "per_pair": pairs}), flush=True)
    ctx.close()
    return 0


PS_GRAPHS = {
    "chung_lu n=1e4 d=8 g=2.1": ("chung_lu", 10_000, 8, 2.1, 21),
    "chung_lu n=1e5 d=8 g=2.3": ("chung_lu", 100_000, 8, 2.3, 22),
    "rmat scale=12 ef=8": ("rmat", 12, 8, 0.57, 0.19, 0.19, 24),
    "erdos_renyi n=1e5 m=4e5": ("erdos_renyi", 100_000, 400_000, 25),
}
PS_QUERIES = ["C4", "C5", "C6", "C5_pendant_path", "C6_2pendants"]


def run_ps_compare(args):
    """DB against PS (the paper's Section "Performance Comparison of PS and DB
    Algorithms") on synthetic graphs: one colouring of each (graph, query)
    under the PS procedure and under DB on the same general per-source
    kernel (the improvement factor IF = PS time / DB time isolates the
    procedure), and under DB with the library's default kernels."""
    import torch

    import graphgen as gg
    import paper_1602_04478_gb300 as P

    ctx = P.Context(0)
    stream = ctx.stream
    P.cc_set_coloring_seed(ctx.h, 5)

    def timed(fn):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b), out

    rows = []
    for gname, spec in PS_GRAPHS.items():
        g = getattr(gg, spec[0])(*spec[1:])
        gid = ctx.load_graph(g)
        for q in PS_QUERIES:
            qid = ctx.set_query(*gg.query(q))
            row = {"graph": gname, "query": q}
            for form, proc, hd in (("db_default", P.PROC_DB, -1), ("db_general", P.PROC_DB, 1 << 30),
                                   ("ps", P.PROC_PS, -1)):
                P.cc_set_procedure(ctx.h, proc)
                P.cc_set_heavy_degree(ctx.h, hd)
                ctx.count(gid, qid, 1, 1, allow_overflow=True)  # warm-up (scratch, structure)
                ms, (col, _, _) = timed(lambda: ctx.count(gid, qid, 0, 1, allow_overflow=True))
                row[f"ms_{form}"] = ms
                row[f"count_{form}"] = int(col[0])
            P.cc_set_procedure(ctx.h, P.PROC_DB)
            P.cc_set_heavy_degree(ctx.h, -1)
            row["counts_equal"] = row["count_ps"] == row["count_db_general"] == row["count_db_default"]
            row["improvement_factor"] = row["ms_ps"] / row["ms_db_general"]
            row["improvement_factor_vs_default"] = row["ms_ps"] / row["ms_db_default"]
            rows.append(row)
            print(json.dumps({"partial": True, **row}), flush=True)
        ctx.free_graph(gid)
    ifs = [r["improvement_factor"] for r in rows]
    print(json.dumps({"impl": "ours", "mode": "ps_compare", "pairs": len(rows),
                      "db_faster_share": sum(x > 1 for x in ifs) / len(ifs), "max_if": max(ifs),
                      "avg_if": sum(ifs) / len(ifs), "all_counts_equal": all(r["counts_equal"] for r in rows),
                      "per_pair": rows}), flush=True)
    ctx.close()
    return 0


PLAN_QUERIES = {
    "chord_pendant": None, "glasses": None, "diamond": None,
    # three triangles in a strip (0-1-2, 1-2-3, 2-3-4)
    "triangle_strip": (5, [(0, 1), (1, 2), (2, 0), (1, 3), (2, 3), (2, 4), (3, 4)]),
    # two triangles on one node with a pendant on each
    "bowtie_pendants": (7, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 2), (0, 5), (4, 6)]),
    # 4-cycle with a triangle on one edge
    "house": (5, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (4, 1)]),
}
PLAN_GRAPHS = {
    "chung_lu n=1e5 d=16 g=2.1": ("chung_lu", 100_000, 16, 2.1, 31),
    "chung_lu n=1e6 d=16 g=2.1": ("chung_lu", 1_000_000, 16, 2.1, 2),
    "rmat scale=16 ef=8": ("rmat", 16, 8, 0.57, 0.19, 0.19, 32),
}


def run_plan_eval(args):
    """The paper's plan heuristic (Section "Finding Good Decomposition
    Trees": rank every tree by longest cycle block, then boundary nodes, then
    annotations) against the measured best tree (Section "Evaluation of Plan
    Generation Heuristic"): every supported tree of each query timed on each
    graph (CUDA events, best of 3 colourings), and the heuristic's tree
    compared with the fastest."""
    import torch

    import graphgen as gg
    import paper_1602_04478_gb300 as P

    ctx = P.Context(0)
    stream = ctx.stream
    P.cc_set_coloring_seed(ctx.h, 3)

    def timed(fn):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b), out

    rows = []
    for gname, spec in PLAN_GRAPHS.items():
        g = getattr(gg, spec[0])(*spec[1:])
        gid = ctx.load_graph(g)
        for q, shape in PLAN_QUERIES.items():
            k, e = shape if shape else gg.query(q)
            trees = [t for t in P.cc_plan_enumerate(k, e) if t["supported"]]
            if len(trees) < 2:
                continue
            times, counts = [], set()
            for t in trees:
                qid = ctx.set_query(k, e)
                P.cc_set_decomposition(ctx.h, qid, t["seq"])
                ctx.count(gid, qid, 9, 1, allow_overflow=True)  # warm-up
                best = None
                for rep in range(3):
                    ms, (col, _, _) = timed(lambda: ctx.count(gid, qid, 0, 1, allow_overflow=True))
                    best = ms if best is None else min(best, ms)
                    counts.add(int(col[0]))
                times.append(best)
            # the paper's heuristic (its factors alone), the library's static
            # pick, and the measured choice (cc_autotune_plan, timed separately)
            h = [i for i, t in enumerate(trees) if t["paper"]][0]
            lib_pick = [i for i, t in enumerate(trees) if t["default"]][0]
            qa = ctx.set_query(k, e)
            tuned = P.cc_autotune_plan(ctx.h, gid, qa)
            key = [(t["longest"], t["boundary"], t["annotations"]) for t in trees]
            ties = [i for i in range(len(trees)) if key[i] == key[h]]
            opt = min(range(len(trees)), key=lambda i: times[i])
            row = {"graph": gname, "query": q, "trees": len(trees), "ms": times, "heuristic": h, "optimal": opt,
                   "heuristic_is_optimal": h == opt, "heuristic_over_optimal": times[h] / times[opt],
                   "library_pick": lib_pick, "library_is_optimal": lib_pick == opt,
                   "library_over_optimal": times[lib_pick] / times[opt],
                   "measured_pick": tuned, "measured_over_optimal": times[tuned] / times[opt],
                   "trees_tied_with_heuristic": len(ties), "counts_equal": len(counts) == 1,
                   "factors": key, "join_cost": [t["cost"] for t in trees]}
            rows.append(row)
            print(json.dumps({"partial": True, **row}), flush=True)
        ctx.free_graph(gid)
    print(json.dumps({"impl": "ours", "mode": "plan_eval", "pairs": len(rows),
                      "heuristic_optimal_share": sum(r["heuristic_is_optimal"] for r in rows) / max(1, len(rows)),
                      "within_15pct_share": sum(r["heuristic_over_optimal"] <= 1.15 for r in rows) / max(1, len(rows)),
                      "max_heuristic_over_optimal": max((r["heuristic_over_optimal"] for r in rows), default=None),
                      "library_optimal_share": sum(r["library_is_optimal"] for r in rows) / max(1, len(rows)),
                      "library_within_15pct_share": sum(r["library_over_optimal"] <= 1.15 for r in rows) / max(1, len(rows)),
                      "max_library_over_optimal": max((r["library_over_optimal"] for r in rows), default=None),
                      "measured_within_15pct_share": sum(r["measured_over_optimal"] <= 1.15 for r in rows) / max(1, len(rows)),
                      "max_measured_over_optimal": max((r["measured_over_optimal"] for r in rows), default=None),
                      "all_counts_equal": all(r["counts_equal"] for r in rows), "per_pair": rows}), flush=True)
    ctx.close()
    return 0


CASE2_QUERIES = {
    # a square and a triangle on one edge (Case-2 square, or Case-2 triangle)
    "house": (5, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (4, 1)]),
    # a 5-cycle and a path of two edges between its nodes 0 and 2
    "theta_5_2": (6, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (0, 5), (5, 2)]),
    # a 5-cycle and a square on one edge
    "pentagon_house": (7, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (0, 5), (5, 6), (6, 1)]),
    # paths of 3, 3 and 3 edges between two nodes
    "theta_333": (8, [(0, 2), (2, 3), (3, 1), (0, 4), (4, 5), (5, 1), (0, 6), (6, 7), (7, 1)]),
}
CASE2_GRAPHS = {
    "erdos_renyi n=1e5 m=4e5": ("erdos_renyi", 100_000, 400_000, 41),
    "chung_lu n=2e4 d=8 g=2.1": ("chung_lu", 20_000, 8, 2.1, 42),
}


def run_case2(args):
    """Case-2 blocks of length >= 4 (two boundary nodes): one colouring of
    each supported tree of each query, with the library's stage timings
    (the pair-list count and append launches and the pair-graph build are
    inside the non-root cycle stage), and the satellite query of the paper's
    worked decomposition on the smaller graph."""
    import torch

    import graphgen as gg
    import paper_1602_04478_gb300 as P

    queries = dict(CASE2_QUERIES)
    # the Satellite query of the worked decomposition (Section 4.1): 5-cycle
    # a..e, f on a and g on c, leaf h on f, triangle i, j, k on i with i on f, g
    queries["satellite"] = (11, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (0, 5), (5, 6), (6, 2), (5, 7), (5, 8),
                                 (6, 8), (8, 9), (9, 10), (10, 8)])
    ctx = P.Context(0)
    stream = ctx.stream
    P.cc_set_coloring_seed(ctx.h, 9)

    def timed(fn):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b), out

    rows = []
    for gname, spec in CASE2_GRAPHS.items():
        g = getattr(gg, spec[0])(*spec[1:])
        gid = ctx.load_graph(g)
        for qname, (k, e) in queries.items():
            if qname == "satellite" and not gname.startswith("chung_lu"):
                continue
            for t in P.cc_plan_enumerate(k, e):
                if not t["supported"]:
                    continue
                blocks, _ = P.cc_plan_inspect(k, e, t["seq"] or None)
                shape = " ".join(f"{b['kind']}{len(b['nodes'])}/{len(b['boundary'])}" for b in blocks)
                qid = ctx.set_query(k, e)
                if t["seq"]:
                    P.cc_set_decomposition(ctx.h, qid, t["seq"])
                ctx.count(gid, qid, 1, 1, allow_overflow=True)  # warm-up
                P.cc_reset_timing(ctx.h)
                P.cc_set_timing(ctx.h, True)
                ms, (col, _, _) = timed(lambda: ctx.count(gid, qid, 0, 1, allow_overflow=True))
                stages = P.cc_get_timing(ctx.h)
                P.cc_set_timing(ctx.h, False)
                row = {"graph": gname, "query": qname, "tree": shape, "default": t["default"],
                       "ms_per_colouring": ms, "count": int(col[0]),
                       "stage_ms": {name: round(v[0], 3) for name, v in stages.items()}}
                rows.append(row)
                print(json.dumps({"partial": True, **row}), flush=True)
        ctx.free_graph(gid)
    print(json.dumps({"impl": "ours", "mode": "case2", "rows": rows}), flush=True)
    ctx.close()
    return 0


def run_profile_case(args):
    """Count QUERY (comma-separated list) for `--profile-reps` colourings on a
    Chung-Lu graph of the benchmark's shape (n = --profile-n, mean degree
    --profile-mean; the benchmark graph by default) after one untimed
    colouring that builds the per-graph structure: the command a profiler
    wraps to capture a few launches of one kernel.  Prints the algorithmic
    bytes of each stage of each query (cc_work_detail) beside the counts."""
    import graphgen as gg
    import paper_1602_04478_gb300 as P

    w = WORKLOAD
    n = args.profile_n or w["n"]
    mean = args.profile_mean or w["mean_deg"]
    g = gg.chung_lu(n, mean, w["gamma"], w["seed"])
    ctx = P.Context(0, budget_bytes=int(args.profile_budget * (1 << 30)))
    gid = ctx.load_graph(g)
    P.cc_set_coloring_seed(ctx.h, COLOR_SEED)
    hd = args.heavy_degree if args.heavy_degree >= 0 else 384
    P.cc_set_heavy_degree(ctx.h, hd)
    # --profile-trees NAME=I,...: the I-th supported tree (cc_autotune_plan's
    # index, as the benchmark line reports it) instead of the default tree;
    # timing the trees under a profiler would mislead the choice
    trees = dict((kv.split("=")[0], int(kv.split("=")[1])) for kv in args.profile_trees.split(",") if kv)
    out = {"profile_case": args.profile_case, "n": n, "mean_deg": mean, "heavy_degree": hd, "trees": trees,
           "budget_gib": args.profile_budget, "queries": {}}
    for name in args.profile_case.split(","):
        k, e = CASE2_QUERIES[name] if name in CASE2_QUERIES else gg.query(name)
        q = ctx.set_query(k, e)
        if name in trees:
            seq = [t for t in P.cc_plan_enumerate(k, e) if t["supported"]][trees[name]]["seq"]
            if seq:
                P.cc_set_decomposition(ctx.h, q, seq)
        detail = P.cc_work_detail(ctx.h, gid, q)
        ctx.count(gid, q, 100, 1, allow_overflow=True)  # per-graph structure, outside the captured launches
        cols = [int(ctx.count(gid, q, t, 1, allow_overflow=True)[0][0]) for t in range(args.profile_reps)]
        out["queries"][name] = {"colorful": cols, "stages": detail}
    out["kernel_launches"] = P.cc_kernel_launches(ctx.h)
    print(json.dumps(out))
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve", action="store_true", help="run the serving workload instead")
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--serve-small", action="store_true", help="one n = 1e6 graph instead of nine")
    ap.add_argument("--serve-leg", type=int, default=100,
                    help="requests of the short serving leg of the default run (0: skip it)")
    ap.add_argument("--serve-budget", type=int, default=64, help="server table budget in GiB")
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--batch-trials", type=int, default=64,
                    help="colourings per query in the batched-configuration leg (0: skip it)")
    ap.add_argument("--heavy-degree", type=int, default=-1,
                    help="heavy/light source degree threshold (default: autotuned)")
    ap.add_argument("--profile-case", default=None, metavar="QUERY",
                    help="count QUERY (comma-separated) on a benchmark-shaped graph for profiler captures")
    ap.add_argument("--profile-n", type=int, default=0, help="graph size of --profile-case (0: the benchmark's)")
    ap.add_argument("--profile-mean", type=float, default=0, help="mean degree of --profile-case (0: 16)")
    ap.add_argument("--profile-reps", type=int, default=1, help="colourings counted by --profile-case")
    ap.add_argument("--profile-trees", default="",
                    help="NAME=I,...: --profile-case counts NAME with its I-th supported tree")
    ap.add_argument("--profile-budget", type=float, default=0,
                    help="device memory budget of --profile-case in GiB (0: none); caps the per-CTA push's slots")
    ap.add_argument("--rmat-pendants", action="store_true",
                    help="R-MAT graph with the 8-node 6-cycle-with-two-pendants query instead")
    ap.add_argument("--rmat-scale", type=int, default=22)
    ap.add_argument("--rmat-trials", type=int, default=16)
    ap.add_argument("--precision", action="store_true",
                    help="precision study: coefficient of variation against the number of colourings")
    ap.add_argument("--precision-trials", type=int, default=50)
    ap.add_argument("--ps-compare", action="store_true", help="DB against PS improvement factors")
    ap.add_argument("--plan-eval", action="store_true", help="plan heuristic against the measured best tree")
    ap.add_argument("--case2", action="store_true", help="Case-2 blocks of length >= 4 (two boundary nodes)")
    args = ap.parse_args()
    if args.rmat_pendants:
        return run_rmat_pendants(args)
    if args.precision:
        return run_precision(args)
    if args.ps_compare:
        return run_ps_compare(args)
    if args.plan_eval:
        return run_plan_eval(args)
    if args.case2:
        return run_case2(args)
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return run_serve(args)

    import numpy as np
    import torch

    import graphgen as gg
    import paper_1602_04478_gb300 as P

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    g = make_graph()
    ctx = P.Context(local)
    gid = ctx.load_graph(g)
    qids = {name: ctx.set_query(*gg.query(name)) for name in WORKLOAD["queries"]}
    P.cc_set_coloring_seed(ctx.h, COLOR_SEED)
    units = {name: P.cc_work_units(ctx.h, gid, q) for name, q in qids.items()}
    units_step = sum(units.values())
    if args.heavy_degree >= 0:
        P.cc_set_heavy_degree(ctx.h, args.heavy_degree)
        tuned = {name: args.heavy_degree for name in qids}
    else:
        tuned = {name: P.cc_autotune(ctx.h, gid, q) for name, q in qids.items()}
    # the decomposition tree measured fastest on this graph (queries with one tree keep it)
    trees = {name: P.cc_autotune_plan(ctx.h, gid, q) for name, q in qids.items()}
    trial_base = rank * 1_000_000

    def step(i):
        out = {}
        trial = rank_trials(rank, 1, i)[0]
        for name, q in qids.items():
            col, _, _ = ctx.count(gid, q, trial, 1)
            out[name] = int(col[0])
        return out

    for w in range(args.warmup):
        step(10_000 + w)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=f"cuda:{local}")
    stream = ctx.stream
    P.cc_set_timing(ctx.h, True)
    P.cc_reset_timing(ctx.h)
    sampler = ClockSampler(local)
    barrier()
    sampler.start()
    launches0 = P.cc_kernel_launches(ctx.h)
    evs = []
    counts = []
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        counts.append(step(i))
        b.record(stream)
        evs.append((a, b))
    barrier()
    wall = time.perf_counter() - wall0
    launches = P.cc_kernel_launches(ctx.h) - launches0
    clocks = sampler.stop()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    kern = P.cc_get_timing(ctx.h)
    P.cc_set_timing(ctx.h, False)
    ms = max_over_ranks(ms, dist, device=f"cuda:{local}")
    value = units_step * args.steps * world / (ms / 1e3) / 1e9
    colourings = len(qids) * args.steps * world / (ms / 1e3)

    # Rooflines.  Algorithmic bytes per colouring of each kernel family come
    # from the library's structural counter (cc_work_detail): the C6 closure
    # reads 4 bytes (one neighbour id) per data edge its path extensions scan;
    # a leaf join gathers 8 bytes per update and reads 4 per edge, 8 per entry
    # of the annotating node block and writes 8 per output entry; a triangle
    # block reads 4 bytes per wedge and writes 8 per output entry.
    peak, peak_kind = measured_peaks()
    detail = {name: P.cc_work_detail(ctx.h, gid, q) for name, q in qids.items()}
    fam_bytes = {"cycle_closure": sum(d["alg_bytes"] for d in detail["C6"] if d["kind"] == "root_cycle"),
                 "leaf_join": sum(d["alg_bytes"] for d in detail["glasses"] if d["kind"] == "leaf"),
                 "triangle": sum(d["alg_bytes"] for d in detail["glasses"] if d["kind"] == "triangle"),
                 "root_sum": sum(d["alg_bytes"] for d in detail["glasses"] if d["kind"] == "root_node")}
    fam_of = {"cycle_closure": lambda k: k.startswith("cycle_"), "leaf_join": lambda k: k == "leaf_join",
              "triangle": lambda k: k.startswith("triangle"), "root_sum": lambda k: k == "root_sum"}
    kernel_rooflines = {}
    for fam, nbytes in fam_bytes.items():
        names = sorted(k for k in kern if fam_of[fam](k))
        f_ms = sum(kern[k][0] for k in names) / args.steps
        if not names or f_ms <= 0:
            continue
        ach = nbytes / (f_ms / 1e3) / 1e9
        ratio = TRAFFIC_PER_ALG_BYTE.get(fam)
        tr = ratio * nbytes if ratio else None
        kernel_rooflines[fam] = {
            "kernels": names, "bound": "hbm", "alg_bytes_per_colouring": nbytes, "ms_per_colouring": f_ms,
            "launches_per_colouring": sum(kern[k][1] for k in names) / args.steps,
            "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "dram_bytes_per_colouring": tr, "dram_frac": (tr / (f_ms / 1e3) / 1e9 / peak) if tr else None,
            "share_of_step": f_ms * args.steps / ms}
    c6_scans = [d["scans"] for d in detail["C6"] if d["kind"] == "root_cycle"][0]
    clo = kernel_rooflines["cycle_closure"]
    roofline = {"bound": "hbm", "kernel": "C6 root-cycle closure (" + " + ".join(clo["kernels"]) + ")",
                "achieved": clo["achieved"], "peak": peak, "peak_source": peak_kind, "unit": "GB/s",
                "frac": clo["frac"], "traffic": clo["dram_bytes_per_colouring"],
                "alg_bytes": clo["alg_bytes_per_colouring"],
                "alg_bytes_rule": "4 B per data edge scanned by the path extensions, both halves, every level",
                "scanned_edges_by_level": [x for x in c6_scans if x],
                "avg_launch_ms": clo["ms_per_colouring"], "launches_per_colouring": clo["launches_per_colouring"],
                "share_of_step": clo["share_of_step"],
                "note": "issue-bound (integer ALU / warp-instruction issue), not DRAM-bound: see dram_frac"}

    def dev_ms(fn):
        """Device time of fn's work on the library's stream (CUDA events), fn's result."""
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        barrier()
        a.record(stream)
        out = fn()
        b.record(stream)
        barrier()
        return max_over_ranks(a.elapsed_time(b), dist, device=f"cuda:{local}"), out

    # batched form: the same kind of step (one colouring of each query per
    # step) for K colourings in one cc_count_batch call, recorded once as a
    # CUDA graph and then replayed
    reqs = [(gid, q, trial_base + 20_000, args.steps) for q in qids.values()]
    P.cc_count_batch(ctx.h, reqs)  # eager run + capture (untimed)
    flush.zero_()
    b_ms, _ = dev_ms(lambda: P.cc_count_batch(ctx.h, reqs))
    batched = {"value": units_step * args.steps * world / (b_ms / 1e3) / 1e9, "unit": UNIT,
               "colorings_per_s": len(qids) * args.steps * world / (b_ms / 1e3),
               "ms_per_step": b_ms / args.steps, "timing": "CUDA events on the library's stream",
               "form": f"{len(qids)} requests x {args.steps} colourings per cc_count_batch call, CUDA-graph replay"}

    # the batched configuration: T colourings x 3 queries (C5, 4-cycle with a
    # chord and a pendant, glasses) on the same graph in one cc_count_batch
    # call replayed as a CUDA graph, against the same colourings counted one
    # cc_count call per colouring; both timed with CUDA events on the stream
    batch_cfg = None
    if args.batch_trials > 0:
        q3 = {name: ctx.set_query(*gg.query(name)) for name in BATCH_QUERIES}
        if args.heavy_degree < 0:
            for q in q3.values():
                P.cc_autotune(ctx.h, gid, q)
        for q in q3.values():
            P.cc_autotune_plan(ctx.h, gid, q)
        T3 = args.batch_trials
        first3 = trial_base + 30_000

        def both_forms(graph_id):
            reqs3 = [(graph_id, q, first3, T3) for q in q3.values()]
            P.cc_count_batch(ctx.h, reqs3)  # eager run + capture (untimed)
            flush.zero_()
            bm, (res3, st3) = dev_ms(lambda: P.cc_count_batch(ctx.h, reqs3))
            flush.zero_()
            pm, plain3 = dev_ms(lambda: {name: [int(ctx.count(graph_id, q, first3 + t, 1, allow_overflow=True)[0][0])
                                                for t in range(T3)] for name, q in q3.items()})
            equal = all([int(x) for x in res3[i]] == plain3[name] for i, name in enumerate(q3))
            return {"colorings_per_s_batched": len(q3) * T3 * world / (bm / 1e3),
                    "colorings_per_s_plain": len(q3) * T3 * world / (pm / 1e3),
                    "ms_batched": bm, "ms_plain": pm, "counts_equal_batched_vs_plain": bool(equal),
                    "status": st3}

        big = both_forms(gid)
        # the same comparison on a small graph (n = 1e4), where a colouring is
        # ~1 ms of kernels and per-call overhead is a large share
        gs = gg.chung_lu(10_000, 8, 2.1, 3)
        gid_s = ctx.load_graph(gs)
        small = both_forms(gid_s)
        ctx.free_graph(gid_s)
        small["workload"] = f"chung_lu n=10000 mean_deg=8 gamma=2.1 seed=3; {T3} colourings x {len(q3)} queries"
        batch_cfg = {"workload": f"{workload_name()}; {T3} colourings x {len(q3)} queries per cc_count_batch call",
                     "queries": list(q3), "trials": T3, **big, "small_graph": small,
                     "timing": "CUDA events on the library's stream around the whole batched call / all plain calls"}

    # configuration 1: Erdos-Renyi G(2000, 10^4), C5, seed 1; plain (one
    # cc_count per colouring) and batched (one cc_count_batch call)
    g1 = gg.erdos_renyi(2000, 10_000, 1)
    gid1 = ctx.load_graph(g1)
    q1 = ctx.set_query(*gg.query("C5"))
    T1 = 64
    P.cc_count_batch(ctx.h, [(gid1, q1, trial_base, T1)])  # eager run + capture (untimed)
    ctx.count(gid1, q1, trial_base, 1)
    p1_ms, c1_plain = dev_ms(lambda: [int(ctx.count(gid1, q1, trial_base + t, 1)[0][0]) for t in range(T1)])
    b1_ms, (c1_batch, _) = dev_ms(lambda: P.cc_count_batch(ctx.h, [(gid1, q1, trial_base, T1)]))
    config1 = {"workload": "erdos_renyi n=2000 m=10000 seed=1; C5; colouring seed 1", "colourings": T1,
               "first_colouring_count": c1_plain[0] if rank == 0 else None,
               "colorings_per_s_plain": T1 * world / (p1_ms / 1e3),
               "colorings_per_s_batched": T1 * world / (b1_ms / 1e3),
               "counts_equal_batched_vs_plain": [int(x) for x in c1_batch[0]] == c1_plain,
               "timing": "CUDA events on the library's stream"}
    ctx.free_graph(gid1)

    # end to end through the C-ABI with host buffers: load the CSR from
    # pinned host memory (the caller's buffers, filled once before the timed
    # steps), count both queries, read the counts back, free the graph
    import types
    g_pin = types.SimpleNamespace(
        n=g.n, nnz=g.nnz,
        row_ptr=torch.from_numpy(np.ascontiguousarray(g.row_ptr, dtype=np.int64)).pin_memory().numpy(),
        col=torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).pin_memory().numpy())
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        gid2 = ctx.load_graph(g_pin)
        for name, q in qids.items():
            ctx.count(gid2, q, trial_base + 50_000 + i, 1)
        ctx.free_graph(gid2)
    barrier()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    h2d = g.row_ptr.nbytes + g.col.nbytes
    e2e = {"value": units_step / e2e_s / 1e9 * world, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": 8 * len(qids) * 3, "ms_per_step": 1e3 * e2e_s, "host_buffers": "pinned"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": workload_name(), **WORKLOAD, "parallelism": f"replicas x{world}",
                       "l2": "256 MB flush between steps, outside the events; working set > L2",
                       "units_per_step": units_step, "units_by_query": units},
            "colorings_per_s": colourings, "wall_s": wall, "batched": batched, "batched_config": batch_cfg,
            "config1": config1,
            "heavy_degree": tuned, "decomposition_tree": trees,
            "kernel_ms": {k: {"ms": v[0], "launches": v[1]} for k, v in kern.items()},
            "gpu_launches": launches, "roofline": roofline, "kernel_rooflines": kernel_rooflines,
            "clocks": clocks, "e2e": e2e,
            "counts_first_step": counts[0] if counts else None}
    ctx.close()
    if rank == 0 and world == 1 and args.serve_leg > 0:
        # serving leg: a short Poisson stream at 70% of the measured capacity
        # (graph pool with one n = 1e6 graph), latency from arrival to result
        line["serving"] = serve_workload(args.serve_leg, True, args.workers, args.serve_budget, loads=(0.7,),
                                         progress=False)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_baseline(rounds=1)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
