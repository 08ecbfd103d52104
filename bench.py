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

--impl reference times the CPU oracle (single thread) on a bounded sample of
the same workload and prints the same line with "impl": "reference".
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
# DRAM bytes (read + written) of all C6 closure launches of one colouring of
# the workload at heavy threshold 384 (the autotuned one), from one ncu
# capture of the current kernels
CLOSURE_TRAFFIC_BYTES = 243.6e9
FLUSH_BYTES = 256 << 20


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
def oracle_sample(g, seconds_target: float, seed: int = 0, max_degree: int = 512):
    """Time the oracle's DP for C6 on a random sample of sources (highest
    cycle vertices) of degree <= max_degree, sized to about `seconds_target`
    seconds (hub sources are left out so the sample stays bounded).
    Returns (units of the sample, seconds, number of sources)."""
    import numpy as np

    import graphgen as gg
    import oracle as O
    k, e = gg.query("C6")
    col = O.colors(COLOR_SEED, 0, g.n, k)
    rng = np.random.default_rng(seed)
    deg = np.diff(g.row_ptr)
    cand = np.flatnonzero(deg <= max_degree)
    m = 200
    best = None
    for _ in range(4):
        pick = rng.choice(cand, size=min(m, cand.size), replace=False)
        filt = np.zeros(g.n, dtype=np.uint8)
        filt[pick] = 1
        t = {}
        O.dp_count(g, k, e, col, root_filter=filt, timing=t)
        secs = max(t["dp_seconds"], 1e-6)
        units = O.cycle_units(g, 6, k, source_filter=filt)
        best = (units, secs, int(filt.sum()))
        if secs >= seconds_target * 0.5 or m >= cand.size:
            break
        m = int(m * min(20.0, 0.8 * seconds_target / secs))
    return best


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    g = make_graph()
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for w in range(args.warmup):
        oracle_sample(g, min(per_step, 2.0), seed=100 + w)
    units_tot, secs_tot, srcs = 0.0, 0.0, 0
    for s in range(args.steps):
        u, sec, n = oracle_sample(g, per_step, seed=s)
        units_tot += u
        secs_tot += sec
        srcs += n
    value = units_tot / secs_tot / 1e9
    sample = (f"C6 DP restricted to {srcs} random highest-cycle-vertex sources of degree <= 512 over {args.steps} steps "
              f"(~{per_step:.0f} s of single-thread CPU each); glasses' table stages cannot be sampled by "
              f"source and are not timed")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs_tot / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": workload_name(), **WORKLOAD},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------ GPU arm ------------------------------------
def run_serve(args):
    """Serving workload: Chung-Lu graphs n in {1e4, 1e5, 1e6}, mean degree
    8-16, exponent 2.1-2.5 resident on the device; a Poisson stream of
    requests for treewidth-2 queries with k = 4..8 and 1-32 colourings each,
    served by the library's continuous-batching loop (cc_server_*).  Arrival
    rate: the given fraction of the capacity measured by a closed-loop
    burst.  Reports p50/p99 arrival-to-result latency and throughput."""
    import numpy as np

    import graphgen as gg
    import paper_1602_04478_gb300 as P

    rng = np.random.default_rng(5)
    sizes = [10_000, 100_000, 1_000_000]
    graphs = []
    for n in sizes:
        for d in (8, 12, 16):
            for gm in (2.1, 2.3, 2.5):
                if n == 1_000_000 and (d, gm) != (16, 2.5) and args.serve_small:
                    continue
                graphs.append(gg.chung_lu(n, d, gm, int(rng.integers(1 << 30))))
    srv = P.Server(0, workers=args.workers, memory_budget=args.serve_budget << 30)
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

    def drain(expected, submit_times):
        got, lat = 0, []
        while got < expected:
            for r in srv.poll(timeout_ms=500):
                got += 1
                lat.append(r["done_s"] - r["submit_s"])
        return lat

    # capacity: closed-loop burst of requests
    burst = [make_req() for _ in range(args.serve_requests // 4 or 1)]
    t0 = time.perf_counter()
    for rq in burst:
        srv.submit(*rq)
    drain(len(burst), None)
    cap = len(burst) / (time.perf_counter() - t0)
    out = {"impl": "ours", "mode": "serve", "graphs": len(graphs), "queries": qnames,
           "capacity_req_per_s": cap, "requests_per_rate": args.serve_requests, "rates": []}
    # progress lines (a cut-off run still leaves its measurements); the last line is the summary
    print(json.dumps({**out, "partial": True}), flush=True)
    for frac in (0.7, 1.0):
        lam = frac * cap
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=args.serve_requests))
        reqs = [make_req() for _ in range(args.serve_requests)]
        t0 = time.perf_counter()
        for at, rq in zip(arrivals, reqs):
            dt = at - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            srv.submit(*rq)
        lat = drain(len(reqs), None)
        wall = time.perf_counter() - t0
        colourings = sum(r[3] for r in reqs)
        out["rates"].append({"load": frac, "lambda_req_per_s": lam, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                             "p99_ms": 1e3 * float(np.percentile(lat, 99)), "req_per_s": len(reqs) / wall,
                             "colorings_per_s": colourings / wall})
        print(json.dumps({**out, "partial": True}), flush=True)
    srv.close()
    print(json.dumps(out), flush=True)
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


def run_profile_case(args):
    """One colouring of one query on the benchmark graph, nothing else: the
    command a profiler wraps to capture a few launches of one kernel."""
    import graphgen as gg
    import paper_1602_04478_gb300 as P

    g = make_graph()
    ctx = P.Context(0)
    gid = ctx.load_graph(g)
    P.cc_set_coloring_seed(ctx.h, COLOR_SEED)
    P.cc_set_heavy_degree(ctx.h, args.heavy_degree if args.heavy_degree >= 0 else 256)
    q = ctx.set_query(*gg.query(args.profile_case))
    col, _, _ = ctx.count(gid, q, 0, 1)
    print(json.dumps({"profile_case": args.profile_case, "colorful": int(col[0]),
                      "kernel_launches": P.cc_kernel_launches(ctx.h)}))
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
    ap.add_argument("--serve-budget", type=int, default=64, help="server table budget in GiB")
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--batch-trials", type=int, default=64,
                    help="colourings per query in the batched-configuration leg (0: skip it)")
    ap.add_argument("--heavy-degree", type=int, default=-1,
                    help="heavy/light source degree threshold (default: autotuned)")
    ap.add_argument("--profile-case", default=None, metavar="QUERY",
                    help="count QUERY once on the benchmark graph (one colouring, no timing) for profiler captures")
    ap.add_argument("--rmat-pendants", action="store_true",
                    help="R-MAT graph with the 8-node 6-cycle-with-two-pendants query instead")
    ap.add_argument("--rmat-scale", type=int, default=22)
    ap.add_argument("--rmat-trials", type=int, default=16)
    args = ap.parse_args()
    if args.rmat_pendants:
        return run_rmat_pendants(args)
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

    # Roofline of the dominant stage: the C6 root-cycle closure, a sequence of
    # kernels per colouring (heavy-source level builds and pulls, the per-CTA
    # push for the other sources).  Algorithmic bytes: 8 bytes per
    # edge-subset update (one u64 table entry read per update).
    closure = [k for k in kern if k.startswith("cycle_")]
    clo_ms = sum(kern[k][0] for k in closure)
    per_colouring_ms = clo_ms / args.steps
    peak, peak_kind = measured_peaks()
    achieved = 8.0 * units["C6"] / (per_colouring_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": "C6 root-cycle closure (" + " + ".join(sorted(closure)) + ")",
                "achieved": achieved, "peak": peak, "peak_source": peak_kind, "unit": "GB/s",
                "frac": achieved / peak, "traffic": CLOSURE_TRAFFIC_BYTES,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum over every closure launch of one "
                                  "colouring (profiles/dram_traffic_chunglu1e6_C6_colouring.md)",
                "avg_launch_ms": per_colouring_ms,
                "launches_per_colouring": sum(kern[k][1] for k in closure) / args.steps,
                "share_of_step": clo_ms / ms}

    # batched form: the same kind of step (one colouring of each query per
    # step) for K colourings in one cc_count_batch call, recorded once as a
    # CUDA graph and then replayed; timed on the host around the synchronous call
    reqs = [(gid, q, trial_base + 20_000, args.steps) for q in qids.values()]
    P.cc_count_batch(ctx.h, reqs)  # eager run + capture (untimed)
    barrier()
    tb0 = time.perf_counter()
    reps = 2
    for _ in range(reps):
        P.cc_count_batch(ctx.h, reqs)
    barrier()
    batched_s = (time.perf_counter() - tb0) / reps
    batched = {"value": units_step * args.steps * world / batched_s / 1e9, "unit": UNIT,
               "colorings_per_s": len(qids) * args.steps * world / batched_s,
               "ms_per_step": 1e3 * batched_s / args.steps, "timing": "host clock around synchronous calls",
               "form": f"{len(qids)} requests x {args.steps} colourings per cc_count_batch call, CUDA-graph replay"}

    # the batched configuration: T colourings x 3 queries (C5, 4-cycle with a
    # chord and a pendant, glasses) on the same graph in one cc_count_batch
    # call replayed as a CUDA graph, against the same colourings counted one
    # cc_count call per colouring (a subset of them, to keep the leg short)
    batch_cfg = None
    if args.batch_trials > 0:
        q3 = {name: ctx.set_query(*gg.query(name)) for name in BATCH_QUERIES}
        if args.heavy_degree < 0:
            for q in q3.values():
                P.cc_autotune(ctx.h, gid, q)
        T3 = args.batch_trials
        first3 = trial_base + 30_000
        reqs3 = [(gid, q, first3, T3) for q in q3.values()]
        P.cc_count_batch(ctx.h, reqs3)  # eager run + capture (untimed)
        barrier()
        t0 = time.perf_counter()
        res3, st3 = P.cc_count_batch(ctx.h, reqs3)
        barrier()
        b3 = time.perf_counter() - t0
        Tp = min(T3, 8)
        plain3 = {}
        barrier()
        t0 = time.perf_counter()
        for name, q in q3.items():
            plain3[name] = [int(ctx.count(gid, q, first3 + t, 1)[0][0]) for t in range(Tp)]
        barrier()
        p3 = time.perf_counter() - t0
        equal = all([int(x) for x in res3[i][:Tp]] == plain3[name] for i, name in enumerate(q3))
        # the same comparison on a small graph (n = 1e4), where a colouring is
        # ~1 ms of kernels and per-call overhead is what batching removes
        gs = gg.chung_lu(10_000, 8, 2.1, 3)
        gid_s = ctx.load_graph(gs)
        reqs_s = [(gid_s, q, first3, T3) for q in q3.values()]
        P.cc_count_batch(ctx.h, reqs_s)  # eager run + capture (untimed)
        barrier()
        t0 = time.perf_counter()
        res_s, _ = P.cc_count_batch(ctx.h, reqs_s)
        barrier()
        bs = time.perf_counter() - t0
        plain_s = {}
        barrier()
        t0 = time.perf_counter()
        for name, q in q3.items():
            plain_s[name] = [int(ctx.count(gid_s, q, first3 + t, 1)[0][0]) for t in range(T3)]
        barrier()
        ps = time.perf_counter() - t0
        equal_s = all([int(x) for x in res_s[i]] == plain_s[name] for i, name in enumerate(q3))
        ctx.free_graph(gid_s)
        batch_cfg_small = {"workload": f"chung_lu n=10000 mean_deg=8 gamma=2.1 seed=3; {T3} colourings x "
                                       f"{len(q3)} queries per cc_count_batch call",
                           "colorings_per_s_batched": len(q3) * T3 * world / bs,
                           "colorings_per_s_plain": len(q3) * T3 * world / ps,
                           "counts_equal_batched_vs_plain": bool(equal_s)}
        batch_cfg = {"workload": f"{workload_name()}; {T3} colourings x {len(q3)} queries per cc_count_batch call",
                     "small_graph": batch_cfg_small,
                     "queries": list(q3), "trials": T3,
                     "colorings_per_s_batched": len(q3) * T3 * world / b3,
                     "colorings_per_s_plain": len(q3) * Tp * world / p3,
                     "ms_batched_call": 1e3 * b3, "plain_trials_timed": Tp,
                     "counts_equal_batched_vs_plain": bool(equal), "status": st3,
                     "timing": "host clock around synchronous calls; batched = CUDA-graph replay of all passes"}

    # end to end through the C-ABI with host buffers: load the CSR from host
    # memory, count both queries, read the counts back, free the graph
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        gid2 = ctx.load_graph(g)
        for name, q in qids.items():
            ctx.count(gid2, q, trial_base + 50_000 + i, 1)
        ctx.free_graph(gid2)
    barrier()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    h2d = g.row_ptr.nbytes + g.col.nbytes
    e2e = {"value": units_step / e2e_s / 1e9 * world, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": 8 * len(qids) * 3, "ms_per_step": 1e3 * e2e_s}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": workload_name(), **WORKLOAD, "parallelism": f"replicas x{world}",
                       "l2": "256 MB flush between steps, outside the events; working set > L2",
                       "units_per_step": units_step, "units_by_query": units},
            "colorings_per_s": colourings, "wall_s": wall, "batched": batched, "batched_config": batch_cfg,
            "heavy_degree": tuned,
            "kernel_ms": {k: {"ms": v[0], "launches": v[1]} for k, v in kern.items()},
            "gpu_launches": launches, "roofline": roofline, "clocks": clocks, "e2e": e2e,
            "counts_first_step": counts[0] if counts else None}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        u, s, nsrc = oracle_sample(g, 15.0)
        line["cpu_baseline"] = {"value": u / s / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"C6 DP (single thread) restricted to {nsrc} random highest-vertex "
                                          f"sources of degree <= 512 of the same graph and colouring: "
                                          f"{u:.3g} updates in {s:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
