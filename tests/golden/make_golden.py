#!/usr/bin/env python3
"""Write the stored expected values under tests/golden/ -- oracle only.

Every value written here is computed by the CPU oracle (``oracle/``, pinned
in tests/test_oracle_pins.py) on seeded graphs from ``graphgen``; nothing
comes from the CUDA library.  The GPU tests compare the library's counts with
these values where the oracle is too slow to run inside a test (queries with
k >= 7 on graphs of thousands of vertices, hub sources of the 10^6-vertex
benchmark graph).  Each file records the fingerprint (sha1 of the CSR) of
every graph it uses, so a test can check that it regenerated the same graph.

    python tests/golden/make_golden.py [--jobs N] [SET ...]

Sets: k7plus, mid, cl1e6, serving (default: all).  Counts are colourful
matches (Section 2 of the paper), colouring = (seed, trial) of the library's
hash colouring, which the oracle implements on its own.
"""
from __future__ import annotations

import argparse
import hashlib
import multiprocessing as mp
import os
import sys
import time
from concurrent.futures import ProcessPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

GRAPHS = {
    "er2000": "gg.erdos_renyi(2000, 10000, 1)",
    "cl3000": "gg.chung_lu(3000, 8, 2.1, 3)",
    "rmat10": "gg.rmat(10, 8, 0.57, 0.19, 0.19, 4)",
    "wheel": "gg.wheel_with_chords()",
    "cl30000": "gg.chung_lu(30000, 16, 2.1, 7)",
    "rmat13": "gg.rmat(13, 8, 0.57, 0.19, 0.19, 5)",
    "cl20000": "gg.chung_lu(20000, 12, 2.3, 4)",
    "cl1e6": "gg.chung_lu(1000000, 16, 2.1, 2)",
}
K7Q = ["glasses", "C5_pendant_path", "C6_2pendants", "C6_2pendants_adj", "C6_2pendants_same", "C7", "C8"]
SERVE_QUERIES = ["C4", "diamond", "C5", "chord_pendant", "C6", "glasses", "C6_2pendants"]
SERVE_GRAPHS = ["cl3000", "er2000", "cl20000"]

_graphs = {}


def graph(name):
    import graphgen as gg
    if name not in _graphs:
        _graphs[name] = eval(GRAPHS[name], {"gg": gg})
    return _graphs[name]


def fingerprint(g) -> str:
    import numpy as np
    h = hashlib.sha1()
    h.update(np.ascontiguousarray(g.row_ptr, dtype="<i8").tobytes())
    h.update(np.ascontiguousarray(g.col, dtype="<i4").tobytes())
    return h.hexdigest()


def run_task(task):
    """One oracle run.  task = (kind, graph, query, seed, trial, vertices):
    kind "count": the count; "all": the count and the per-source values of
    `vertices` (root cycle: split by highest cycle vertex); "filtered": the
    root cycle's highest vertex restricted to `vertices`, their values."""
    import numpy as np

    import graphgen as gg
    import oracle as O
    kind, gname, q, seed, trial, verts = task
    g = graph(gname)
    k, e = gg.query(q)
    col = O.colors(seed, trial, g.n, k)
    t0 = time.time()
    if kind == "count":
        cnt, ovf = O.dp_count(g, k, e, col)
        return task, {"value": cnt, "overflow": int(ovf)}, time.time() - t0
    filt = None
    if kind == "filtered":
        filt = np.zeros(g.n, dtype=np.uint8)
        filt[list(verts)] = 1
    cnt, ovf, per = O.dp_count(g, k, e, col, root_filter=filt, per_source=True)
    return task, {"value": cnt, "overflow": int(ovf), "per": {int(v): per[v] for v in verts}}, time.time() - t0


# ------------------------------------ sets ------------------------------------
def tasks_k7plus():
    t = []
    for gname in ["er2000", "cl3000", "rmat10"]:
        for q in K7Q:
            for trial in (0, 1):
                t.append(("count", gname, q, 7, trial, None))
    for q in ["glasses", "C5_pendant_path", "C6_2pendants", "C7"]:
        t.append(("count", "wheel", q, 5, 0, None))
    return t


def pick_sources(g, top, ranges, seed):
    """The `top` highest-degree vertices, then `count` random vertices with
    degree in [lo, hi) for each (lo, hi, count) of `ranges`."""
    import numpy as np
    deg = np.diff(g.row_ptr)
    rng = np.random.default_rng(seed)
    out = [int(v) for v in np.argsort(-deg, kind="stable")[:top]]
    for lo, hi, cnt in ranges:
        cand = np.setdiff1d(np.flatnonzero((deg >= lo) & (deg < hi)), out)
        out += [int(v) for v in rng.choice(cand, size=min(cnt, cand.size), replace=False)]
    return out


def tasks_mid():
    t = []
    for gname in ["rmat13", "cl30000"]:
        g = graph(gname)
        for q in ["triangle", "C4", "diamond", "chord_pendant", "glasses"]:
            t.append(("count", gname, q, 7, 0, None))
        srcs = tuple(pick_sources(g, 32, [(16, 256, 16), (256, 100000, 16)], 1))
        for q in ["C5", "C6"]:
            t.append(("all", gname, q, 7, 0, srcs))
        few = pick_sources(g, 6, [(64, 100000, 6), (8, 64, 6)], 2)
        for q in ["C5_pendant_path", "C6_2pendants"]:
            for v in few:
                t.append(("filtered", gname, q, 7, 0, (v,)))
    return t


def tasks_cl1e6():
    g = graph("cl1e6")
    t = []
    # C6 under the benchmark's colouring (seed 1, trial 0): one source per run
    for v in pick_sources(g, 8, [(1000, 100000, 12), (384, 1000, 8), (256, 384, 4)], 2):
        t.append(("filtered", "cl1e6", "C6", 1, 0, (v,)))
    for v in pick_sources(g, 4, [(1000, 100000, 4)], 3):
        t.append(("filtered", "cl1e6", "C5", 3, 0, (v,)))
    return t


def serving_requests():
    """The mixed request list of the serving test: (graph, query, first trial, trials)."""
    import numpy as np
    rng = np.random.default_rng(5)
    reqs = []
    for _ in range(36):
        gname = SERVE_GRAPHS[int(rng.integers(len(SERVE_GRAPHS)))]
        q = SERVE_QUERIES[int(rng.integers(len(SERVE_QUERIES)))]
        reqs.append((gname, q, int(rng.integers(0, 5)), int(rng.integers(1, 4))))
    return reqs


def tasks_serving():
    need = set()
    for gname, q, t0, T in serving_requests():
        for t in range(t0, t0 + T):
            need.add(("count", gname, q, 21, t, None))
    for t in range(6):
        need.add(("count", "cl20000", "chord_pendant", 3, t, None))
    for t in range(10, 14):
        need.add(("count", "cl3000", "C4", 9, t, None))
    for t in range(24):
        need.add(("count", "cl20000", "C6", 9, t, None))
    return sorted(need)


SETS = {"k7plus": tasks_k7plus, "mid": tasks_mid, "cl1e6": tasks_cl1e6, "serving": tasks_serving}


def write(name, tasks, results):
    used = sorted({t[1] for t in tasks})
    lines = [f"# Expected colourful-match counts computed by the CPU oracle (oracle/dp_count:",
             f"# the paper's decomposition, Section 4.1, and DB dynamic program, Section 5).",
             f"# Written by tests/golden/make_golden.py {name}; colouring = library hash (seed, trial)."]
    for gname in used:
        g = graph(gname)
        lines.append(f"graph {gname} {GRAPHS[gname].replace(' ', '')} n={g.n} nnz={g.nnz} sha1={fingerprint(g)}")
    if name == "serving":
        for i, (gname, q, t0, T) in enumerate(serving_requests()):
            lines.append(f"request {i} {gname} {q} first={t0} trials={T}")
    for task in tasks:
        kind, gname, q, seed, trial, verts = task
        r = results[task]
        lines.append(f"count {gname} {q} seed={seed} trial={trial} value={r['value']} overflow={r['overflow']}"
                     if kind != "filtered" else
                     f"filtered {gname} {q} seed={seed} trial={trial} sources={','.join(map(str, verts))} "
                     f"value={r['value']} overflow={r['overflow']}")
        if kind != "count":
            for v in verts:
                lines.append(f"source {gname} {q} seed={seed} trial={trial} vertex={v} value={r['per'][v]}")
    with open(os.path.join(HERE, f"{name}.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("sets", nargs="*", default=list(SETS))
    args = ap.parse_args()
    plan = {name: SETS[name]() for name in args.sets}
    # the longest runs (hub sources of the 10^6-vertex graph) first
    todo = sorted({t for ts in plan.values() for t in ts}, key=lambda t: (t[1] != "cl1e6", t[1], t[2], str(t[5])))
    results = {}
    with ProcessPoolExecutor(args.jobs, mp_context=mp.get_context("spawn")) as ex:
        for task, res, secs in ex.map(run_task, todo):
            results[task] = res
            print(f"{secs:8.1f} s  {task[:5]}", flush=True)
    for name, tasks in plan.items():
        write(name, tasks, results)


if __name__ == "__main__":
    main()
