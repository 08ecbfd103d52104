"""Serving loop: continuous batching with admission by table memory.

Each request's counts must equal the oracle's (stored values,
tests/golden/serving.txt, written by tests/golden/make_golden.py) and be the
same alone (a plain cc_count on its own context, same seed) and in the mix
(served concurrently with others); the server must actually run requests side
by side while keeping the memory it admits within the budget.
"""
import time

import numpy as np
import pytest

import golden_io
import graphgen as gg

pytestmark = pytest.mark.gpu

QUERIES = ["C4", "diamond", "C5", "chord_pendant", "C6", "glasses", "C6_2pendants"]


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_04478_gb300 as P
    gold = golden_io.load("serving")
    graphs = [gold.graph(name) for name in GRAPH_NAMES]
    return P, graphs, gold


GRAPH_NAMES = ["cl3000", "er2000", "cl20000"]


def _alone(P, g, k, e, seed, t0, T):
    ctx = P.Context(0)
    try:
        gid = ctx.load_graph(g)
        qid = ctx.set_query(k, e)
        P.cc_set_coloring_seed(ctx.h, seed)
        col, _, _ = ctx.count(gid, qid, t0, T, allow_overflow=True)
        return [int(x) for x in col]
    finally:
        ctx.close()


def _serve_all(srv, reqs, timeout_s=300):
    tickets = {}
    for i, (gi, qi, t0, T) in enumerate(reqs):
        tickets[srv.submit(gi, qi, t0, T)] = i
    out = {}
    t_end = time.time() + timeout_s
    while len(out) < len(reqs) and time.time() < t_end:
        for r in srv.poll(timeout_ms=200):
            out[tickets[r["ticket"]]] = r
    assert len(out) == len(reqs), "requests did not finish"
    return out


def test_results_same_alone_and_in_mix(env):
    P, graphs, gold = env
    srv = P.Server(0, workers=4)
    try:
        srv.set_seed(21)
        gids = [srv.load_graph(g) for g in graphs]
        qids = {name: srv.set_query(*gg.query(name)) for name in QUERIES}
        reqs = []
        for gname, qn, t0, T in gold.requests:
            gi = GRAPH_NAMES.index(gname)
            reqs.append((gids[gi], qids[qn], t0, T, gi, qn))
        out = _serve_all(srv, [r[:4] for r in reqs])
        for i, (gid, qid, t0, T, gi, qn) in enumerate(reqs):
            k, e = gg.query(qn)
            got = [int(x) for x in out[i]["colorful"]]
            oracle = [gold.counts[(GRAPH_NAMES[gi], qn, 21, t)][0] for t in range(t0, t0 + T)]
            assert got == oracle, (i, qn, gi)
            assert got == _alone(P, graphs[gi], k, e, 21, t0, T), (i, qn, gi)
            assert out[i]["status"] == 0
        # work of different requests overlapped on the device
        iv = sorted((r["admit_s"], r["done_s"]) for r in out.values())
        overlap = max(sum(1 for a, b in iv if a <= t < b) for t, _ in iv)
        assert overlap >= 2
    finally:
        srv.close()


def test_admission_respects_memory_budget(env):
    P, graphs, gold = env
    g = graphs[2]
    # edge-keyed table of chord_pendant on this graph: nnz x 3 x 8 bytes, plus colours
    need = g.nnz * 3 * 8 + g.n + 256
    srv = P.Server(0, workers=4, memory_budget=int(need * 1.5))
    try:
        srv.set_seed(3)
        gid = srv.load_graph(g)
        qid = srv.set_query(*gg.query("chord_pendant"))
        out = _serve_all(srv, [(gid, qid, t, 1) for t in range(6)])
        iv = sorted((r["admit_s"], r["done_s"]) for r in out.values())
        # at most one such request in flight at a time
        for (a0, b0), (a1, b1) in zip(iv, iv[1:]):
            assert a1 >= b0 - 1e-6
        k, e = gg.query("chord_pendant")
        for i in range(6):
            assert [int(x) for x in out[i]["colorful"]] == _alone(P, g, k, e, 3, i, 1)
            assert int(out[i]["colorful"][0]) == gold.counts[("cl20000", "chord_pendant", 3, i)][0]
        # a request that alone exceeds the budget is refused at submission
        big = srv.set_query(*gg.query("diamond"))
        small = P.Server(0, workers=1, memory_budget=1 << 20)
        try:
            sg = small.load_graph(g)
            sq = small.set_query(*gg.query("chord_pendant"))
            with pytest.raises(P.CCError) as ei:
                small.submit(sg, sq, 0, 1)
            assert P.ERRORS[ei.value.code] == "CC_ERR_OOM"
        finally:
            small.close()
        del big
    finally:
        srv.close()


def test_requests_arriving_while_others_run_are_admitted(env):
    P, graphs, gold = env
    srv = P.Server(0, workers=3)
    try:
        srv.set_seed(9)
        gids = [srv.load_graph(g) for g in graphs]
        q6 = srv.set_query(*gg.query("C6"))
        q4 = srv.set_query(*gg.query("C4"))
        # one long request and two short ones occupy the three workers
        long_t = srv.submit(gids[2], q6, 0, 24)
        short = [srv.submit(gids[0], q4, t, 1) for t in range(2)]
        time.sleep(0.01)
        # these arrive while the long one runs
        late = [srv.submit(gids[0], q4, 10 + t, 1) for t in range(4)]
        res = {}
        t_end = time.time() + 300
        while len(res) < 7 and time.time() < t_end:
            for r in srv.poll(timeout_ms=200):
                res[r["ticket"]] = r
        assert len(res) == 7
        long_done = res[long_t]["done_s"]
        # late arrivals took the slots the short requests freed, before the long one finished
        assert sum(res[t]["admit_s"] < long_done for t in late) >= 2
        k, e = gg.query("C4")
        for i, t in enumerate(late):
            assert [int(x) for x in res[t]["colorful"]] == _alone(P, graphs[0], k, e, 9, 10 + i, 1)
            assert int(res[t]["colorful"][0]) == gold.counts[("cl3000", "C4", 9, 10 + i)][0]
        k6, e6 = gg.query("C6")
        got = [int(x) for x in res[long_t]["colorful"]]
        assert got == _alone(P, graphs[2], k6, e6, 9, 0, 24)
        assert got == [gold.counts[("cl20000", "C6", 9, t)][0] for t in range(24)]
    finally:
        srv.close()
