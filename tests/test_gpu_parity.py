"""CUDA path against the CPU oracle: bit-exact uint64 colourful counts.

Every count goes through the C-ABI (``paper_1602_04478_gb300`` binding) and is
compared with ``oracle.dp_count`` (pinned to brute force and closed forms in
test_oracle_pins.py) on the same seeded graph and the same colouring.
"""
import math

import numpy as np
import pytest

import golden_io
import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu

QUERIES = dict(gg.QUERIES)
QUERIES.update({
    "path4": (4, [(0, 1), (1, 2), (2, 3)]),
    "star4": (5, [(0, 1), (0, 2), (0, 3), (0, 4)]),
    "tailed_triangle": (4, [(0, 1), (1, 2), (2, 0), (2, 3)]),
    "bowtie": (5, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 2)]),
    "house": (5, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (4, 1)]),
    "chord_pendant0": (5, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2), (0, 4)]),
    "C6_2pendants_adj": (8, [(i, (i + 1) % 6) for i in range(6)] + [(0, 6), (1, 7)]),
    "C6_2pendants_same": (8, [(i, (i + 1) % 6) for i in range(6)] + [(0, 6), (0, 7)]),
    "C7": gg.cycle(7),
    "C8": gg.cycle(8),
    "triangle_strip": (5, [(0, 1), (1, 2), (2, 0), (1, 3), (2, 3), (2, 4), (3, 4)]),
    "C5_pendant_path": (7, [(i, (i + 1) % 5) for i in range(5)] + [(0, 5), (5, 6)]),
})


@pytest.fixture(scope="module")
def cc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_04478_gb300 as P
    ctx = P.Context(0)
    yield ctx
    ctx.close()


GRAPHS = {
    "er60": lambda: gg.erdos_renyi(60, 300, 1),
    "er2000": lambda: gg.erdos_renyi(2000, 10000, 1),
    "cl3000": lambda: gg.chung_lu(3000, 8, 2.1, 3),
    "rmat10": lambda: gg.rmat(10, 8, 0.57, 0.19, 0.19, 4),
}
_cache = {}


def graph(name):
    if name not in _cache:
        _cache[name] = GRAPHS[name]()
    return _cache[name]


def gpu_count(cc, g, gid, k, edges, seed, trials):
    import paper_1602_04478_gb300 as P
    qid = cc.set_query(k, edges)
    P.cc_set_coloring_seed(cc.h, seed)
    col, est, aut = cc.count(gid, qid, 0, trials)
    return col, est, aut, qid


@pytest.mark.parametrize("gname", ["er60", "er2000", "cl3000", "rmat10"])
@pytest.mark.parametrize("qname", sorted(QUERIES))
def test_count_matches_oracle(cc, gname, qname):
    g = graph(gname)
    k, e = QUERIES[qname]
    # queries with k >= 7 on the larger graphs: the oracle's values are stored
    # (tests/golden/k7plus.txt, written by tests/golden/make_golden.py)
    stored = None
    if gname != "er60" and k >= 7:
        gold = golden_io.load("k7plus")
        assert golden_io.fingerprint(g) == gold.graph_sha[gname]
        stored = gold.counts
    gid = cc.load_graph(g)
    try:
        seed = 7
        trials = 2
        col, est, aut, qid = gpu_count(cc, g, gid, k, e, seed, trials)
        assert aut == O.automorphisms(k, e)
        for t in range(trials):
            if stored is not None:
                expect, ovf = stored[(gname, qname, seed, t)]
            else:
                expect, ovf = O.dp_count(g, k, e, O.colors(seed, t, g.n, k))
            assert not ovf
            assert int(col[t]) == expect, (qname, gname, t)
            scale = k ** k / math.factorial(k) / aut
            assert est[t] == pytest.approx(expect * scale, rel=1e-12)
    finally:
        cc.free_graph(gid)


@pytest.mark.parametrize("heavy", [0, 3, 12, 1 << 30])
@pytest.mark.parametrize("qname", ["C4", "C5", "C6", "C6_2pendants", "C6_2pendants_adj", "C7", "C8",
                                   "C5_pendant_path"])
def test_heavy_light_split(cc, heavy, qname):
    # every source through the grouped heavy path (0), mixed splits, or the
    # per-CTA path only: identical counts, equal to the oracle's
    import paper_1602_04478_gb300 as P
    k, e = QUERIES[qname]
    g = graph("cl3000") if k <= 6 else graph("er60")
    gid = cc.load_graph(g)
    try:
        P.cc_set_heavy_degree(cc.h, heavy)
        P.cc_set_coloring_seed(cc.h, 4)
        qid = cc.set_query(k, e)
        pv, total = cc.count_per_vertex(gid, qid, 0)
        expect, _, per = O.dp_count(g, k, e, O.colors(4, 0, g.n, k), per_source=True)
        assert total == expect
        assert [int(x) for x in pv] == per
    finally:
        P.cc_set_heavy_degree(cc.h, -1)
        cc.free_graph(gid)


def _same_root(k, e, seq=None):
    """Whether the library's root block (default or explicit tree) is the
    oracle's root block: then their per-vertex splits are the same."""
    import paper_1602_04478_gb300 as P
    blocks, root, _ = O.decompose(k, e)
    lib_root = P.cc_plan_inspect(k, e, seq or None)[0][-1]
    if lib_root["kind"] in ("root_cycle", "triangle") and blocks[root]["kind"] == "root_cycle":
        return sorted(lib_root["nodes"]) == sorted(blocks[root]["nodes"])
    return lib_root["kind"] == "root_node" == blocks[root]["kind"] and lib_root["nodes"] == blocks[root]["nodes"]


def _wheel_with_chords():
    # a hub adjacent to all 9000 other vertices (more lower neighbours than
    # the shared-memory hash holds: the CTA kernel scans it by binary search),
    # a ring through them and random chords (many hashed sources of degree >= 32)
    return gg.wheel_with_chords()


@pytest.mark.parametrize("listed", [True, False])
@pytest.mark.parametrize("qname", ["triangle", "diamond", "chord_pendant", "tailed_triangle", "bowtie"])
def test_triangle_sources_of_every_degree(cc, qname, listed):
    # triangle blocks listed from sources of low degree (one warp each),
    # hashed hub sources (one CTA each) and a source above the hash capacity;
    # streamed from the graph's triangle list, or scanned every colouring
    import paper_1602_04478_gb300 as P
    g = _wheel_with_chords()
    k, e = QUERIES[qname]
    P.cc_set_triangle_list(cc.h, listed)
    gid = cc.load_graph(g)
    try:
        P.cc_set_coloring_seed(cc.h, 5)
        qid = cc.set_query(k, e)
        # the tree the paper's factors pick: its root is the triangle block the
        # oracle's split is by (the library's own pick may end at a leaf)
        seq = [t for t in P.cc_plan_enumerate(k, e) if t["paper"]][0]["seq"]
        if seq:
            P.cc_set_decomposition(cc.h, qid, seq)
        P.cc_set_timing(cc.h, True)
        P.cc_reset_timing(cc.h)
        pv, total = cc.count_per_vertex(gid, qid, 0)
        names = P.cc_get_timing(cc.h)
        P.cc_set_timing(cc.h, False)
        assert any(n.startswith("triangle_list_") and n != "triangle_list_build" for n in names) == listed, names
        expect, _, per = O.dp_count(g, k, e, O.colors(5, 0, g.n, k), per_source=True)
        assert total == expect
        if _same_root(k, e, seq):
            assert [int(x) for x in pv] == per
    finally:
        P.cc_set_triangle_list(cc.h, True)
        cc.free_graph(gid)


@pytest.mark.parametrize("gname", ["cl3000", "rmat10"])
def test_triangle_list_against_wedge_scan(cc, gname):
    # the same counts whether triangle blocks stream the list or scan wedges,
    # for every triangle form (plain, one annotation, general; unary,
    # edge-keyed and root outputs), equal to the oracle's
    import paper_1602_04478_gb300 as P
    g = graph(gname)
    gid = cc.load_graph(g)
    try:
        P.cc_set_coloring_seed(cc.h, 12)
        for qname in ["triangle", "diamond", "chord_pendant", "chord_pendant0", "bowtie", "triangle_strip", "house"]:
            k, e = QUERIES[qname]
            qid = cc.set_query(k, e)
            got = {}
            for listed in (True, False):
                P.cc_set_triangle_list(cc.h, listed)
                got[listed] = [int(x) for x in cc.count(gid, qid, 0, 2)[0]]
            P.cc_set_triangle_list(cc.h, True)
            want = [O.dp_count(g, k, e, O.colors(12, t, g.n, k))[0] for t in range(2)]
            assert got[True] == got[False] == want, qname
    finally:
        P.cc_set_triangle_list(cc.h, True)
        cc.free_graph(gid)


def test_triangle_list_above_memory_cap_falls_back(cc):
    # a list that would not fit a quarter of the budget is not built: the
    # triangle kernels scan wedges instead, with the same counts
    import paper_1602_04478_gb300 as P
    ctx = P.Context(0)
    try:
        # the wheel graph: 39,078 triangles (1.4 MB listed), 1.4 MB of graph
        # arrays, 3.6 MB of glasses tables: a 6 MB budget leaves the list
        # less than its size
        g = _wheel_with_chords()
        gid = ctx.load_graph(g)
        P.cc_set_memory_budget(ctx.h, 6 << 20)
        k, e = QUERIES["glasses"]
        qid = ctx.set_query(k, e)
        P.cc_set_coloring_seed(ctx.h, 2)
        P.cc_set_timing(ctx.h, True)
        got = int(ctx.count(gid, qid, 0, 1)[0][0])
        names = P.cc_get_timing(ctx.h)
        # the build was tried and given up: the blocks scanned wedges
        assert "triangle_list_build" in names, names
        assert not any(n.startswith("triangle_list_") and n != "triangle_list_build" for n in names), names
        assert any(n in ("triangle_plain", "triangle_join1", "triangle_join") for n in names), names
        P.cc_set_memory_budget(ctx.h, 0)
        assert got == O.dp_count(g, k, e, O.colors(2, 0, g.n, k))[0]
    finally:
        ctx.close()


@pytest.mark.parametrize("qname", ["glasses", "C5_pendant_path", "C6_2pendants", "C7"])
def test_large_queries_on_the_wheel(cc, qname):
    # the benchmark's glasses and the doubly annotated cycles on a graph whose
    # triangle blocks reach the hashed hub kernel and the hub above the hash
    # capacity; stored oracle values (tests/golden/k7plus.txt)
    import paper_1602_04478_gb300 as P
    gold = golden_io.load("k7plus")
    g = gold.graph("wheel")
    k, e = QUERIES[qname]
    gid = cc.load_graph(g)
    try:
        P.cc_set_coloring_seed(cc.h, 5)
        qid = cc.set_query(k, e)
        got = int(cc.count(gid, qid, 0, 1)[0][0])
        assert got == gold.counts[("wheel", qname, 5, 0)][0]
    finally:
        cc.free_graph(gid)


@pytest.mark.parametrize("qname", ["C5", "C6"])
def test_both_level_build_forms(cc, qname):
    # with every source heavy, the highest groups build their levels in the
    # pull form and the rest in the push form; both feed the same closure
    import paper_1602_04478_gb300 as P
    k, e = QUERIES[qname]
    g = graph("cl3000")
    gid = cc.load_graph(g)
    P.cc_set_heavy_degree(cc.h, 0)
    try:
        P.cc_set_coloring_seed(cc.h, 8)
        qid = cc.set_query(k, e)
        P.cc_set_timing(cc.h, True)
        P.cc_reset_timing(cc.h)
        pv, total = cc.count_per_vertex(gid, qid, 0)
        names = P.cc_get_timing(cc.h)
        P.cc_set_timing(cc.h, False)
        assert "cycle_plain_levels_pull" in names and "cycle_plain_levels" in names, names
        expect, _, per = O.dp_count(g, k, e, O.colors(8, 0, g.n, k), per_source=True)
        assert total == expect
        assert [int(x) for x in pv] == per
        # and again, from the zero state the pass leaves behind
        col, _, _ = cc.count(gid, qid, 0, 1)
        assert int(col[0]) == expect
    finally:
        P.cc_set_heavy_degree(cc.h, -1)
        cc.free_graph(gid)


def test_scratch_reuse_across_graphs_and_queries(cc):
    # one context counts different graphs and cycle lengths in turn, every
    # source on the heavy path: scratch left by one (graph, query) must not
    # leak into the next, whose layout differs
    import paper_1602_04478_gb300 as P
    seq = [("er60", "C6"), ("cl3000", "C5"), ("er2000", "C6"), ("rmat10", "C4"), ("cl3000", "C6"), ("er60", "C5")]
    P.cc_set_heavy_degree(cc.h, 0)
    try:
        for gname, qname in seq:
            g = graph(gname)
            k, e = QUERIES[qname]
            gid = cc.load_graph(g)
            try:
                P.cc_set_coloring_seed(cc.h, 13)
                qid = cc.set_query(k, e)
                col, _, _ = cc.count(gid, qid, 0, 1)
                expect, _ = O.dp_count(g, k, e, O.colors(13, 0, g.n, k))
                assert int(col[0]) == expect, (gname, qname)
            finally:
                cc.free_graph(gid)
    finally:
        P.cc_set_heavy_degree(cc.h, -1)


def test_explicit_colours_and_brute_force(cc):
    import paper_1602_04478_gb300 as P
    g = graph("er60")
    gid = cc.load_graph(g)
    try:
        for qname in ["C5", "C6", "glasses", "chord_pendant", "C6_2pendants", "diamond"]:
            k, e = QUERIES[qname]
            rng = np.random.default_rng(3)
            cols = rng.integers(0, k, size=(3, g.n)).astype(np.uint8)
            P.cc_set_colors(cc.h, gid, cols)
            qid = cc.set_query(k, e)
            got, _, _ = cc.count(gid, qid, 0, 3)
            for t in range(3):
                assert int(got[t]) == O.brute_colorful(g, k, e, cols[t])
            P.cc_clear_colors(cc.h, gid)
    finally:
        cc.free_graph(gid)


@pytest.mark.parametrize("qname", ["C4", "C5", "C6", "C6_2pendants", "chord_pendant", "diamond", "glasses",
                                   "C7", "C8"])
def test_per_vertex_split_matches_oracle(cc, qname):
    g = graph("er2000") if QUERIES[qname][0] < 7 else graph("er60")
    k, e = QUERIES[qname]
    import paper_1602_04478_gb300 as P
    gid = cc.load_graph(g)
    try:
        qid = cc.set_query(k, e)
        P.cc_set_coloring_seed(cc.h, 11)
        pv, total = cc.count_per_vertex(gid, qid, 0)
        cols = O.colors(11, 0, g.n, k)
        expect, _, per = O.dp_count(g, k, e, cols, per_source=True)
        assert total == expect == int(pv.sum())
        # the split is by the root block: compare when the library's and the
        # oracle's roots are the same block (same kind, same query nodes)
        if _same_root(k, e):
            assert [int(x) for x in pv] == per
    finally:
        cc.free_graph(gid)


def test_decomposition_invariance(cc):
    import paper_1602_04478_gb300 as P
    g = graph("er2000")
    k, e = QUERIES["chord_pendant"]
    orders = [
        [0, 1, 4, 3, 0, 1, 2],   # leaf (1,4), then triangle (0,1,2); root triangle (0,2,3)
        [3, 0, 2, 3, 0, 1, 4],   # triangle (0,2,3) first, then the leaf; root triangle (0,1,2)
        [0, 1, 4, 3, 0, 2, 3],   # leaf, then triangle (0,2,3); root triangle (0,1,2)
    ]
    gid = cc.load_graph(g)
    try:
        P.cc_set_coloring_seed(cc.h, 5)
        got = []
        for seq in orders:
            qid = cc.set_query(k, e)
            P.cc_set_decomposition(cc.h, qid, seq)
            got.append(int(cc.count(gid, qid, 0, 1)[0][0]))
        expect = O.dp_count(g, k, e, O.colors(5, 0, g.n, k))[0]
        assert got == [expect] * len(orders)
    finally:
        cc.free_graph(gid)


def test_relabel_invariance(cc):
    import paper_1602_04478_gb300 as P
    g = graph("cl3000")
    perm = np.random.default_rng(1).permutation(g.n)
    h = gg.relabel(g, perm)
    k, e = QUERIES["C5"]
    cols = O.colors(2, 0, g.n, k)
    colh = np.zeros_like(cols)
    colh[perm] = cols
    a, b = cc.load_graph(g), cc.load_graph(h)
    try:
        P.cc_set_colors(cc.h, a, cols)
        P.cc_set_colors(cc.h, b, colh)
        qid = cc.set_query(k, e)
        assert int(cc.count(a, qid)[0][0]) == int(cc.count(b, qid)[0][0])
    finally:
        cc.free_graph(a)
        cc.free_graph(b)


# ------------------------------ edge cases ------------------------------
def test_empty_and_tiny_graphs(cc):
    import paper_1602_04478_gb300 as P
    P.cc_set_coloring_seed(cc.h, 1)
    for g in [gg.from_edges(5, []), gg.from_edges(3, [(0, 1)]), gg.from_edges(4, [(0, 1), (1, 2), (2, 0)])]:
        gid = cc.load_graph(g)
        try:
            for qname in ["triangle", "C4", "glasses", "path4"]:
                k, e = QUERIES[qname]
                qid = cc.set_query(k, e)
                got = cc.count(gid, qid, 0, 1)[0]
                assert int(got[0]) == O.dp_count(g, k, e, O.colors(1, 0, g.n, k))[0]
        finally:
            cc.free_graph(gid)


def test_complete_graph_closed_form(cc):
    import paper_1602_04478_gb300 as P
    g = gg.complete_graph(40)
    gid = cc.load_graph(g)
    try:
        for L in (3, 4, 5, 6):
            k, e = gg.cycle(L)
            qid = cc.set_query(k, e)
            P.cc_set_coloring_seed(cc.h, 9)
            got = int(cc.count(gid, qid)[0][0])
            nc = np.bincount(O.colors(9, 0, g.n, k), minlength=k).astype(object)
            assert got == math.factorial(k) * int(np.prod(nc))
    finally:
        cc.free_graph(gid)


@pytest.mark.parametrize("edges,code", [
    ([(a, b) for a in range(4) for b in range(a + 1, 4)], "CC_ERR_NOT_TW2"),
    ([(0, 1), (2, 3)], "CC_ERR_NOT_CONNECTED"),
    ([(0, 1), (1, 0)], "CC_ERR_INVALID_ARG"),
    ([(0, 0)], "CC_ERR_INVALID_ARG"),
])
def test_query_errors(cc, edges, code):
    import paper_1602_04478_gb300 as P
    k = 1 + max(max(x) for x in edges)
    with pytest.raises(P.CCError) as ei:
        cc.set_query(max(k, 2), edges)
    assert P.ERRORS[ei.value.code] == code


def test_k_range_error(cc):
    import paper_1602_04478_gb300 as P
    for k in (1, 13):
        with pytest.raises(P.CCError) as ei:
            cc.set_query(k, [(i, i + 1) for i in range(k - 1)] or [(0, 0)])
        assert ei.value.code in (-4, -1)


def test_unsupported_block_reported(cc):
    # a 9-cycle: longer than the cycle kernel's 8 nodes, and its only tree
    import paper_1602_04478_gb300 as P
    e = [(i, (i + 1) % 9) for i in range(9)]
    with pytest.raises(P.CCError) as ei:
        cc.set_query(9, e)
    assert P.ERRORS[ei.value.code] == "CC_ERR_UNSUPPORTED"


@pytest.mark.parametrize("bad", ["asym", "loop", "dup", "range"])
def test_bad_graph_rejected(cc, bad):
    import paper_1602_04478_gb300 as P
    if bad == "asym":
        rp, col = np.array([0, 1, 1, 1]), np.array([1])
    elif bad == "loop":
        rp, col = np.array([0, 2, 3, 4]), np.array([0, 1, 0, 0])
    elif bad == "dup":
        rp, col = np.array([0, 2, 4, 4]), np.array([1, 1, 0, 0])
    else:
        rp, col = np.array([0, 1, 2, 2]), np.array([7, 0])
    with pytest.raises(P.CCError) as ei:
        P.cc_load_csr(cc.h, 3, rp, col)
    assert P.ERRORS[ei.value.code] == "CC_ERR_BAD_GRAPH"


def test_overflow_reported_not_wrapped(cc):
    import paper_1602_04478_gb300 as P
    k = 12
    e = [(0, i) for i in range(1, k)]
    D = 3000
    g = gg.from_edges(D + 1, [(0, i) for i in range(1, D + 1)])
    gid = cc.load_graph(g)
    try:
        qid = cc.set_query(k, e)
        P.cc_set_coloring_seed(cc.h, 1)
        with pytest.raises(P.CCError) as ei:
            cc.count(gid, qid, 0, 1)
        assert P.ERRORS[ei.value.code] == "CC_ERR_OVERFLOW"
        col, _, _ = cc.count(gid, qid, 0, 1, allow_overflow=True)
        assert int(col[0]) == 2**64 - 1
        assert O.dp_count(g, k, e, O.colors(1, 0, g.n, k))[1]
    finally:
        cc.free_graph(gid)


def test_memory_budget_oom(cc):
    # admission by table memory: the edge-keyed table of chord_pendant
    # (nnz x 3 x 8 bytes) does not fit the budget, so the count is refused
    # before any launch and the context stays usable
    import paper_1602_04478_gb300 as P
    ctx = P.Context(0)
    try:
        g = gg.chung_lu(200000, 16, 2.1, 2)
        gid = ctx.load_graph(g)
        qid = ctx.set_query(*QUERIES["chord_pendant"])
        P.cc_set_memory_budget(ctx.h, 64 << 20)
        with pytest.raises(P.CCError) as ei:
            ctx.count(gid, qid)
        assert P.ERRORS[ei.value.code] == "CC_ERR_OOM"
        P.cc_set_memory_budget(ctx.h, 0)
        k, e = QUERIES["chord_pendant"]
        got = int(ctx.count(gid, qid)[0][0])
        P.cc_set_coloring_seed(ctx.h, 1)
        assert got == int(ctx.count(gid, qid)[0][0])
    finally:
        ctx.close()


# ------------------------------ batched form ------------------------------
@pytest.mark.parametrize("lanes", [1, 2, 3])
@pytest.mark.parametrize("capture", [True, False])
def test_batch_equals_plain(cc, capture, lanes):
    # the batched form, replayed as a CUDA graph or run eagerly, on one lane
    # or several concurrent ones: the same counts as one cc_count per colouring
    import paper_1602_04478_gb300 as P
    g1, g2 = graph("cl3000"), graph("er2000")
    a, b = cc.load_graph(g1), cc.load_graph(g2)
    try:
        P.cc_set_graph_capture(cc.h, capture)
        P.cc_set_batch_lanes(cc.h, lanes)
        P.cc_set_coloring_seed(cc.h, 3)
        qs = {name: cc.set_query(*QUERIES[name]) for name in ["C5", "chord_pendant", "glasses", "C6", "C4"]}
        reqs = [(a, qs["C5"], 0, 4), (a, qs["chord_pendant"], 2, 3), (b, qs["glasses"], 0, 2),
                (b, qs["C6"], 5, 2), (a, qs["C4"], 1, 1)]
        for rep in range(3):  # first call runs eagerly and records; later calls replay
            res, st = P.cc_count_batch(cc.h, reqs)
            assert st == [0] * len(reqs)
            for (gid, qid, t0, T), got in zip(reqs, res):
                want = cc.count(gid, qid, t0, T)[0]
                assert [int(x) for x in got] == [int(x) for x in want], (rep, gid, qid)
        # oracle spot check of one request
        k, e = QUERIES["C5"]
        assert int(res[0][1]) == O.dp_count(g1, k, e, O.colors(3, 1, g1.n, k))[0]
    finally:
        P.cc_set_batch_lanes(cc.h, 2)
        P.cc_set_graph_capture(cc.h, True)
        cc.free_graph(a)
        cc.free_graph(b)


def test_autotune_keeps_counts(cc):
    import paper_1602_04478_gb300 as P
    g = graph("cl3000")
    gid = cc.load_graph(g)
    try:
        P.cc_set_coloring_seed(cc.h, 8)
        qid = cc.set_query(*QUERIES["C6"])
        before = [int(x) for x in cc.count(gid, qid, 0, 2)[0]]
        hd = P.cc_autotune(cc.h, gid, qid)
        # the tuner's candidate thresholds
        assert hd in (64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096)
        assert [int(x) for x in cc.count(gid, qid, 0, 2)[0]] == before
        res, _ = P.cc_count_batch(cc.h, [(gid, qid, 0, 2)])
        assert [int(x) for x in res[0]] == before
    finally:
        cc.free_graph(gid)


@pytest.mark.parametrize("gname", ["er2000", "cl3000", "rmat10"])
@pytest.mark.parametrize("L", [4, 5, 6])
def test_work_units_match_oracle(cc, gname, L):
    # the benchmark's work unit, counted on the device, equals the oracle's
    # plain-loop structural count of the DB procedure
    import paper_1602_04478_gb300 as P
    g = graph(gname)
    gid = cc.load_graph(g)
    try:
        qid = cc.set_query(*gg.cycle(L))
        assert P.cc_work_units(cc.h, gid, qid) == O.cycle_units(g, L, L)
    finally:
        cc.free_graph(gid)


@pytest.mark.parametrize("heavy", [-1, 64])
@pytest.mark.parametrize("gname", ["rmat13", "cl30000"])
def test_mid_size_graphs_match_stored_oracle(cc, gname, heavy):
    # R-MAT scale 13 (maximum degree 1,502) and Chung-Lu n = 30,000: every
    # benchmark query against stored oracle values (tests/golden/mid.txt),
    # totals and the split by highest cycle vertex for sampled sources of
    # every degree class, at the library's threshold and with most sources on
    # the grouped heavy path
    import paper_1602_04478_gb300 as P
    gold = golden_io.load("mid")
    g = gold.graph(gname)
    gid = cc.load_graph(g)
    P.cc_set_heavy_degree(cc.h, heavy)
    try:
        for (gn, q, seed, trial), (want, ovf) in gold.counts.items():
            if gn != gname:
                continue
            assert not ovf
            P.cc_set_coloring_seed(cc.h, seed)
            qid = cc.set_query(*gg.query(q))
            assert int(cc.count(gid, qid, trial, 1)[0][0]) == want, (gname, q)
        for (gn, q, seed, trial), per in gold.sources.items():
            if gn != gname:
                continue
            P.cc_set_coloring_seed(cc.h, seed)
            qid = cc.set_query(*gg.query(q))
            pv, total = cc.count_per_vertex(gid, qid, trial)
            assert int(pv.sum()) == total
            for v, want in per.items():
                assert int(pv[v]) == want, (gname, q, v)
    finally:
        P.cc_set_heavy_degree(cc.h, -1)
        cc.free_graph(gid)


@pytest.mark.parametrize("qname", ["chord_pendant", "glasses", "triangle_strip"])
def test_autotune_plan_keeps_counts(cc, qname):
    # the measured choice among the decomposition trees changes the work,
    # never the counts (Section 5.2: every tree gives the same count)
    import paper_1602_04478_gb300 as P
    g = graph("cl3000")
    k, e = QUERIES[qname]
    gid = cc.load_graph(g)
    try:
        P.cc_set_coloring_seed(cc.h, 9)
        qid = cc.set_query(k, e)
        before = [int(x) for x in cc.count(gid, qid, 0, 2)[0]]
        n_sup = sum(t["supported"] for t in P.cc_plan_enumerate(k, e))
        chosen = P.cc_autotune_plan(cc.h, gid, qid)
        assert 0 <= chosen < n_sup
        assert [int(x) for x in cc.count(gid, qid, 0, 2)[0]] == before
        assert before[0] == O.dp_count(g, k, e, O.colors(9, 0, g.n, k))[0]
    finally:
        cc.free_graph(gid)
