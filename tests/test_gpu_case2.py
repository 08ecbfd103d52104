"""Non-root cycle blocks with two boundary nodes (Case 2 of Section 4.1) of
length >= 4.  The cycle kernel builds their table cnt(u, x, alpha | B) cut at
the two boundary nodes (P+ and P- both run from the image u of the first to
the image x of the second).  A boundary pair joined by a data edge fills the
edge-keyed table; any other pair (not adjacent in the cycle, or adjacent over
an edge that is itself such a pair) goes to a pair list and then to a pair
graph that a parent cycle walks like the data graph.  Every supported
decomposition tree of each query must give the oracle's count (Section 5.2:
the count does not depend on the tree)."""
import pytest

import graphgen as gg
import oracle as O
from test_oracle_pins import _read_satellite

pytestmark = pytest.mark.gpu

QUERIES = {
    # a square and a triangle on one edge
    "house": (5, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (4, 1)]),
    # a 5-cycle and a path of two edges between its nodes 0 and 2
    "theta_5_2": (6, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (0, 5), (5, 2)]),
    # paths of 3, 3 and 2 edges between nodes 0 and 1
    "theta_332": (7, [(0, 2), (2, 3), (3, 1), (0, 4), (4, 5), (5, 1), (0, 6), (6, 1)]),
    # a 5-cycle and a square on one edge
    "pentagon_house": (7, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (0, 5), (5, 6), (6, 1)]),
    # paths of 3, 3 and 3 edges between nodes 0 and 1
    "theta_333": (8, [(0, 2), (2, 3), (3, 1), (0, 4), (4, 5), (5, 1), (0, 6), (6, 7), (7, 1)]),
    # paths of 2, 2, 3 and 3 edges between nodes 0 and 2: a square whose
    # boundary edge is itself a pair-keyed edge
    "theta_2233": (8, [(0, 1), (1, 2), (0, 5), (5, 2), (0, 4), (4, 3), (3, 2), (0, 6), (6, 7), (7, 2)]),
    # K_{2,3}: every tree ends in a root triangle over a pair-keyed edge
    "K23": (5, [(0, 2), (2, 1), (1, 3), (3, 0), (0, 4), (4, 1)]),
    # K_{2,3} and a triangle on node 1: a triangle with one boundary node reads a pair
    "K23_tail": (7, [(0, 2), (2, 1), (1, 3), (3, 0), (0, 4), (4, 1), (1, 5), (5, 6), (6, 1)]),
    # K_{2,4}: a triangle with both boundary nodes on a pair-keyed edge writes a pair list
    "K24": (6, [(0, 1), (1, 2), (0, 3), (3, 2), (0, 4), (4, 2), (0, 5), (5, 2)]),
    # a square with pendants on opposite nodes: cut off first, the square
    # leaves its pair as a leaf edge (the leaf join walks the pair graph)
    "square_opposite_pendants": (6, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (2, 5)]),
}
GRAPHS = {"er60": lambda: gg.erdos_renyi(60, 300, 1), "cl1000": lambda: gg.chung_lu(1000, 6, 2.1, 3)}


def _case2_blocks(P, k, e, seq):
    """(L, distance from the first boundary node to the second) per Case-2
    block of length >= 4."""
    blocks, _ = P.cc_plan_inspect(k, e, seq or None)
    out = []
    for b in blocks:
        if b["kind"] == "cycle" and len(b["boundary"]) == 2:
            n, L = b["nodes"], len(b["nodes"])
            out.append((L, (n.index(b["boundary"][1]) - n.index(b["boundary"][0])) % L))
    return out


@pytest.fixture(scope="module")
def cc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_04478_gb300 as P
    ctx = P.Context(0)
    yield ctx
    ctx.close()


def _every_tree(cc, g, k, e, trials=2, seed=10):
    import paper_1602_04478_gb300 as P
    gid = cc.load_graph(g)
    shapes = []
    try:
        P.cc_set_coloring_seed(cc.h, seed)
        want = [O.dp_count(g, k, e, O.colors(seed, t, g.n, k))[0] for t in range(trials)]
        trees = [t for t in P.cc_plan_enumerate(k, e) if t["supported"]]
        assert trees
        for t in trees:
            shapes += _case2_blocks(P, k, e, t["seq"])
            qid = cc.set_query(k, e)
            if t["seq"]:
                P.cc_set_decomposition(cc.h, qid, t["seq"])
            got = [int(x) for x in cc.count(gid, qid, 0, trials)[0]]
            assert got == want, t["seq"]
    finally:
        cc.free_graph(gid)
    return shapes, want


@pytest.mark.parametrize("gname", sorted(GRAPHS))
@pytest.mark.parametrize("qname", sorted(QUERIES))
def test_every_tree_matches_oracle(cc, gname, qname):
    k, e = QUERIES[qname]
    shapes, want = _every_tree(cc, GRAPHS[gname](), k, e)
    assert shapes  # at least one tree takes a Case-2 cycle
    assert any(w > 0 for w in want)


def test_satellite_paper_tree(cc):
    """The paper's worked decomposition of its Satellite query (Section 4.1):
    B1 = 5-cycle with boundary (a, c), B2 = leaf (f, h), B3 = 4-cycle
    (a, f, g, c) reading B1 over the pair (a, c), B4 = triangle (i, j, k),
    root = triangle (i, f, g)."""
    import paper_1602_04478_gb300 as P
    edges, _ = _read_satellite()
    seq = [5, 0, 1, 2, 3, 4, 0, 5, 7, 4, 0, 5, 6, 2, 3, 8, 9, 10]
    g = gg.erdos_renyi(60, 420, 5)
    gid = cc.load_graph(g)
    try:
        P.cc_set_coloring_seed(cc.h, 3)
        want = [O.dp_count(g, 11, edges, O.colors(3, t, g.n, 11))[0] for t in range(3)]
        qid = cc.set_query(11, edges)
        P.cc_set_decomposition(cc.h, qid, seq)
        got = [int(x) for x in cc.count(gid, qid, 0, 3)[0]]
        assert got == want
        assert any(w > 0 for w in want)
        # the library's own tree gives the same counts
        qid2 = cc.set_query(11, edges)
        assert [int(x) for x in cc.count(gid, qid2, 0, 3)[0]] == want
    finally:
        cc.free_graph(gid)


def test_pair_list_plan_in_a_batch(cc):
    """A plan with a pair list sizes it on the host, so a batch runs it
    without graph capture; the counts are the oracle's."""
    import paper_1602_04478_gb300 as P
    k, e = QUERIES["theta_5_2"]
    g = gg.chung_lu(3000, 8, 2.1, 3)
    gid = cc.load_graph(g)
    try:
        P.cc_set_coloring_seed(cc.h, 21)
        want = [O.dp_count(g, k, e, O.colors(21, t, g.n, k))[0] for t in range(3)]
        qid = cc.set_query(k, e)
        for _ in range(2):
            got, st = P.cc_count_batch(cc.h, [(gid, qid, 0, 3)])
            assert [int(x) for x in got[0]] == want and st == [0]
    finally:
        cc.free_graph(gid)


def test_pair_list_outgrows_the_previous_pass(cc):
    """The pair list of a pass is sized from the previous pass on the same
    graph; a colouring with far more pairs than the last one (here after a
    single-colour colouring with none) runs its append again into buffers of
    the exact size and still gives the oracle's count."""
    import numpy as np
    import paper_1602_04478_gb300 as P
    k, e = QUERIES["theta_5_2"]
    g = gg.chung_lu(3000, 8, 2.1, 3)
    gid = cc.load_graph(g)
    try:
        cols = np.stack([np.zeros(g.n, dtype=np.uint8), O.colors(8, 0, g.n, k), O.colors(8, 1, g.n, k)])
        P.cc_set_colors(cc.h, gid, cols)
        want = [0] + [O.dp_count(g, k, e, cols[t])[0] for t in (1, 2)]
        qid = cc.set_query(k, e)
        got = [int(x) for x in cc.count(gid, qid, 0, 3)[0]]
        assert got == want and want[1] > 0
    finally:
        P.cc_clear_colors(cc.h, gid)
        cc.free_graph(gid)


@pytest.mark.parametrize("qname", ["theta_5_2", "theta_333", "theta_2233"])
def test_per_vertex_split_of_a_root_reading_pairs(cc, qname):
    """A root cycle that walks a pair graph (DB procedure): its count split by
    the highest vertex equals the oracle's split for a tree with the same
    root block."""
    import paper_1602_04478_gb300 as P
    k, e = QUERIES[qname]
    g = GRAPHS["cl1000"]()
    lib_root = P.cc_plan_inspect(k, e)[0][-1]
    choice = None
    for p in O.all_plans(k, e, limit=200):
        blocks, root, _ = O.decompose(k, e, choice=p)
        if blocks[root]["kind"] == "root_cycle" and sorted(blocks[root]["nodes"]) == sorted(lib_root["nodes"]):
            choice = p
            break
    assert choice is not None
    expect, _, per = O.dp_count(g, k, e, O.colors(6, 0, g.n, k), choice=choice, per_source=True)
    gid = cc.load_graph(g)
    try:
        P.cc_set_coloring_seed(cc.h, 6)
        qid = cc.set_query(k, e)
        pv, total = cc.count_per_vertex(gid, qid, 0)
        assert total == expect and [int(x) for x in pv] == per
    finally:
        cc.free_graph(gid)


def test_per_vertex_refused_for_a_root_triangle_reading_pairs(cc):
    """K_{2,3}'s root triangle reads a pair-keyed edge and runs without vertex
    order, so its count has no split by the highest vertex."""
    import paper_1602_04478_gb300 as P
    k, e = QUERIES["K23"]
    g = GRAPHS["er60"]()
    gid = cc.load_graph(g)
    try:
        qid = cc.set_query(k, e)
        with pytest.raises(P.CCError) as ei:
            cc.count_per_vertex(gid, qid, 0)
        assert P.ERRORS[ei.value.code] == "CC_ERR_UNSUPPORTED"
    finally:
        cc.free_graph(gid)
