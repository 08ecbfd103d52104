"""Random treewidth-2 queries (series-parallel graphs built by subdividing
and duplicating edges, with pendant paths hung on them): every supported
decomposition tree of each, up to a few per query, must give the oracle's
count on a small random graph (Section 5.2: the count does not depend on the
tree).  The shapes mix every block kind the kernels take: leaves over data
edges and over pair graphs, triangles and longer cycles with one or two
boundary nodes, adjacent and non-adjacent boundary pairs, root cycles and
root nodes."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu


def random_sp_query(seed, k_max=8):
    """A connected simple series-parallel query on at most k_max nodes."""
    rng = np.random.default_rng(seed)
    edges = {(0, 1)}
    k = 2
    while k < k_max:
        op = rng.integers(3)
        a, b = sorted(list(edges))[int(rng.integers(len(edges)))]
        if op == 0:  # series: subdivide (a, b)
            edges.discard((a, b))
            edges |= {(min(a, k), max(a, k)), (min(b, k), max(b, k))}
            k += 1
        elif op == 1 and k + 1 <= k_max:  # parallel: a new path a - k - b beside (a, b)
            edges |= {(min(a, k), max(a, k)), (min(b, k), max(b, k))}
            k += 1
        else:  # pendant on a random node
            v = int(rng.integers(k))
            edges.add((v, k))
            k += 1
    return k, sorted(edges)


SEEDS = list(range(120))


@pytest.fixture(scope="module")
def cc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_04478_gb300 as P
    ctx = P.Context(0)
    yield ctx
    ctx.close()


@pytest.fixture(scope="module")
def graph_and_id(cc):
    g = gg.erdos_renyi(60, 330, 17)
    gid = cc.load_graph(g)
    yield g, gid
    cc.free_graph(gid)


@pytest.mark.parametrize("seed", SEEDS)
def test_random_query_every_tree(cc, graph_and_id, seed):
    import paper_1602_04478_gb300 as P
    g, gid = graph_and_id
    k, e = random_sp_query(seed, 8 + seed % 3)
    trees = [t for t in P.cc_plan_enumerate(k, e) if t["supported"]]
    assert trees, (k, e)
    rng = np.random.default_rng(seed)
    pick = trees if len(trees) <= 6 else [trees[i] for i in sorted(rng.choice(len(trees), 6, replace=False))]
    P.cc_set_coloring_seed(cc.h, 100 + seed)
    want = O.dp_count(g, k, e, O.colors(100 + seed, 0, g.n, k))[0]
    for t in pick:
        qid = cc.set_query(k, e)
        if t["seq"]:
            P.cc_set_decomposition(cc.h, qid, t["seq"])
        got = int(cc.count(gid, qid, 0, 1)[0][0])
        assert got == want, (k, e, t["seq"])


@pytest.fixture(scope="module")
def power_law(cc):
    g = gg.chung_lu(1500, 6, 2.1, 23)
    gid = cc.load_graph(g)
    yield g, gid
    cc.free_graph(gid)


@pytest.mark.parametrize("seed", list(range(200, 230)))
def test_random_query_power_law_heavy_paths(cc, power_law, seed):
    """The same on a heavy-tailed graph with the heavy-source threshold at
    degree 24, so root cycles also take the grouped heavy paths (plain and
    annotated) beside the per-CTA ones."""
    import paper_1602_04478_gb300 as P
    g, gid = power_law
    k, e = random_sp_query(seed, 8)
    trees = [t for t in P.cc_plan_enumerate(k, e) if t["supported"]]
    rng = np.random.default_rng(seed)
    pick = trees if len(trees) <= 3 else [trees[i] for i in sorted(rng.choice(len(trees), 3, replace=False))]
    want = O.dp_count(g, k, e, O.colors(seed, 0, g.n, k))[0]
    P.cc_set_coloring_seed(cc.h, seed)
    P.cc_set_heavy_degree(cc.h, 24)
    try:
        for t in pick:
            qid = cc.set_query(k, e)
            if t["seq"]:
                P.cc_set_decomposition(cc.h, qid, t["seq"])
            got = int(cc.count(gid, qid, 0, 1)[0][0])
            assert got == want, (k, e, t["seq"])
    finally:
        P.cc_set_heavy_degree(cc.h, -1)
