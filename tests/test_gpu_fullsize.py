"""Parity at the benchmark's full size (Chung-Lu n = 1e6, mean degree 16,
exponent 2.1) in the configuration bench.py times.

* C6: the count split by highest cycle vertex; sampled sources are checked
  one by one against the oracle restricted to those sources, live for
  sources of low and medium degree and from stored oracle values
  (tests/golden/cl1e6.txt, written by tests/golden/make_golden.py) for hub
  sources of degree 256 to 4,202, which take the grouped heavy path.
* C5 (the batched configuration's cycle query): sampled sources, as for C6.
* glasses and the 4-cycle with a chord and a pendant: the oracle cannot
  build their tables over the whole graph in test time, so properties that
  hold at any size are checked: the count is the same for different
  decomposition orders and for a relabelled graph.
"""
import numpy as np
import pytest

import golden_io
import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_04478_gb300 as P
    g = gg.chung_lu(1_000_000, 16, 2.1, 2)
    ctx = P.Context(0)
    gid = ctx.load_graph(g)
    yield P, ctx, g, gid
    ctx.close()


def test_c6_sampled_sources_match_oracle(big):
    P, ctx, g, gid = big
    k, e = gg.query("C6")
    P.cc_set_coloring_seed(ctx.h, 1)
    P.cc_set_heavy_degree(ctx.h, 256)
    qid = ctx.set_query(k, e)
    pv, total = ctx.count_per_vertex(gid, qid, 0)
    assert int(pv.sum()) == total
    assert total == int(ctx.count(gid, qid, 0, 1)[0][0])
    deg = np.diff(g.row_ptr)
    rng = np.random.default_rng(0)
    # sources on both sides of the heavy/light split, of a size the oracle handles
    light = rng.choice(np.flatnonzero((deg >= 8) & (deg <= 64)), size=12, replace=False)
    medium = rng.choice(np.flatnonzero((deg >= 256) & (deg <= 300)), size=2, replace=False)
    pick = np.concatenate([light, medium])
    filt = np.zeros(g.n, dtype=np.uint8)
    filt[pick] = 1
    _, _, per = O.dp_count(g, k, e, O.colors(1, 0, g.n, k), root_filter=filt, per_source=True)
    for v in pick:
        assert int(pv[v]) == per[v], int(v)
    # hub sources (grouped heavy path): stored oracle values
    gold = golden_io.load("cl1e6")
    assert golden_io.fingerprint(g) == gold.graph_sha["cl1e6"]
    hubs = gold.sources[("cl1e6", "C6", 1, 0)]
    assert len(hubs) >= 24 and max(deg[v] for v in hubs) == deg.max()
    for v, want in hubs.items():
        assert int(pv[v]) == want, (int(v), int(deg[v]))
    # the same sources at the library's own threshold
    P.cc_set_heavy_degree(ctx.h, -1)
    pv2, total2 = ctx.count_per_vertex(gid, qid, 0)
    assert total2 == total
    for v, want in hubs.items():
        assert int(pv2[v]) == want, (int(v), int(deg[v]))


def test_c5_sampled_sources_match_oracle(big):
    P, ctx, g, gid = big
    k, e = gg.query("C5")
    P.cc_set_coloring_seed(ctx.h, 3)
    qid = ctx.set_query(k, e)
    pv, total = ctx.count_per_vertex(gid, qid, 0)
    assert int(pv.sum()) == total
    deg = np.diff(g.row_ptr)
    rng = np.random.default_rng(1)
    pick = np.concatenate([rng.choice(np.flatnonzero((deg >= 8) & (deg <= 64)), size=12, replace=False),
                           rng.choice(np.flatnonzero((deg >= 200) & (deg <= 260)), size=2, replace=False)])
    filt = np.zeros(g.n, dtype=np.uint8)
    filt[pick] = 1
    _, _, per = O.dp_count(g, k, e, O.colors(3, 0, g.n, k), root_filter=filt, per_source=True)
    for v in pick:
        assert int(pv[v]) == per[v], int(v)
    gold = golden_io.load("cl1e6")
    for v, want in gold.sources[("cl1e6", "C5", 3, 0)].items():
        assert int(pv[v]) == want, (int(v), int(deg[v]))


def test_chord_pendant_decomposition_invariant_at_full_size(big):
    P, ctx, g, gid = big
    k, e = gg.query("chord_pendant")
    P.cc_set_coloring_seed(ctx.h, 2)
    orders = [[0, 1, 4, 3, 0, 1, 2], [3, 0, 2, 3, 0, 1, 4], [0, 1, 4, 3, 0, 2, 3]]
    got = []
    for seq in orders:
        qid = ctx.set_query(k, e)
        P.cc_set_decomposition(ctx.h, qid, seq)
        got.append([int(x) for x in ctx.count(gid, qid, 0, 2)[0]])
    assert got[0] == got[1] == got[2] and got[0][0] > 0


def test_glasses_decomposition_invariant_at_full_size(big):
    P, ctx, g, gid = big
    k, e = gg.query("glasses")
    P.cc_set_coloring_seed(ctx.h, 1)
    q1 = ctx.set_query(k, e)
    q2 = ctx.set_query(k, e)
    # other order: both triangles first, then the two leaf edges towards node 2
    P.cc_set_decomposition(ctx.h, q2, [3, 4, 5, 6, 3, 0, 1, 2, 0, 3, 4, 0, 2, 3])
    a = [int(x) for x in ctx.count(gid, q1, 0, 2)[0]]
    b = [int(x) for x in ctx.count(gid, q2, 0, 2)[0]]
    assert a == b and a[0] > 0


def test_c5_relabel_invariant_at_full_size(big):
    P, ctx, g, gid = big
    k, e = gg.query("C5")
    perm = np.random.default_rng(3).permutation(g.n)
    h = gg.relabel(g, perm)
    cols = O.colors(4, 0, g.n, k)
    colh = np.zeros_like(cols)
    colh[perm] = cols
    hid = ctx.load_graph(h)
    try:
        P.cc_set_colors(ctx.h, gid, cols)
        P.cc_set_colors(ctx.h, hid, colh)
        qid = ctx.set_query(k, e)
        assert int(ctx.count(gid, qid)[0][0]) == int(ctx.count(hid, qid)[0][0])
    finally:
        P.cc_clear_colors(ctx.h, gid)
        ctx.free_graph(hid)
