"""Pins for the CPU oracle: each check ties it to something other than itself.

- closed forms in complete graphs (any connected query; cycles),
- an independent triangle listing and the star's neighbour-histogram formula,
- the exact exhaustive-colouring identity behind the k^k/k! estimator
  (Section 2 of arXiv 1602.04478),
- the paper's worked "Satellite" decomposition (Section 4.1),
- rejection of treewidth-3 queries (Lemma 4.1 gives a block for every
  treewidth-2 query, so a query without one is not treewidth 2),
- the DP against brute-force enumeration on random graphs, for every
  decomposition tree and several vertex orders (Eq. 1 makes the count
  independent of the order; Section 5.2 makes it independent of the tree).
"""
import itertools
import math
import os

import numpy as np
import pytest

import graphgen as gg
import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# extra treewidth-2 shapes that stress the decomposition (asymmetric
# 2-boundary blocks, non-adjacent boundary pairs, several cycles)
EXTRA = {
    "path4": (4, [(0, 1), (1, 2), (2, 3)]),
    "star4": (5, [(0, 1), (0, 2), (0, 3), (0, 4)]),
    "tailed_triangle": (4, [(0, 1), (1, 2), (2, 0), (2, 3)]),
    "bowtie": (5, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 2)]),
    "house": (5, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (4, 1)]),
    # chord 0-2 with the pendant on a boundary node: an asymmetric 2-boundary block
    "chord_pendant0": (5, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2), (0, 4)]),
    # K_{2,3}: a 4-cycle block whose two boundary nodes are not adjacent
    "K23": (5, [(0, 2), (2, 1), (1, 3), (3, 0), (0, 4), (4, 1)]),
    "C6_2pendants_adj": (8, [(i, (i + 1) % 6) for i in range(6)] + [(0, 6), (1, 7)]),
    "C6_2pendants_same": (8, [(i, (i + 1) % 6) for i in range(6)] + [(0, 6), (0, 7)]),
    # theta graphs: paths between two nodes, so that every tree has a Case-2
    # block of length >= 4 whose boundary nodes are not adjacent
    "theta_5_2": (6, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (0, 5), (5, 2)]),
    "theta_332": (7, [(0, 2), (2, 3), (3, 1), (0, 4), (4, 5), (5, 1), (0, 6), (6, 1)]),
    "theta_2233": (8, [(0, 1), (1, 2), (0, 5), (5, 2), (0, 4), (4, 3), (3, 2), (0, 6), (6, 7), (7, 2)]),
}


def all_queries():
    q = {name: gg.query(name) for name in gg.QUERIES}
    q.update(EXTRA)
    return q


# ------------------------------- colouring -------------------------------
def test_splitmix64_published_vector():
    # SplitMix64 reference outputs for the state sequence 1234567 + i * golden
    expect = [6457827717110365317, 3203168211198807973, 9817491932198370423,
              4593380528125082431, 16408922859458223821]
    g = 0x9E3779B97F4A7C15
    assert [O.splitmix64((1234567 + i * g) % 2**64) for i in range(5)] == expect


def test_colour_range_and_balance():
    for k in (3, 5, 8, 12):
        c = O.colors(1, 0, 120000, k)
        assert c.min() == 0 and c.max() == k - 1
        frac = np.bincount(c, minlength=k) / c.size
        assert np.all(np.abs(frac - 1.0 / k) < 0.01)
    # trials are different colourings, seeds are different colourings
    assert not np.array_equal(O.colors(1, 0, 1000, 5), O.colors(1, 1, 1000, 5))
    assert not np.array_equal(O.colors(1, 0, 1000, 5), O.colors(2, 0, 1000, 5))


# ------------------------------ closed forms ------------------------------
@pytest.mark.parametrize("name", ["triangle", "C4", "C5", "diamond", "chord_pendant", "star4", "house"])
def test_brute_colorful_complete_graph(name):
    k, e = all_queries()[name]
    g = gg.complete_graph(9)
    col = O.colors(5, 2, g.n, k)
    nc = np.bincount(col, minlength=k)
    expect = math.factorial(k) * int(np.prod(nc.astype(object)))
    assert O.brute_colorful(g, k, e, col) == expect
    assert O.dp_count(g, k, e, col)[0] == expect


@pytest.mark.parametrize("L", [3, 4, 5, 6])
def test_cycles_in_complete_graph_subgraph_count(L):
    # colourful L-cycles as subgraphs: (L-1)!/2 * prod(n_c); matches = 2L times that
    k, e = gg.cycle(L)
    g = gg.complete_graph(10)
    col = O.colors(11, 0, g.n, k)
    nc = np.bincount(col, minlength=k).astype(object)
    subgraphs = math.factorial(L - 1) // 2 * int(np.prod(nc))
    aut = O.automorphisms(k, e)
    assert aut == 2 * L
    assert O.dp_count(g, k, e, col)[0] == subgraphs * aut


def test_brute_matches_closed_forms():
    g = gg.complete_graph(7)
    for name in ["triangle", "C4", "diamond", "star4", "path4"]:
        k, e = all_queries()[name]
        assert O.brute_matches(g, k, e) == math.perm(7, k)
    for L in (4, 5, 6, 7):
        k, e = gg.cycle(L)
        cg = gg.from_edges(L, e)
        assert O.brute_matches(cg, k, e) == 2 * L


def test_automorphisms_textbook():
    q = all_queries()
    assert O.automorphisms(4, [(a, b) for a in range(4) for b in range(a + 1, 4)]) == 24
    assert O.automorphisms(*q["star4"]) == 24       # K_{1,4}: 4!
    assert O.automorphisms(*q["path4"]) == 2
    assert O.automorphisms(*q["glasses"]) == 8      # swap inside each triangle, mirror
    assert O.automorphisms(*q["diamond"]) == 4
    assert O.automorphisms(*q["chord_pendant"]) == 2
    assert O.automorphisms(*q["C6_2pendants"]) == 4
    assert O.automorphisms(*q["bowtie"]) == 8


def _independent_triangles(g):
    adj = [set(g.col[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(g.n)]
    out = []
    for a in range(g.n):
        for b in adj[a]:
            if b <= a:
                continue
            for c in adj[a] & adj[b]:
                if c > b:
                    out.append((a, b, c))
    return out


def test_triangle_closed_form():
    g = gg.chung_lu(300, 8, 2.3, 4)
    k, e = gg.cycle(3)
    for trial in range(3):
        col = O.colors(3, trial, g.n, k)
        tri = _independent_triangles(g)
        colourful = sum(1 for (a, b, c) in tri if len({col[a], col[b], col[c]}) == 3)
        assert O.brute_colorful(g, k, e, col) == 6 * colourful
        assert O.dp_count(g, k, e, col)[0] == 6 * colourful


def test_star_closed_form():
    g = gg.erdos_renyi(60, 400, 9)
    k, e = EXTRA["star4"]
    col = O.colors(8, 0, g.n, k)
    total = 0
    for v in range(g.n):
        nb = g.col[g.row_ptr[v]:g.row_ptr[v + 1]]
        h = np.bincount(col[nb], minlength=k).astype(object)
        total += math.factorial(k - 1) * math.prod(int(h[c]) for c in range(k) if c != col[v])
    assert O.brute_colorful(g, k, e, col) == total
    assert O.dp_count(g, k, e, col)[0] == total


@pytest.mark.parametrize("name,n,k", [("triangle", 7, 3), ("C4", 7, 4), ("path4", 7, 4),
                                      ("tailed_triangle", 6, 4)])
def test_exhaustive_colouring_identity(name, n, k):
    # every match is colourful under exactly k! * k^(n-k) of the k^n colourings
    kq, e = all_queries()[name]
    assert kq == k
    g = gg.erdos_renyi(n, 13, 21)
    total = 0
    for col in itertools.product(range(k), repeat=n):
        total += O.brute_colorful(g, k, e, np.array(col, dtype=np.uint8))
    assert total == O.brute_matches(g, k, e) * math.factorial(k) * k ** (n - k)


def test_estimator_converges():
    g = gg.erdos_renyi(40, 160, 3)
    k, e = gg.query("C5")
    n_true = O.brute_matches(g, k, e)
    scale = k ** k / math.factorial(k)
    est = np.array([O.dp_count(g, k, e, O.colors(77, t, g.n, k))[0] * scale for t in range(3000)])
    assert abs(est.mean() - n_true) < 4 * est.std() / math.sqrt(est.size)


# ------------------------------ decomposition ------------------------------
def _read_satellite():
    blocks, edges = [], []
    for line in open(os.path.join(GOLDEN, "satellite_decomposition.txt")):
        line = line.split("#")[0].strip()
        if line.startswith("edges"):
            edges = [tuple(int(x) for x in p.split("-")) for p in line.split()[1:]]
        elif line.startswith("block"):
            parts = [p.strip() for p in line[len("block"):].split("|")]
            name, kind = parts[0], parts[1]
            nodes = [int(x) for x in parts[2].split()]
            bd = [int(x) for x in parts[3].split()] if parts[3] else []
            kids = parts[4].split() if len(parts) > 4 and parts[4] else []
            blocks.append((name, kind, nodes, bd, kids))
    return edges, blocks


def _same_cycle(a, b):
    if len(a) != len(b):
        return False
    L = len(a)
    for s in range(L):
        if all(a[i] == b[(s + i) % L] for i in range(L)) or all(a[i] == b[(s - i) % L] for i in range(L)):
            return True
    return False


def test_satellite_decomposition_matches_paper():
    edges, expect = _read_satellite()
    assert len(edges) == 14
    found = False
    for plan in O.all_plans(11, edges):
        blocks, root, _ = O.decompose(11, edges, plan)
        if len(blocks) != len(expect):
            continue
        names = {}
        ok = True
        for i, (blk, (name, kind, nodes, bd, kids)) in enumerate(zip(blocks, expect)):
            names[name] = i
            if blk["kind"] != kind:
                ok = False
                break
            same = _same_cycle(blk["nodes"], nodes) if "cycle" in kind else blk["nodes"] == nodes
            if not same or sorted(blk["boundary"]) != sorted(bd):
                ok = False
                break
            if sorted(blk["children"]) != sorted(names[c] for c in kids):
                ok = False
                break
        if ok:
            assert root == len(blocks) - 1
            found = True
            break
    assert found, "no decomposition reproduces the paper's Satellite tree"


def test_satellite_first_step_excludes_ifg():
    # (i,f,g) has three boundary nodes at the start: no plan contracts it first
    edges, _ = _read_satellite()
    for plan in O.all_plans(11, edges):
        blocks, _, _ = O.decompose(11, edges, plan)
        first = blocks[0]
        assert not (first["kind"] == "cycle" and sorted(first["nodes"]) == [5, 6, 8])


@pytest.mark.parametrize("edges", [
    [(a, b) for a in range(4) for b in range(a + 1, 4)],                      # K4
    [(a, b) for a in range(5) for b in range(a + 1, 5) if (a, b) != (0, 1)],  # K5 minus an edge
    [(a, b) for a in range(4) for b in range(a + 1, 4)] + [(3, 4)],           # K4 plus a tail
])
def test_treewidth3_rejected(edges):
    k = 1 + max(max(e) for e in edges)
    with pytest.raises(O.NotTreewidth2):
        O.decompose(k, edges)
    g = gg.complete_graph(6)
    with pytest.raises(O.NotTreewidth2):
        O.dp_count(g, k, edges, O.colors(1, 0, g.n, k))


# ------------------------- DP against brute force -------------------------
SMALL_GRAPHS = [
    lambda: gg.erdos_renyi(30, 90, 7),
    lambda: gg.erdos_renyi(40, 160, 8),
    lambda: gg.chung_lu(60, 6, 2.2, 9),
    lambda: gg.erdos_renyi(60, 300, 1),   # the brute-force check graph of the ER workload
]


@pytest.mark.parametrize("name", sorted(all_queries()))
@pytest.mark.parametrize("gi", range(len(SMALL_GRAPHS)))
def test_dp_equals_brute_force(name, gi):
    k, e = all_queries()[name]
    g = SMALL_GRAPHS[gi]()
    col = O.colors(1, gi, g.n, k)
    expect = O.brute_colorful(g, k, e, col)
    plans = O.all_plans(k, e, limit=40)
    for order in ("degree", "id", "ps"):
        got, ovf = O.dp_count(g, k, e, col, order=order)
        assert not ovf
        assert got == expect, (order, got, expect)
    rng = np.random.default_rng(gi)
    rank = rng.permutation(g.n).astype(np.int64)
    assert O.dp_count(g, k, e, col, order=rank)[0] == expect
    for p in plans:
        assert O.dp_count(g, k, e, col, choice=p)[0] == expect, p


def test_satellite_dp_equals_brute_force():
    edges, _ = _read_satellite()
    g = gg.erdos_renyi(30, 110, 1)
    # every colour class non-empty (two or three vertices each)
    col = np.random.default_rng(1).permutation(np.arange(g.n) % 11).astype(np.uint8)
    expect = O.brute_colorful(g, 11, edges, col)
    assert expect > 0
    for p in O.all_plans(11, edges, limit=12):
        assert O.dp_count(g, 11, edges, col, choice=p)[0] == expect


def test_relabel_invariance():
    g = gg.chung_lu(80, 6, 2.2, 3)
    perm = np.random.default_rng(0).permutation(g.n)
    h = gg.relabel(g, perm)
    for name in ["C5", "glasses", "chord_pendant"]:
        k, e = all_queries()[name]
        col = O.colors(9, 0, g.n, k)
        colh = np.zeros_like(col)
        colh[perm] = col
        assert O.dp_count(g, k, e, col)[0] == O.dp_count(h, k, e, colh)[0]


def test_per_source_partition():
    # Eq. 1: summing the root cycle's count over its highest vertex gives the total
    g = gg.chung_lu(120, 8, 2.2, 6)
    for name in ["C5", "C6_2pendants", "chord_pendant"]:
        k, e = all_queries()[name]
        col = O.colors(2, 0, g.n, k)
        total, _, per = O.dp_count(g, k, e, col, per_source=True)
        assert sum(per) == total == O.brute_colorful(g, k, e, col)
        # restricting the highest vertex to a subset gives that subset's share
        filt = (np.arange(g.n) % 3 == 0).astype(np.uint8)
        part = O.dp_count(g, k, e, col, root_filter=filt)[0]
        assert part == sum(p for v, p in enumerate(per) if filt[v])


def test_per_vertex_brute_force_for_cycle_sources():
    # per-source counts equal brute force restricted to matches whose highest
    # cycle vertex (degree order) is that source
    g = gg.erdos_renyi(30, 100, 12)
    k, e = gg.query("C5")
    col = O.colors(3, 0, g.n, k)
    _, _, per = O.dp_count(g, k, e, col, per_source=True)
    deg = np.diff(g.row_ptr)
    rank = np.lexsort((np.arange(g.n), deg)).argsort()
    for u in range(g.n):
        # C5 is vertex transitive: matches with a_0 = u and u highest, times 5
        sub = np.where(rank <= rank[u])[0]
        keep = np.zeros(g.n, bool)
        keep[sub] = True
        el = g.edge_list()
        el = el[keep[el[:, 0]] & keep[el[:, 1]]]
        h = gg.from_edges(g.n, el)
        cnt = O.brute_colorful(h, k, e, col, fixed_node=0, fixed_vertex=u)
        assert per[u] == 5 * cnt


def test_overflow_is_reported_not_wrapped():
    # star query with k = 12 on a star graph: (k-1)! * prod n_c(center) > 2^64
    k = 12
    e = [(0, i) for i in range(1, k)]
    D = 3000
    g = gg.from_edges(D + 1, [(0, i) for i in range(1, D + 1)])
    col = O.colors(1, 0, g.n, k)
    h = np.bincount(col[1:], minlength=k).astype(object)
    expect = math.factorial(k - 1) * math.prod(int(h[c]) for c in range(k) if c != col[0])
    assert expect > 2**64
    got, ovf = O.dp_count(g, k, e, col)
    assert ovf and got == expect


# ------------------------- structural work counter -------------------------
@pytest.mark.parametrize("L", [4, 5, 6])
def test_cycle_scans_complete_graph_closed_form(L):
    # In K_n every vertex has degree n-1, so the degree order is the id order.
    # A source u (u >= 2 lower neighbours) scans u edges out of level 0 per
    # half; level 1 is {0..u-1}, each of whose members has u-1 neighbours
    # below u; level 2 is again {0..u-1}.  Slots per level j: 1, then
    # C(k-2, j-1) (Section 5: high-starting paths, signatures holding chi(u)
    # and the end's colour).
    n = 30
    g = gg.complete_graph(n)
    k = L
    depths = [L // 2, L - L // 2]
    scans = [0] * 8
    units = 0
    for u in range(2, n):
        for d in depths:
            per_level = [u] + [u * (u - 1)] * (d - 1)
            for j, e in enumerate(per_level):
                scans[j] += e
                units += e * (1 if j == 0 else math.comb(k - 2, j - 1))
    tot, sc = O.cycle_units(g, L, k, scans=True)
    assert sc == [float(x) for x in scans]
    assert tot == units


def test_cycle_scans_star_graph():
    # a star: only the centre has lower neighbours; its leaves have none below it
    n = 50
    g = gg.from_edges(n, [(0, i) for i in range(1, n)])
    tot, sc = O.cycle_units(g, 6, 6, scans=True)
    assert sc == [2.0 * (n - 1)] + [0.0] * 7
    assert tot == 2.0 * (n - 1)
