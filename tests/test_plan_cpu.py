"""Host-side query planning of the CUDA library, checked on the CPU.

cc_plan_inspect runs the library's own decomposition (Section 4.1, Cases 1-3)
and aut(Q) without a device.  Checks: aut(Q) equals the oracle's enumeration,
every plan is a well-formed decomposition tree, an explicit order reproduces
the paper's worked Satellite tree, and treewidth-3 queries are rejected.
"""
import os

import pytest

import graphgen as gg
import oracle as O
import paper_1602_04478_gb300 as P

from test_oracle_pins import EXTRA, _read_satellite, _same_cycle

QUERIES = dict(gg.QUERIES)
QUERIES.update(EXTRA)


@pytest.mark.parametrize("name", sorted(QUERIES))
def test_aut_and_plan_shape(name):
    k, e = QUERIES[name]
    try:
        blocks, aut = P.cc_plan_inspect(k, e)
    except P.CCError as ex:
        assert P.ERRORS[ex.code] == "CC_ERR_UNSUPPORTED"
        return
    assert aut == O.automorphisms(k, e)
    covered = set()
    edges = {tuple(sorted(x)) for x in e}
    seen_children = set()
    for i, b in enumerate(blocks):
        for c in b["children"]:
            assert c < i and c not in seen_children  # each block has one parent, built before it
            seen_children.add(c)
        if b["kind"] in ("triangle", "root_cycle", "cycle"):
            L = len(b["nodes"])
            assert (L == 3) == (b["kind"] == "triangle")
        covered.update(b["nodes"])
    assert covered == set(range(k))
    assert blocks[-1]["kind"] in ("root_cycle", "root_node", "triangle")
    assert len(seen_children) == len(blocks) - 1  # a tree: every block but the root is a child
    # every original edge lies in some block as a leaf edge or a cycle edge
    block_edges = set()
    for b in blocks:
        nodes = b["nodes"]
        if b["kind"] == "leaf":
            block_edges.add(tuple(sorted(nodes)))
        elif b["kind"] != "root_node":
            for i in range(len(nodes)):
                block_edges.add(tuple(sorted((nodes[i], nodes[(i + 1) % len(nodes)]))))
    assert edges <= block_edges


def test_satellite_explicit_order_reproduces_paper_tree():
    edges, expect = _read_satellite()
    # B1 = 5-cycle a..e, B2 = leaf (f,h), B3 = 4-cycle (a,f,g,c), B4 = triangle (i,j,k)
    seq = [5, 0, 1, 2, 3, 4, 0, 5, 7, 4, 0, 5, 6, 2, 3, 8, 9, 10]
    # B1's boundary (a, c) is not an edge: its table is pair-keyed, read by
    # the 4-cycle B3 only, whose own boundary (f, g) is a data edge
    assert P.cc_plan_supported(11, edges, seq) == 1
    blocks, _ = P.cc_plan_inspect(11, edges, seq)
    names = {}
    for i, (blk, (name, kind, nodes, bd, kids)) in enumerate(zip(blocks, expect)):
        names[name] = i
        want_kind = {"cycle": ("cycle", "triangle"), "leaf": ("leaf",), "root_cycle": ("triangle", "root_cycle")}
        assert blk["kind"] in want_kind[kind]
        if kind == "leaf":
            assert blk["nodes"] == nodes
        else:
            assert _same_cycle(blk["nodes"], nodes)
        assert sorted(blk["boundary"]) == sorted(bd)
        assert sorted(blk["children"]) == sorted(names[c] for c in kids)
    assert len(blocks) == len(expect)


def _inspect_anyway(k, edges, seq):
    return P.cc_plan_inspect(k, edges, seq, allow_unsupported=True)


@pytest.mark.parametrize("edges", [
    [(a, b) for a in range(4) for b in range(a + 1, 4)],
    [(a, b) for a in range(5) for b in range(a + 1, 5) if (a, b) != (0, 1)],
])
def test_treewidth3_rejected(edges):
    k = 1 + max(max(x) for x in edges)
    with pytest.raises(P.CCError) as ei:
        P.cc_plan_inspect(k, edges)
    assert P.ERRORS[ei.value.code] == "CC_ERR_NOT_TW2"


def test_explicit_orders_of_chord_pendant():
    k, e = QUERIES["chord_pendant"]
    b1, _ = P.cc_plan_inspect(k, e, [0, 1, 4, 3, 0, 1, 2])
    assert [x["kind"] for x in b1] == ["leaf", "triangle", "triangle"]
    assert sorted(b1[1]["boundary"]) == [0, 2] and b1[1]["children"] == [0]
    b2, _ = P.cc_plan_inspect(k, e, [3, 0, 2, 3, 0, 1, 4])
    assert [x["kind"] for x in b2] == ["triangle", "leaf", "triangle"]
    assert sorted(b2[-1]["children"]) == [0, 1]
    with pytest.raises(P.CCError):
        P.cc_plan_inspect(k, e, [3, 0, 1, 3])  # (0,1,3) is not a cycle of the query


def test_default_plans_of_workload_queries_are_supported():
    for name in ["C4", "C5", "C6", "diamond", "chord_pendant", "glasses", "C6_2pendants"]:
        k, e = QUERIES[name]
        blocks, _ = P.cc_plan_inspect(k, e)
        assert all(b["kind"] != "cycle" for b in blocks)


def test_tree_enumeration_and_ranking():
    # every decomposition tree (Section 5.3) once; the paper's heuristic picks
    # the least by (longest cycle, boundary nodes, annotations), the library
    # the least by (longest cycle, join cost, boundary nodes, annotations)
    import paper_1602_04478_gb300 as P
    shapes = {
        "chord_pendant": gg.query("chord_pendant"),
        "diamond": gg.query("diamond"),
        "bowtie_pendants": (7, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 2), (0, 5), (4, 6)]),
        "C6_2pendants": gg.query("C6_2pendants"),
    }
    counts = {"chord_pendant": 4, "diamond": 2, "bowtie_pendants": 28, "C6_2pendants": 11}
    for name, (k, e) in shapes.items():
        trees = P.cc_plan_enumerate(k, e)
        assert len(trees) == counts[name], name
        assert len({tuple(t["seq"]) for t in trees}) == len(trees)
        sup = [t for t in trees if t["supported"]]
        paper = [t for t in sup if t["paper"]]
        lib = [t for t in sup if t["default"]]
        assert len(paper) == 1 and len(lib) == 1, name
        pk = lambda t: (t["longest"], t["boundary"], t["annotations"])
        lk = lambda t: (t["longest"], t["cost"], t["boundary"], t["annotations"])
        assert pk(paper[0]) == min(pk(t) for t in sup)
        assert lk(lib[0]) == min(lk(t) for t in sup)
        # the default plan is that tree
        blocks, _ = P.cc_plan_inspect(k, e)
        again, _ = P.cc_plan_inspect(k, e, lib[0]["seq"]) if lib[0]["seq"] else (blocks, 0)
        assert blocks == again, name


def test_shapes_cover_both_cut_orientations():
    """The Case-2 parity queries' trees include Case-2 blocks whose second boundary node lies
    within half the cycle of the first in the cycle's own order and beyond it
    (the kernel then walks the cycle the other way), adjacent pairs (a cut of
    one edge) and non-adjacent ones."""
    from test_gpu_case2 import QUERIES as CASE2, _case2_blocks
    seen = set()
    for k, e in CASE2.values():
        for t in P.cc_plan_enumerate(k, e):
            if t["supported"]:
                for L, d in _case2_blocks(P, k, e, t["seq"]):
                    seen.add(("adjacent" if d in (1, L - 1) else "apart", d > L // 2))
    assert seen >= {("adjacent", False), ("apart", False), ("apart", True)}


def test_support_of_pair_keyed_tables():
    """A Case-2 table keyed by pairs that are not data edges is produced and
    read by the cycle kernel (a triangle that reads one runs there too) and
    by the leaf join over its pair graph."""
    k, e = 6, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (0, 5), (5, 2)]
    seen = {}
    for t in P.cc_plan_enumerate(k, e):
        blocks, _ = P.cc_plan_inspect(k, e, t["seq"], allow_unsupported=True)
        seen[(len(blocks[0]["nodes"]), blocks[-1]["kind"])] = t["supported"]
    # the square (0,1,2,5) cut off leaves a root 4-cycle; either 5-cycle, a root triangle
    assert seen == {(4, "root_cycle"): True, (5, "triangle"): True}
    # K_{2,3}: every tree ends in a triangle over the pair (0, 1)
    k23 = [(0, 2), (2, 1), (0, 3), (3, 1), (0, 4), (4, 1)]
    assert all(t["supported"] for t in P.cc_plan_enumerate(5, k23))
    # a square with pendants on opposite nodes: cut off first, the square
    # leaves the pair (0, 2) as a leaf edge
    sq = [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (2, 5)]
    sup = {}
    for t in P.cc_plan_enumerate(6, sq):
        blocks, _ = P.cc_plan_inspect(6, sq, t["seq"], allow_unsupported=True)
        sup.setdefault(blocks[0]["kind"], set()).add(t["supported"])
    assert sup["cycle"] == {True} and sup["leaf"] == {True}
    # a 7-cycle whose boundary nodes are adjacent: the long side has 6 edges
    c7 = [(i, (i + 1) % 7) for i in range(7)] + [(0, 7), (7, 1)]
    sup = {tuple(len(b["nodes"]) for b in P.cc_plan_inspect(8, c7, t["seq"], allow_unsupported=True)[0]):
           t["supported"] for t in P.cc_plan_enumerate(8, c7)}
    assert sup[(7, 3)] is False and sup[(3, 7)] is True
