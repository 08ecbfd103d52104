"""The bounds-check build (libcc_boundscheck.so, CC_BOUNDS_CHECK set) on small
parity cases: every index the benchmark-path kernels read from data -- CSR
entries, level lists and local indices of the plain-cycle closure, triangle
records and edge positions, leaf-join neighbours and slots, and in the
general cycle kernel the neighbours, table positions and pair-table rows of
every walk (data graph or pair graph) -- is checked against its array; a
violation sets a status flag (the access is skipped) and the count returns
CC_ERR_BOUNDS.  The build stands in for a memory checker such as
compute-sanitizer, which these tests do not run.  Every case must come back
CC_OK with the oracle's count."""
import ctypes

import numpy as np
import pytest

import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_04478_gb300 as P
    return P.variant_library("libcc_boundscheck.so")


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


CASES = [("cl3000", q, hd) for q in ["C4", "C5", "C6"] for hd in (0, 64, 1 << 10)]
CASES += [("cl3000", q, -1) for q in ["glasses", "chord_pendant", "path4", "star4", "bowtie"]]
CASES += [("wheel", q, -1) for q in ["triangle", "diamond", "chord_pendant"]]
# the general cycle kernel: annotated root cycles, non-root blocks of both
# cases, pair lists and the walks over their pair graphs
CASES += [("cl1000", q, -1) for q in ["C6_2pendants", "C5_pendant_path", "double_square", "theta_5_2",
                                       "theta_2233", "K24", "square_opposite_pendants"]]
GRAPHS = {"cl3000": lambda: gg.chung_lu(3000, 8, 2.1, 3), "wheel": gg.wheel_with_chords,
          "cl1000": lambda: gg.chung_lu(1000, 6, 2.1, 3)}
SHAPES = dict(gg.QUERIES)
SHAPES.update({"path4": (4, [(0, 1), (1, 2), (2, 3)]), "star4": (5, [(0, 1), (0, 2), (0, 3), (0, 4)]),
               "bowtie": (5, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 2)]),
               "double_square": (7, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (4, 5), (5, 6), (6, 0)]),
               "theta_5_2": (6, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (0, 5), (5, 2)]),
               "theta_2233": (8, [(0, 1), (1, 2), (0, 5), (5, 2), (0, 4), (4, 3), (3, 2), (0, 6), (6, 7), (7, 2)]),
               "K24": (6, [(0, 1), (1, 2), (0, 3), (3, 2), (0, 4), (4, 2), (0, 5), (5, 2)]),
               "square_opposite_pendants": (6, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (2, 5)])})


@pytest.mark.parametrize("gname,qname,heavy", CASES)
def test_no_index_leaves_its_array(V, gname, qname, heavy):
    g = GRAPHS[gname]()
    k, e = SHAPES[qname]
    h = ctypes.c_void_p()
    assert V.cc_create(ctypes.byref(h), 0, None) == 0
    try:
        gid, qid = ctypes.c_int32(), ctypes.c_int32()
        rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
        cl = np.ascontiguousarray(g.col, dtype=np.int32)
        assert V.cc_load_csr(h, g.n, _p(rp, ctypes.c_int64), _p(cl, ctypes.c_int32), g.nnz, ctypes.byref(gid)) == 0
        ea = np.ascontiguousarray(np.asarray(e, dtype=np.int32).reshape(-1))
        assert V.cc_set_query(h, k, len(e), _p(ea, ctypes.c_int32), ctypes.byref(qid)) == 0
        assert V.cc_set_coloring_seed(h, 4) == 0
        assert V.cc_set_heavy_degree(h, heavy) == 0
        out = np.zeros(2, dtype=np.uint64)
        rc = V.cc_count(h, gid, qid, 0, 2, _p(out, ctypes.c_uint64), None, None)
        assert rc == 0, rc
        for t in range(2):
            assert int(out[t]) == O.dp_count(g, k, e, O.colors(4, t, g.n, k))[0], (qname, t)
    finally:
        V.cc_destroy(h)


@pytest.mark.parametrize("qname", ["theta_5_2", "K24", "square_opposite_pendants"])
def test_every_tree_of_case2_queries(V, qname):
    """Every supported tree (so every Case-2 placement: pair lists, pair
    graphs walked by cycles, triangles and leaves) through the bounds-check
    build, against the oracle."""
    import paper_1602_04478_gb300 as P
    g = GRAPHS["cl1000"]()
    k, e = SHAPES[qname]
    want = [O.dp_count(g, k, e, O.colors(4, t, g.n, k))[0] for t in range(2)]
    h = ctypes.c_void_p()
    assert V.cc_create(ctypes.byref(h), 0, None) == 0
    try:
        gid = ctypes.c_int32()
        rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
        cl = np.ascontiguousarray(g.col, dtype=np.int32)
        assert V.cc_load_csr(h, g.n, _p(rp, ctypes.c_int64), _p(cl, ctypes.c_int32), g.nnz, ctypes.byref(gid)) == 0
        assert V.cc_set_coloring_seed(h, 4) == 0
        ea = np.ascontiguousarray(np.asarray(e, dtype=np.int32).reshape(-1))
        trees = [t for t in P.cc_plan_enumerate(k, e) if t["supported"]]
        assert trees
        for t in trees:
            qid = ctypes.c_int32()
            assert V.cc_set_query(h, k, len(e), _p(ea, ctypes.c_int32), ctypes.byref(qid)) == 0
            if t["seq"]:
                sq = np.ascontiguousarray(np.asarray(t["seq"], dtype=np.int32))
                assert V.cc_set_decomposition(h, qid, _p(sq, ctypes.c_int32), len(sq)) == 0
            out = np.zeros(2, dtype=np.uint64)
            rc = V.cc_count(h, gid, qid, 0, 2, _p(out, ctypes.c_uint64), None, None)
            assert rc == 0, (rc, t["seq"])
            assert [int(x) for x in out] == want, t["seq"]
    finally:
        V.cc_destroy(h)
