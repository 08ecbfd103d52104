"""The PS procedure on the GPU (the paper's path-splitting algorithm, figure
"PS Algorithm", Procedures 1-2): root cycles split once at a_0 and its
opposite node, paths extended through any vertex, no vertex order.  Counts
must equal the oracle's (which runs PS and DB on its own), and the split by
a_0's image must equal the oracle's PS split."""
import pytest

import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_04478_gb300 as P
    ctx = P.Context(0)
    yield ctx
    ctx.close()


CASES = [("er60", q) for q in ["C4", "C5", "C6", "C7", "C8", "C6_2pendants", "C6_2pendants_adj",
                               "C5_pendant_path", "chord_pendant", "glasses"]]
CASES += [("cl3000", q) for q in ["C4", "C5", "C6"]] + [("rmat10", q) for q in ["C4", "C5"]]
GRAPHS = {"er60": lambda: gg.erdos_renyi(60, 300, 1), "cl3000": lambda: gg.chung_lu(3000, 8, 2.1, 3),
          "rmat10": lambda: gg.rmat(10, 8, 0.57, 0.19, 0.19, 4)}


@pytest.mark.parametrize("gname,qname", CASES)
def test_ps_counts_match_oracle(cc, gname, qname):
    import paper_1602_04478_gb300 as P
    g = GRAPHS[gname]()
    k, e = gg.query(qname)
    gid = cc.load_graph(g)
    try:
        P.cc_set_coloring_seed(cc.h, 6)
        qid = cc.set_query(k, e)
        P.cc_set_procedure(cc.h, P.PROC_PS)
        pv, total = cc.count_per_vertex(gid, qid, 0)
        ps_count, _, ps_per = O.dp_count(g, k, e, O.colors(6, 0, g.n, k), order="ps", per_source=True)
        assert total == ps_count
        blocks, root, _ = O.decompose(k, e)
        if blocks[root]["kind"] == "root_cycle" and len(blocks[root]["nodes"]) >= 4:
            assert [int(x) for x in pv] == ps_per
        # DB gives the same count
        P.cc_set_procedure(cc.h, P.PROC_DB)
        assert int(cc.count(gid, qid, 0, 1)[0][0]) == total
    finally:
        P.cc_set_procedure(cc.h, P.PROC_DB)
        cc.free_graph(gid)


def test_procedure_argument_checked(cc):
    import paper_1602_04478_gb300 as P
    with pytest.raises(P.CCError):
        P.cc_set_procedure(cc.h, 2)
