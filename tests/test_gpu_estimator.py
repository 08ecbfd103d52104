"""The colour-coding estimator on the GPU (Section 2, "Approximate subgraph
counting via color coding"): the mean over many colourings of
n_colorful * k^k / k! / aut(Q) converges to the number of subgraphs, which
brute force gives on a small graph (oracle.brute_matches / aut).  The
colourings run in the batched form; the precision study of bench.py
(--precision) uses the same statistics."""
import math

import numpy as np
import pytest

import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("qname", ["C5", "chord_pendant", "glasses"])
def test_mean_estimate_converges_to_brute_force(qname):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    import paper_1602_04478_gb300 as P
    g = gg.erdos_renyi(40, 160, 21)
    k, e = gg.query(qname)
    truth = O.brute_matches(g, k, e) / O.automorphisms(k, e)
    assert truth > 0
    ctx = P.Context(0)
    try:
        gid = ctx.load_graph(g)
        qid = ctx.set_query(k, e)
        P.cc_set_coloring_seed(ctx.h, 99)
        P.cc_set_graph_capture(ctx.h, False)
        T = 2000
        res, st = P.cc_count_batch(ctx.h, [(gid, qid, 0, T)])
        assert st == [0]
        scale = k ** k / math.factorial(k) / O.automorphisms(k, e)
        est = np.array([float(c) for c in res[0]]) * scale
        se = est.std(ddof=1) / math.sqrt(T)
        assert abs(est.mean() - truth) <= 4 * se, (est.mean(), truth, se)
        # the precision statistics: the coefficient of variation of the mean
        # shrinks like 1 / sqrt(colourings)
        cv3, cvm3 = bench.precision_stats(est, 3)
        cvT, cvmT = bench.precision_stats(est, T)
        assert cvmT < 0.1 and cvmT == pytest.approx(cvT / math.sqrt(T))
    finally:
        ctx.close()
