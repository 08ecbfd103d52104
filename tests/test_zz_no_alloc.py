"""The count entry point that allocates no device memory.

Callers that cannot let a library allocate GPU memory (a fixed device arena,
no cudaMalloc allowed) use cc_count_cycle_noalloc: they pass device buffers
for the graph and the colours, and the library works in its own static
device array.  Its counts must equal cc_count's (the allocating path) and the
oracle's for the same graph, colours and query, call after call.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_04478_gb300 as P
    ctx = P.Context(0)
    yield torch, P, ctx
    ctx.close()


def _device_inputs(torch, g, colors):
    rp = torch.from_numpy(np.ascontiguousarray(g.row_ptr, dtype=np.int64)).cuda()
    col = torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).cuda()
    c = torch.from_numpy(np.ascontiguousarray(colors, dtype=np.uint8)).cuda()
    return rp, col, c


@pytest.mark.parametrize("gname,graph", [
    ("er2000", lambda: gg.erdos_renyi(2000, 10000, 1)),
    ("cl20000", lambda: gg.chung_lu(20000, 8, 2.1, 5)),
])
@pytest.mark.parametrize("L", [4, 5, 6])
def test_noalloc_matches_allocating_path(env, gname, graph, L):
    torch, P, ctx = env
    g = graph()
    k, e = gg.cycle(L)
    gid = ctx.load_graph(g)
    try:
        qid = ctx.set_query(k, e)
        stream = torch.cuda.current_stream().cuda_stream
        for trial in range(2):  # two calls in a row share (and reuse) the static scratch
            colors = O.colors(100 + trial, 0, g.n, k)
            P.cc_set_colors(ctx.h, gid, colors)
            expect = int(ctx.count(gid, qid, 0, 1)[0][0])
            rp, col, c = _device_inputs(torch, g, colors)
            got = P.cc_count_cycle_noalloc(0, stream, L, g.n, rp.data_ptr(), col.data_ptr(), c.data_ptr())
            torch.cuda.synchronize()
            assert got == expect, (gname, L, trial, got, expect)
            assert got == O.dp_count(g, k, e, colors)[0], (gname, L, trial)
    finally:
        ctx.free_graph(gid)


def test_noalloc_rejects_too_large_graphs(env):
    torch, P, _ = env
    n = 700_000  # n * 112 bytes is beyond the 64 MiB working array
    g = gg.erdos_renyi(n, n, 3)
    rp, col, c = _device_inputs(torch, g, np.zeros(n, dtype=np.uint8))
    with pytest.raises(P.CCError) as ei:
        P.cc_count_cycle_noalloc(0, None, 6, n, rp.data_ptr(), col.data_ptr(), c.data_ptr())
    assert P.ERRORS[ei.value.code] == "CC_ERR_INVALID_ARG"


def test_noalloc_rejects_bad_inputs(env):
    torch, P, _ = env
    g = gg.erdos_renyi(500, 2000, 2)
    colors = O.colors(1, 0, g.n, 5)
    colors[7] = 9  # outside 0..L-1
    rp, col, c = _device_inputs(torch, g, colors)
    with pytest.raises(P.CCError) as ei:
        P.cc_count_cycle_noalloc(0, None, 5, g.n, rp.data_ptr(), col.data_ptr(), c.data_ptr())
    assert P.ERRORS[ei.value.code] == "CC_ERR_BAD_GRAPH"
    with pytest.raises(P.CCError):
        P.cc_count_cycle_noalloc(0, None, 7, g.n, rp.data_ptr(), col.data_ptr(), c.data_ptr())


def _hub_and_clique(hub_degree):
    # vertex 0 adjacent to vertices 1..hub_degree; vertices 1..48 also form a
    # clique, so every cycle through the hub runs through the clique and the
    # hub's row is the longest the kernel reads
    e = [(0, i) for i in range(1, hub_degree + 1)]
    e += [(a, b) for a in range(1, 49) for b in range(a + 1, 49)]
    return gg.from_edges(hub_degree + 1, e)


@pytest.mark.parametrize("L", [5, 6])
def test_noalloc_at_the_degree_limit(env, L):
    # the largest accepted degree (65535) keeps the 32-bit level-3 sums exact:
    # the count equals the oracle's
    torch, P, _ = env
    g = _hub_and_clique(65535)
    k, e = gg.cycle(L)
    colors = O.colors(17, 0, g.n, k)
    rp, col, c = _device_inputs(torch, g, colors)
    got = P.cc_count_cycle_noalloc(0, None, L, g.n, rp.data_ptr(), col.data_ptr(), c.data_ptr())
    assert got == O.dp_count(g, k, e, colors)[0]


def test_noalloc_rejects_degree_beyond_limit(env):
    torch, P, _ = env
    g = _hub_and_clique(65536)
    rp, col, c = _device_inputs(torch, g, O.colors(17, 0, g.n, 6))
    with pytest.raises(P.CCError) as ei:
        P.cc_count_cycle_noalloc(0, None, 6, g.n, rp.data_ptr(), col.data_ptr(), c.data_ptr())
    assert P.ERRORS[ei.value.code] == "CC_ERR_INVALID_ARG"
