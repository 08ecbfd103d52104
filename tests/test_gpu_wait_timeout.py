"""A bounded device wait that gives up reaches the caller as CC_ERR_TIMEOUT.

One wait exists inside a kernel: in the per-CTA push of the plain-cycle path a
thread that finds a vertex claimed by another thread of its CTA waits, with an
iteration limit, for the claimant to publish the vertex's local index.  When
the limit is reached the contribution is skipped and the kernel sets the
timeout flag, so the count is incomplete and must never come back as CC_OK.

The test build libcc_waittest.so (same sources, CC_TEST_WAIT_EXPIRES set)
sends every such thread into the wait with a limit of zero, so the wait gives
up at its first entry on any graph where a vertex is reached twice at one
level.  No memory access changes and no wait can last: nothing here can hang
or fault the GPU.  Both the allocating count and the count without device
allocation must report CC_ERR_TIMEOUT, and the context must stay usable.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu

TIMEOUT = -7


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_04478_gb300 as P
    return torch, P, P.variant_library("libcc_waittest.so")


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def test_wait_that_gives_up_is_reported(env):
    torch, P, V = env
    g = gg.erdos_renyi(2000, 10000, 1)
    h = ctypes.c_void_p()
    assert V.cc_create(ctypes.byref(h), 0, None) == 0
    try:
        gid, qid = ctypes.c_int32(), ctypes.c_int32()
        rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
        cl = np.ascontiguousarray(g.col, dtype=np.int32)
        assert V.cc_load_csr(h, g.n, _p(rp, ctypes.c_int64), _p(cl, ctypes.c_int32), g.nnz, ctypes.byref(gid)) == 0
        k, e = gg.query("C5")
        ea = np.ascontiguousarray(np.asarray(e, dtype=np.int32).reshape(-1))
        assert V.cc_set_query(h, k, len(e), _p(ea, ctypes.c_int32), ctypes.byref(qid)) == 0
        assert V.cc_set_coloring_seed(h, 3) == 0
        out = np.zeros(1, dtype=np.uint64)
        # every source on the per-CTA push of the plain-cycle path (a threshold
        # above every degree, small enough to keep its 32-bit rows exact): its
        # wait gives up, the count is refused
        assert V.cc_set_heavy_degree(h, 1 << 16) == 0
        assert V.cc_count(h, gid, qid, 0, 1, _p(out, ctypes.c_uint64), None, None) == TIMEOUT
        # the context stays usable: the grouped path has no wait and counts exactly
        expect = O.dp_count(g, k, e, O.colors(3, 0, g.n, k))[0]
        assert V.cc_set_heavy_degree(h, 0) == 0
        assert V.cc_count(h, gid, qid, 0, 1, _p(out, ctypes.c_uint64), None, None) == 0
        assert int(out[0]) == expect
        # the count without device allocation reports it too
        colors = O.colors(3, 0, g.n, k)
        d_rp = torch.from_numpy(rp).cuda()
        d_col = torch.from_numpy(cl).cuda()
        d_c = torch.from_numpy(colors).cuda()
        cnt = ctypes.c_uint64(0)
        torch.cuda.synchronize()
        rc = V.cc_count_cycle_noalloc(0, None, 5, g.n, ctypes.c_void_p(d_rp.data_ptr()),
                                      ctypes.c_void_p(d_col.data_ptr()), ctypes.c_void_p(d_c.data_ptr()),
                                      ctypes.byref(cnt))
        assert rc == TIMEOUT
    finally:
        V.cc_destroy(h)
