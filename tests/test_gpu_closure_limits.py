"""Plain-cycle closure at the edge of uint64: exact counts just below 2^64,
overflow reported (never wrapped) just above, on both closure paths (the
grouped heavy path -- level builds in both forms, single and paired pulls --
and the per-CTA push).

In the complete graph K_n every connected query on k nodes has exactly
k! * prod_c n_c colourful matches, n_c the size of colour class c (one vertex
per class, mapped onto the query's nodes in any order, is a match because all
pairs are adjacent; Section 2's definitions).  The oracle is pinned to this
closed form (tests/test_oracle_pins.py).  With balanced explicit colours
(v mod k) the closed form is k! * (n/k)^k:
  C6: K_3000 -> 720 * 500^6  = 1.125e19 < 2^64 (exact);
      K_3360 -> 720 * 560^6  = 2.22e19  > 2^64 (overflow);
  C5: K_12500 -> 120 * 2500^5 = 1.17e19 < 2^64 (exact);
      K_14000 -> 120 * 2800^5 = 2.07e19 > 2^64 (overflow).
Parity here means the exact value, or CC_ERR_OVERFLOW with the count entry
set to UINT64_MAX.  The C5 cases run on the grouped path only: the per-CTA
push of K_12500 is about 10^12 pushes.
"""
import ctypes
import math

import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu

U64_MAX = 2**64 - 1


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1602_04478_gb300 as P
    return P


def _count_complete(P, n, L, heavy):
    k, e = gg.cycle(L)
    g = gg.complete_graph(n)
    ctx = P.Context(0)
    try:
        gid = ctx.load_graph(g)
        P.cc_set_colors(ctx.h, gid, (np.arange(n) % k).astype(np.uint8))
        P.cc_set_heavy_degree(ctx.h, heavy)
        qid = ctx.set_query(k, e)
        col = np.zeros(1, dtype=np.uint64)
        rc = P.lib().cc_count(ctx.h, gid, qid, 0, 1, col.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                              None, None)
        return rc, int(col[0])
    finally:
        ctx.close()


def _closed_form(n, k):
    return math.factorial(k) * (n // k) ** k


@pytest.mark.parametrize("path", ["grouped", "per_cta"])
@pytest.mark.parametrize("n", [3000, 3360])
def test_c6_near_2_64(P, path, n):
    expect = _closed_form(n, 6)
    # grouped: every source heavy; per-CTA: every source light (threshold
    # above the maximum degree, which keeps the push's 32-bit rows exact)
    rc, got = _count_complete(P, n, 6, 0 if path == "grouped" else n)
    if expect <= U64_MAX:
        assert rc == 0 and got == expect
    else:
        assert P.ERRORS[rc] == "CC_ERR_OVERFLOW" and got == U64_MAX


@pytest.mark.parametrize("n", [12500, 14000])
def test_c5_near_2_64_grouped(P, n):
    expect = _closed_form(n, 5)
    rc, got = _count_complete(P, n, 5, 0)
    if expect <= U64_MAX:
        assert rc == 0 and got == expect
    else:
        assert P.ERRORS[rc] == "CC_ERR_OVERFLOW" and got == U64_MAX
