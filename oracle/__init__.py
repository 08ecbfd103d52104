"""CPU oracle for colour-coding subgraph counting (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does, and this
package never imports the CUDA library: the two share no code.

``oracle.cpp`` holds the arithmetic (brute-force enumeration from the
definitions of Section 2 of arXiv 1602.04478, the decomposition of Section 4.1
and the DB / PS dynamic programs of Section 5).  This module only marshals
numpy arrays and Python ints.

Parity status of each function (what pins it, see tests/test_oracle_pins.py):
  brute_colorful   closed form k!*prod(n_c) in K_n; triangle and star closed
                   forms; exhaustive-colouring identity against brute_matches
  brute_matches    n!/(n-k)! in K_n; 2n for C_n in C_n
  automorphisms    textbook values (C_k: 2k, K_n: n!, stars, glasses)
  dp_count         brute_colorful on random graphs, every decomposition and
                   order; closed forms in K_n
  decompose        the paper's worked "Satellite" decomposition (Section 4.1);
                   rejection of K4 and K5 minus an edge (treewidth 3)
  colors           SplitMix64 published test vector
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "_oracle.so")
_lib = None

ORDER_PS, ORDER_DEGREE, ORDER_ID, ORDER_RANK = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle library in place (host C++ only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t)) if a is not None else None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        I64P, I32P = ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)
        U64P, U8P = ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint8)
        lib.or_splitmix64.argtypes = [ctypes.c_uint64]
        lib.or_splitmix64.restype = ctypes.c_uint64
        lib.or_color.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int]
        lib.or_color.restype = ctypes.c_int
        lib.or_colors.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, U8P]
        lib.or_colors.restype = None
        lib.or_brute_colorful.argtypes = [ctypes.c_int64, I64P, I32P, ctypes.c_int, ctypes.c_int, I32P,
                                          U8P, ctypes.c_int, ctypes.c_int32, U64P]
        lib.or_brute_matches.argtypes = [ctypes.c_int64, I64P, I32P, ctypes.c_int, ctypes.c_int, I32P, U64P]
        lib.or_automorphisms.argtypes = [ctypes.c_int, ctypes.c_int, I32P]
        lib.or_automorphisms.restype = ctypes.c_int64
        lib.or_dp_count.argtypes = [ctypes.c_int64, I64P, I32P, ctypes.c_int, ctypes.c_int, I32P, U8P,
                                    ctypes.c_int, I64P, I32P, ctypes.c_int, U8P, U64P, U64P,
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
        lib.or_cycle_units.argtypes = [ctypes.c_int64, I64P, I32P, ctypes.c_int, ctypes.c_int, U8P,
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        lib.or_cycle_units.restype = ctypes.c_double
        lib.or_decompose.argtypes = [ctypes.c_int, ctypes.c_int, I32P, I32P, ctypes.c_int, I32P,
                                     ctypes.c_int, I32P, ctypes.c_int, I32P]
        for f in (lib.or_brute_colorful, lib.or_brute_matches, lib.or_dp_count, lib.or_decompose):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _graph_arrays(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(g.col, dtype=np.int32)
    if cl.size == 0:
        cl = np.zeros(1, dtype=np.int32)
    return rp, cl


def _qedges(edges):
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    return e, int(e.shape[0])


def _u128(a) -> int:
    return int(a[0]) | (int(a[1]) << 64)


def splitmix64(x: int) -> int:
    """SplitMix64 next() from state x (the mix used by the colouring hash)."""
    return int(_load().or_splitmix64(x))


def color(seed: int, trial: int, v: int, k: int) -> int:
    return _load().or_color(seed, trial, v, k)


def colors(seed: int, trial: int, n: int, k: int) -> np.ndarray:
    out = np.zeros(max(n, 1), dtype=np.uint8)
    _load().or_colors(seed, trial, n, k, _p(out, ctypes.c_uint8))
    return out[:n]


def brute_colorful(g, k, edges, col, fixed_node=-1, fixed_vertex=-1) -> int:
    rp, cl = _graph_arrays(g)
    e, ne = _qedges(edges)
    c = np.ascontiguousarray(col, dtype=np.uint8)
    out = np.zeros(2, dtype=np.uint64)
    rc = _load().or_brute_colorful(g.n, _p(rp, ctypes.c_int64), _p(cl, ctypes.c_int32), k, ne,
                                   _p(e, ctypes.c_int32), _p(c, ctypes.c_uint8), fixed_node,
                                   fixed_vertex, _p(out, ctypes.c_uint64))
    if rc != 0:
        raise ValueError("invalid query")
    return _u128(out)


def brute_matches(g, k, edges) -> int:
    rp, cl = _graph_arrays(g)
    e, ne = _qedges(edges)
    out = np.zeros(2, dtype=np.uint64)
    rc = _load().or_brute_matches(g.n, _p(rp, ctypes.c_int64), _p(cl, ctypes.c_int32), k, ne,
                                  _p(e, ctypes.c_int32), _p(out, ctypes.c_uint64))
    if rc != 0:
        raise ValueError("invalid query")
    return _u128(out)


def automorphisms(k, edges) -> int:
    e, ne = _qedges(edges)
    return int(_load().or_automorphisms(k, ne, _p(e, ctypes.c_int32)))


class NotTreewidth2(ValueError):
    pass


def dp_count(g, k, edges, col, order="degree", choice=None, root_filter=None, per_source=False,
             timing=None):
    """Colourful matches by the paper's dynamic program.

    order: "degree" (DB, Section 5.1 order), "id" (DB with ids as the order),
    "ps" (one split, no order), or an int64 rank array (DB with that order).
    choice: decomposition choices (index into the candidate blocks per step).
    root_filter: optional 0/1 array restricting the root cycle's highest vertex.
    Returns (count, overflow) or (count, overflow, per_source list of ints).
    """
    rp, cl = _graph_arrays(g)
    e, ne = _qedges(edges)
    c = np.ascontiguousarray(col, dtype=np.uint8)
    rank = None
    if isinstance(order, str):
        kind = {"ps": ORDER_PS, "degree": ORDER_DEGREE, "id": ORDER_ID}[order]
    else:
        kind = ORDER_RANK
        rank = np.ascontiguousarray(order, dtype=np.int64)
    ch = np.ascontiguousarray(choice if choice is not None else [0], dtype=np.int32)
    filt = np.ascontiguousarray(root_filter, dtype=np.uint8) if root_filter is not None else None
    ps = np.zeros(2 * max(g.n, 1), dtype=np.uint64) if per_source else None
    out = np.zeros(2, dtype=np.uint64)
    ovf = ctypes.c_int(0)
    secs = ctypes.c_double(0)
    rc = _load().or_dp_count(g.n, _p(rp, ctypes.c_int64), _p(cl, ctypes.c_int32), k, ne,
                             _p(e, ctypes.c_int32), _p(c, ctypes.c_uint8), kind,
                             _p(rank, ctypes.c_int64), _p(ch, ctypes.c_int32),
                             len(choice) if choice is not None else 0,
                             _p(filt, ctypes.c_uint8), _p(ps, ctypes.c_uint64),
                             _p(out, ctypes.c_uint64), ctypes.byref(ovf), ctypes.byref(secs))
    if timing is not None:
        timing["dp_seconds"] = secs.value
    if rc == -2:
        raise NotTreewidth2("query has no decomposition into blocks (treewidth above 2)")
    if rc != 0:
        raise ValueError("invalid query")
    if per_source:
        p2 = ps.reshape(-1, 2)[: g.n]
        return _u128(out), bool(ovf.value), [int(a) | (int(b) << 64) for a, b in p2]
    return _u128(out), bool(ovf.value)


KIND_NAMES = {0: "leaf", 1: "cycle", 2: "root_cycle", 3: "root_node"}


def decompose(k, edges, choice=None, max_steps=64):
    """Blocks of the decomposition tree for a choice sequence.

    Returns (blocks, root, n_candidates) where each block is a dict with kind,
    nodes, boundary and children (block indices).
    """
    e, ne = _qedges(edges)
    ch = np.ascontiguousarray(choice if choice is not None else [0], dtype=np.int32)
    ncand = np.zeros(max_steps, dtype=np.int32)
    words = np.zeros(4096, dtype=np.int32)
    root = ctypes.c_int32(-1)
    nb = _load().or_decompose(k, ne, _p(e, ctypes.c_int32), _p(ch, ctypes.c_int32),
                              len(choice) if choice is not None else 0, _p(ncand, ctypes.c_int32),
                              max_steps, _p(words, ctypes.c_int32), words.size, ctypes.byref(root))
    steps = [int(x) for x in ncand if x > 0]
    if nb == -2:
        raise NotTreewidth2("query has no decomposition into blocks (treewidth above 2)")
    if nb < 0:
        raise ValueError("invalid query")
    blocks, w = [], 0
    for _ in range(nb):
        kind = int(words[w]); w += 1
        nn = int(words[w]); w += 1
        nodes = [int(x) for x in words[w:w + nn]]; w += nn
        nbd = int(words[w]); w += 1
        bd = [int(x) for x in words[w:w + nbd]]; w += nbd
        nk = int(words[w]); w += 1
        kids = [int(x) for x in words[w:w + nk]]; w += nk
        blocks.append({"kind": KIND_NAMES[kind], "nodes": nodes, "boundary": bd, "children": kids})
    return blocks, int(root.value), steps


def all_plans(k, edges, limit=10000):
    """Every choice sequence (one per decomposition tree order) by DFS."""
    plans = []

    def rec(prefix):
        if len(plans) >= limit:
            return
        _, _, steps = decompose(k, edges, prefix)
        depth = len(prefix)
        if depth >= len(steps):
            plans.append(list(prefix))
            return
        for c in range(steps[depth]):
            rec(prefix + [c])

    rec([])
    return plans


def cycle_units(g, L, k, source_filter=None, per_source=False, scans=False):
    """Structural DB work (edge-subset updates) of a plain root L-cycle.

    per_source: also the units by source; scans: also the data edges scanned
    out of each level (list of 8, both halves summed)."""
    rp, cl = _graph_arrays(g)
    filt = np.ascontiguousarray(source_filter, dtype=np.uint8) if source_filter is not None else None
    ps = np.zeros(max(g.n, 1), dtype=np.float64) if per_source else None
    sc = np.zeros(8, dtype=np.float64) if scans else None
    tot = _load().or_cycle_units(g.n, _p(rp, ctypes.c_int64), _p(cl, ctypes.c_int32), L, k,
                                 _p(filt, ctypes.c_uint8), _p(ps, ctypes.c_double), _p(sc, ctypes.c_double))
    out = [tot]
    if per_source:
        out.append(ps[:g.n])
    if scans:
        out.append([float(x) for x in sc])
    return tuple(out) if len(out) > 1 else tot
