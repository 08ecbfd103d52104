"""Seeded synthetic data graphs and query shapes (inputs only, no method arithmetic).

Graphs come from ``graphgen.c`` (Erdos-Renyi, Chung-Lu, R-MAT, explicit edge
lists) and are returned as a symmetric CSR: ``row_ptr`` int64 [n+1] and ``col``
int32 [nnz], rows sorted, no self-loops, no duplicate edges.  Both the CPU
oracle and the CUDA library read these arrays; neither is imported here.

The named query shapes are the treewidth-2 patterns the benchmarks use.  The
paper's own query drawings are not available, so these are synthetic shapes
with the sizes the workloads name.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "_graphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator library in place (plain C, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P64 = ctypes.POINTER(ctypes.POINTER(ctypes.c_int64))
        P32 = ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))
        I64P = ctypes.POINTER(ctypes.c_int64)
        lib.gg_erdos_renyi.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, P64, P32, I64P]
        lib.gg_chung_lu.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                    P64, P32, I64P]
        lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_uint64, P64, P32, I64P]
        lib.gg_from_edges.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_int32), ctypes.c_int64,
                                      P64, P32, I64P]
        lib.gg_free.argtypes = [ctypes.c_void_p]
        for f in (lib.gg_erdos_renyi, lib.gg_chung_lu, lib.gg_rmat, lib.gg_from_edges):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass
class Graph:
    """Symmetric simple graph in CSR form (caller's vertex labelling)."""
    n: int
    row_ptr: np.ndarray  # int64 [n+1]
    col: np.ndarray      # int32 [nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def m(self) -> int:
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def edge_list(self) -> np.ndarray:
        """Undirected edges (a < b) as an int32 [m, 2] array."""
        src = np.repeat(np.arange(self.n, dtype=np.int64), self.degrees())
        sel = src < self.col
        return np.stack([src[sel], self.col[sel].astype(np.int64)], axis=1).astype(np.int32)


def _wrap(fn, *args, n: int, name: str) -> Graph:
    lib = _load()
    rp = ctypes.POINTER(ctypes.c_int64)()
    cl = ctypes.POINTER(ctypes.c_int32)()
    nnz = ctypes.c_int64(0)
    rc = fn(*args, ctypes.byref(rp), ctypes.byref(cl), ctypes.byref(nnz))
    if rc != 0:
        raise RuntimeError(f"graph generator failed (rc={rc}) for {name}")
    try:
        row_ptr = np.ctypeslib.as_array(rp, shape=(n + 1,)).copy()
        col = np.ctypeslib.as_array(cl, shape=(max(nnz.value, 1),))[: nnz.value].copy()
    finally:
        lib.gg_free(ctypes.cast(rp, ctypes.c_void_p))
        lib.gg_free(ctypes.cast(cl, ctypes.c_void_p))
    return Graph(n=n, row_ptr=row_ptr, col=col, name=name)


def erdos_renyi(n: int, m: int, seed: int) -> Graph:
    """G(n, m): m distinct uniformly drawn non-loop pairs."""
    return _wrap(_load().gg_erdos_renyi, n, m, seed, n=n, name=f"er_n{n}_m{m}_s{seed}")


def chung_lu(n: int, mean_deg: float, gamma: float, seed: int) -> Graph:
    """Chung-Lu power-law graph with degree exponent ``gamma`` (P(d) ~ d^-gamma)."""
    return _wrap(_load().gg_chung_lu, n, float(mean_deg), float(gamma), seed, n=n,
                 name=f"cl_n{n}_d{mean_deg:g}_g{gamma:g}_s{seed}")


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int) -> Graph:
    """R-MAT graph on 2^scale vertices from edge_factor * 2^scale draws."""
    n = 1 << scale
    return _wrap(_load().gg_rmat, scale, edge_factor, a, b, c, seed, n=n,
                 name=f"rmat_s{scale}_ef{edge_factor}_s{seed}")


def from_edges(n: int, edges) -> Graph:
    """CSR of an explicit undirected edge list (duplicates and loops dropped)."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    return _wrap(_load().gg_from_edges, n, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                 int(e.shape[0]), n=n, name=f"edges_n{n}_m{e.shape[0]}")


def complete_graph(n: int) -> Graph:
    """K_n, built directly as a CSR (row v holds every other vertex)."""
    if n <= 1:
        return Graph(n=max(n, 0), row_ptr=np.zeros(max(n, 0) + 1, dtype=np.int64),
                     col=np.zeros(0, dtype=np.int32), name=f"complete_n{n}")
    ids = np.arange(n, dtype=np.int32)
    col = np.broadcast_to(ids, (n, n))[~np.eye(n, dtype=bool)].astype(np.int32)
    row_ptr = np.arange(n + 1, dtype=np.int64) * (n - 1)
    return Graph(n=n, row_ptr=row_ptr, col=np.ascontiguousarray(col), name=f"complete_n{n}")


def wheel_with_chords(n_ring: int = 9000, chords: int = 30000, seed: int = 11) -> Graph:
    """A hub adjacent to all ring vertices 1..n_ring, the ring itself and
    `chords` random chords between ring vertices: one vertex of very high
    degree and many of moderate degree."""
    rng = np.random.default_rng(seed)
    n = n_ring + 1
    e = [(0, i) for i in range(1, n)] + [(i, i % n_ring + 1) for i in range(1, n)]
    e += [tuple(x) for x in rng.integers(1, n, size=(chords, 2)) if x[0] != x[1]]
    return from_edges(n, np.array(e))


def relabel(g: Graph, perm: np.ndarray) -> Graph:
    """The same graph with vertex v renamed perm[v]."""
    el = g.edge_list()
    perm = np.asarray(perm, dtype=np.int64)
    return from_edges(g.n, np.stack([perm[el[:, 0]], perm[el[:, 1]]], axis=1))


# ------------------------------ query shapes ------------------------------
def cycle(L: int):
    return L, [(i, (i + 1) % L) for i in range(L)]


QUERIES = {
    # k, edge list
    "triangle": cycle(3),
    "C4": cycle(4),
    "C5": cycle(5),
    "C6": cycle(6),
    # 4-cycle 0-1-2-3 with chord 0-2
    "diamond": (4, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2)]),
    # 4-cycle 0-1-2-3 with chord 0-2 and pendant 4 on vertex 1
    "chord_pendant": (5, [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2), (1, 4)]),
    # triangles {0,1,2} and {4,5,6} joined by the path 2-3-4
    "glasses": (7, [(0, 1), (1, 2), (2, 0), (4, 5), (5, 6), (6, 4), (2, 3), (3, 4)]),
    # 6-cycle 0..5 with pendants 6-0 and 7-3 (opposite cycle vertices)
    "C6_2pendants": (8, [(i, (i + 1) % 6) for i in range(6)] + [(0, 6), (3, 7)]),
    # the same with the pendants on adjacent cycle vertices, or both on one
    "C6_2pendants_adj": (8, [(i, (i + 1) % 6) for i in range(6)] + [(0, 6), (1, 7)]),
    "C6_2pendants_same": (8, [(i, (i + 1) % 6) for i in range(6)] + [(0, 6), (0, 7)]),
    # 5-cycle with a path of two edges hanging from one node
    "C5_pendant_path": (7, [(i, (i + 1) % 5) for i in range(5)] + [(0, 5), (5, 6)]),
    "C7": cycle(7),
    "C8": cycle(8),
}


def query(name: str):
    k, e = QUERIES[name]
    return k, [tuple(x) for x in e]
