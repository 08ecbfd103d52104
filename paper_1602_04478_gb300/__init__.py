"""GB300 colour-coding counts of treewidth-2 queries (arXiv 1602.04478).

Thin Python binding of the C-ABI in ``include/cc.h``: the functions below
carry the C names and only marshal arguments; every step of a count runs in
the library's CUDA kernels (``libcc.so``, built by ``_build.build()``).  There
is no CPU fallback: without the compiled library or a CUDA device the calls
raise.

PyTorch supplies the device memory (through the library's allocator hooks,
backed by torch's caching allocator) and the CUDA stream (torch's current
stream when the context is created).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcc.so")

CC_OK = 0
ERRORS = {
    -1: "CC_ERR_INVALID_ARG", -2: "CC_ERR_BAD_GRAPH", -3: "CC_ERR_NOT_TW2", -4: "CC_ERR_K_RANGE",
    -5: "CC_ERR_OOM", -6: "CC_ERR_OVERFLOW", -7: "CC_ERR_TIMEOUT", -8: "CC_ERR_CUDA",
    -9: "CC_ERR_UNSUPPORTED", -10: "CC_ERR_NOT_CONNECTED", -11: "CC_ERR_BOUNDS",
}
EXPORTED = [
    "cc_create", "cc_destroy", "cc_set_allocator", "cc_set_memory_budget", "cc_set_heavy_degree",
    "cc_set_procedure", "cc_set_triangle_list",
    "cc_load_csr", "cc_free_graph",
    "cc_graph_info", "cc_set_query", "cc_set_decomposition", "cc_plan_inspect", "cc_plan_supported", "cc_plan_enumerate",
    "cc_query_info",
    "cc_set_coloring_seed",
    "cc_set_colors", "cc_clear_colors", "cc_count", "cc_count_per_vertex", "cc_work_units", "cc_work_detail",
    "cc_set_timing",
    "cc_get_timing", "cc_reset_timing", "cc_kernel_launches", "cc_count_cycle_noalloc", "cc_count_batch", "cc_set_graph_capture",
    "cc_set_batch_lanes", "cc_autotune_plan",
    "cc_autotune", "cc_server_create", "cc_server_destroy", "cc_server_load_csr", "cc_server_set_query",
    "cc_server_set_coloring_seed", "cc_server_submit", "cc_server_poll", "cc_server_stats", "cc_strerror",
]


class cc_server_result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_int64), ("status", ctypes.c_int32), ("trials", ctypes.c_int32),
                ("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double)]


class cc_request(ctypes.Structure):
    _fields_ = [("graph_id", ctypes.c_int32), ("query_id", ctypes.c_int32), ("first_trial", ctypes.c_int32),
                ("trials", ctypes.c_int32)]

_lib = None

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class CCError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        msg = lib().cc_strerror(code).decode() if _lib is not None else ERRORS.get(code, str(code))
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({msg})")


def build(force: bool = False) -> str:
    return _build.build(force=force)


def load_library(path: str):
    """A CDLL of `path` with the C-ABI's argument and result types set."""
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I32, I64, U64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    I32P, I64P = ctypes.POINTER(I32), ctypes.POINTER(I64)
    U64P, U8P, DP = ctypes.POINTER(U64), ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ctypes.c_double)
    sig = {
        "cc_create": ([ctypes.POINTER(P), ctypes.c_int, P], ctypes.c_int),
        "cc_destroy": ([P], None),
        "cc_set_allocator": ([P, ALLOC_FN, FREE_FN, P], ctypes.c_int),
        "cc_set_memory_budget": ([P, ctypes.c_size_t], ctypes.c_int),
        "cc_set_heavy_degree": ([P, ctypes.c_int], ctypes.c_int),
        "cc_set_procedure": ([P, ctypes.c_int], ctypes.c_int),
        "cc_set_triangle_list": ([P, ctypes.c_int], ctypes.c_int),
        "cc_load_csr": ([P, I64, I64P, I32P, I64, I32P], ctypes.c_int),
        "cc_free_graph": ([P, I32], ctypes.c_int),
        "cc_graph_info": ([P, I32, I64P, I64P, I64P], ctypes.c_int),
        "cc_set_query": ([P, ctypes.c_int, ctypes.c_int, I32P, I32P], ctypes.c_int),
        "cc_set_decomposition": ([P, I32, I32P, ctypes.c_int], ctypes.c_int),
        "cc_plan_inspect": ([ctypes.c_int, ctypes.c_int, I32P, I32P, ctypes.c_int, I32P, ctypes.c_int, I64P],
                            ctypes.c_int),
        "cc_plan_supported": ([ctypes.c_int, ctypes.c_int, I32P, I32P, ctypes.c_int], ctypes.c_int),
        "cc_plan_enumerate": ([ctypes.c_int, ctypes.c_int, I32P, I32P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
                              ctypes.c_int),
        "cc_query_info": ([P, I32, ctypes.POINTER(ctypes.c_int), I64P, ctypes.POINTER(ctypes.c_int),
                           ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cc_set_coloring_seed": ([P, U64], ctypes.c_int),
        "cc_set_colors": ([P, I32, U8P, ctypes.c_int], ctypes.c_int),
        "cc_clear_colors": ([P, I32], ctypes.c_int),
        "cc_count": ([P, I32, I32, ctypes.c_int, ctypes.c_int, U64P, DP, DP], ctypes.c_int),
        "cc_count_per_vertex": ([P, I32, I32, ctypes.c_int, U64P, U64P], ctypes.c_int),
        "cc_work_units": ([P, I32, I32, DP], ctypes.c_int),
        "cc_work_detail": ([P, I32, I32, ctypes.c_int, I32P, DP, DP, DP], ctypes.c_int),
        "cc_set_timing": ([P, ctypes.c_int], ctypes.c_int),
        "cc_get_timing": ([P, ctypes.c_char_p, DP, I64P, ctypes.c_int], ctypes.c_int),
        "cc_reset_timing": ([P], ctypes.c_int),
        "cc_kernel_launches": ([P, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "cc_count_cycle_noalloc": ([ctypes.c_int, P, ctypes.c_int, I64, P, P, P, U64P], ctypes.c_int),
        "cc_count_batch": ([P, ctypes.POINTER(cc_request), ctypes.c_int, U64P, ctypes.POINTER(ctypes.c_int)],
                           ctypes.c_int),
        "cc_set_graph_capture": ([P, ctypes.c_int], ctypes.c_int),
        "cc_set_batch_lanes": ([P, ctypes.c_int], ctypes.c_int),
        "cc_autotune_plan": ([P, I32, I32, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cc_autotune": ([P, I32, I32, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cc_server_create": ([ctypes.POINTER(P), ctypes.c_int, ctypes.c_int, ctypes.c_size_t], ctypes.c_int),
        "cc_server_destroy": ([P], None),
        "cc_server_load_csr": ([P, I64, I64P, I32P, I64, I32P], ctypes.c_int),
        "cc_server_set_query": ([P, ctypes.c_int, ctypes.c_int, I32P, I32P], ctypes.c_int),
        "cc_server_set_coloring_seed": ([P, U64], ctypes.c_int),
        "cc_server_submit": ([P, I32, I32, ctypes.c_int, ctypes.c_int, U64P, I64P], ctypes.c_int),
        "cc_server_poll": ([P, ctypes.POINTER(cc_server_result), ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "cc_server_stats": ([P, I64P, I64P, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
        "cc_strerror": ([ctypes.c_int], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


def lib():
    """The loaded C library (built first if its sources changed)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH) or _build.build() != LIB_PATH:
            raise ImportError("libcc.so is missing; build it with paper_1602_04478_gb300._build.build()")
        _lib = load_library(LIB_PATH)
    return _lib


def variant_library(name: str):
    """A test build of the library (see _build.VARIANTS), loaded beside libcc.so."""
    if name not in _build.VARIANTS:
        raise KeyError(name)
    _build.build()
    path = _build.variant_path(name)
    if not os.path.exists(path):
        raise ImportError(f"{name} is missing; build it with paper_1602_04478_gb300._build.build()")
    return load_library(path)


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _check(rc: int, where: str):
    if rc != CC_OK:
        raise CCError(rc, where)


# ------------------------- C-ABI calls, same names -------------------------
def cc_create(device: int = 0, stream: int | None = None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().cc_create(ctypes.byref(h), device, ctypes.c_void_p(stream or 0)), "cc_create")
    return h


def cc_destroy(h) -> None:
    lib().cc_destroy(h)


def cc_set_allocator(h, alloc, free, user=None) -> None:
    _check(lib().cc_set_allocator(h, alloc, free, user), "cc_set_allocator")


def cc_set_memory_budget(h, nbytes: int) -> None:
    _check(lib().cc_set_memory_budget(h, nbytes), "cc_set_memory_budget")


def cc_set_heavy_degree(h, degree: int) -> None:
    _check(lib().cc_set_heavy_degree(h, degree), "cc_set_heavy_degree")


PROC_DB, PROC_PS = 0, 1


def cc_set_procedure(h, procedure: int) -> None:
    _check(lib().cc_set_procedure(h, procedure), "cc_set_procedure")


def cc_set_triangle_list(h, enable: bool) -> None:
    _check(lib().cc_set_triangle_list(h, 1 if enable else 0), "cc_set_triangle_list")


def cc_load_csr(h, n: int, row_ptr: np.ndarray, col: np.ndarray) -> int:
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    if cl.size == 0:
        cl = np.zeros(1, dtype=np.int32)
    gid = ctypes.c_int32(0)
    _check(lib().cc_load_csr(h, n, _ptr(rp, ctypes.c_int64), _ptr(cl, ctypes.c_int32), int(rp[-1]),
                             ctypes.byref(gid)), "cc_load_csr")
    return gid.value


def cc_free_graph(h, gid: int) -> None:
    _check(lib().cc_free_graph(h, gid), "cc_free_graph")


def cc_graph_info(h, gid: int):
    n, nnz, md = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().cc_graph_info(h, gid, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(md)), "cc_graph_info")
    return n.value, nnz.value, md.value


def cc_set_query(h, k: int, edges) -> int:
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    qid = ctypes.c_int32(0)
    _check(lib().cc_set_query(h, k, int(e.shape[0]), _ptr(e, ctypes.c_int32), ctypes.byref(qid)), "cc_set_query")
    return qid.value


def cc_set_decomposition(h, qid: int, block_seq) -> None:
    s = np.ascontiguousarray(np.asarray(block_seq, dtype=np.int32).reshape(-1))
    if s.size == 0:
        s = np.zeros(1, dtype=np.int32)
        n = 0
    else:
        n = int(s.size)
    _check(lib().cc_set_decomposition(h, qid, _ptr(s, ctypes.c_int32), n), "cc_set_decomposition")


PLAN_KINDS = {0: "leaf", 1: "triangle", 2: "root_cycle", 3: "root_node", 4: "cycle"}


def decode_plan_records(out, w=None):
    """Blocks from cc_plan_inspect's int32 records."""
    w = len(out) if w is None else w
    blocks, i = [], 0
    while i < w:
        kind = int(out[i]); L = int(out[i + 1]); i += 2
        nodes = [int(x) for x in out[i:i + L]]; i += L
        nb = int(out[i]); i += 1
        bd = [int(x) for x in out[i:i + nb]]; i += nb
        nk = int(out[i]); i += 1
        kids = [int(x) for x in out[i:i + nk]]; i += nk
        blocks.append({"kind": PLAN_KINDS[kind], "nodes": nodes, "boundary": bd, "children": kids})
    return blocks


def cc_plan_inspect(k: int, edges, block_seq=None, allow_unsupported: bool = False):
    """Decomposition the library uses (host only).  Returns (blocks, aut).

    Raises CCError(CC_ERR_UNSUPPORTED) when the kernels cannot run the plan
    (cc_plan_supported) unless allow_unsupported."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    s = np.ascontiguousarray(np.asarray(block_seq if block_seq else [0], dtype=np.int32).reshape(-1))
    out = np.zeros(4096, dtype=np.int32)
    aut = ctypes.c_int64(0)
    w = lib().cc_plan_inspect(k, int(e.shape[0]), _ptr(e, ctypes.c_int32), _ptr(s, ctypes.c_int32),
                              len(block_seq) if block_seq else 0, _ptr(out, ctypes.c_int32), out.size,
                              ctypes.byref(aut))
    if w < 0:
        raise CCError(w, "cc_plan_inspect")
    blocks = decode_plan_records(out, w)
    if not allow_unsupported and cc_plan_supported(k, edges, block_seq) == 0:
        raise CCError(-9, "cc_plan_inspect")
    return blocks, aut.value


def cc_plan_supported(k: int, edges, block_seq=None) -> int:
    """1 if the kernels run the plan (host only), else 0."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    s = np.ascontiguousarray(np.asarray(block_seq if block_seq else [0], dtype=np.int32).reshape(-1))
    rc = lib().cc_plan_supported(k, int(e.shape[0]), _ptr(e, ctypes.c_int32), _ptr(s, ctypes.c_int32),
                                 len(block_seq) if block_seq else 0)
    if rc < 0:
        raise CCError(rc, "cc_plan_supported")
    return rc


def cc_plan_enumerate(k: int, edges):
    """Every decomposition tree of the query (host only): list of dicts with
    the contraction sequence (for cc_set_decomposition), whether the library
    supports it, the paper's ranking factors, the library's join cost, and
    whether cc_set_query (default) or the paper's factors alone (paper) pick it."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    out = np.zeros(1 << 16, dtype=np.int32)
    n = ctypes.c_int(0)
    w = lib().cc_plan_enumerate(k, int(e.shape[0]), _ptr(e, ctypes.c_int32), _ptr(out, ctypes.c_int32), out.size,
                                ctypes.byref(n))
    if w < 0:
        raise CCError(w, "cc_plan_enumerate")
    plans, i = [], 0
    while i < min(w, out.size):
        m = int(out[i])
        plans.append({"supported": bool(out[i + 1]), "longest": int(out[i + 2]), "boundary": int(out[i + 3]),
                      "annotations": int(out[i + 4]), "default": bool(out[i + 5]), "paper": bool(out[i + 6]),
                      "cost": int(out[i + 7]), "seq": [int(x) for x in out[i + 8:i + 8 + m]]})
        i += 8 + m
    return plans


def cc_query_info(h, qid: int):
    k, nb, lc = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    aut = ctypes.c_int64()
    _check(lib().cc_query_info(h, qid, ctypes.byref(k), ctypes.byref(aut), ctypes.byref(nb), ctypes.byref(lc)),
           "cc_query_info")
    return {"k": k.value, "aut": aut.value, "n_blocks": nb.value, "longest_cycle": lc.value}


def cc_set_coloring_seed(h, seed: int) -> None:
    _check(lib().cc_set_coloring_seed(h, seed), "cc_set_coloring_seed")


def cc_set_colors(h, gid: int, colors: np.ndarray) -> None:
    c = np.ascontiguousarray(colors, dtype=np.uint8)
    T = 1 if c.ndim == 1 else int(c.shape[0])
    _check(lib().cc_set_colors(h, gid, _ptr(c, ctypes.c_uint8), T), "cc_set_colors")


def cc_clear_colors(h, gid: int) -> None:
    _check(lib().cc_clear_colors(h, gid), "cc_clear_colors")


def cc_count(h, gid: int, qid: int, first_trial: int = 0, T: int = 1, allow_overflow: bool = False):
    """Returns (colorful uint64[T], estimate float64[T], aut)."""
    col = np.zeros(T, dtype=np.uint64)
    est = np.zeros(T, dtype=np.float64)
    aut = ctypes.c_double(0)
    rc = lib().cc_count(h, gid, qid, first_trial, T, _ptr(col, ctypes.c_uint64), _ptr(est, ctypes.c_double),
                        ctypes.byref(aut))
    if not (allow_overflow and rc == -6):
        _check(rc, "cc_count")
    return col, est, aut.value


def cc_count_per_vertex(h, gid: int, qid: int, n: int, trial: int = 0):
    pv = np.zeros(n, dtype=np.uint64)
    tot = ctypes.c_uint64(0)
    _check(lib().cc_count_per_vertex(h, gid, qid, trial, _ptr(pv, ctypes.c_uint64), ctypes.byref(tot)),
           "cc_count_per_vertex")
    return pv, tot.value


def cc_work_units(h, gid: int, qid: int) -> float:
    u = ctypes.c_double(0)
    _check(lib().cc_work_units(h, gid, qid, ctypes.byref(u)), "cc_work_units")
    return u.value


STAGE_KINDS = {0: "leaf", 1: "triangle", 2: "root_cycle", 3: "root_node", 4: "cycle"}


def cc_work_detail(h, gid: int, qid: int):
    """Per-stage structural work: list of dicts with kind, units,
    alg_bytes and (root cycle) scans, the data edges scanned per level."""
    cap = 64
    kind = np.zeros(cap, dtype=np.int32)
    units = np.zeros(cap, dtype=np.float64)
    nbytes = np.zeros(cap, dtype=np.float64)
    scans = np.zeros(8 * cap, dtype=np.float64)
    n = lib().cc_work_detail(h, gid, qid, cap, _ptr(kind, ctypes.c_int32), _ptr(units, ctypes.c_double),
                             _ptr(nbytes, ctypes.c_double), _ptr(scans, ctypes.c_double))
    if n < 0:
        raise CCError(n, "cc_work_detail")
    return [{"kind": STAGE_KINDS[int(kind[i])], "units": float(units[i]), "alg_bytes": float(nbytes[i]),
             "scans": [float(x) for x in scans[8 * i:8 * i + 8]]} for i in range(min(n, cap))]


def cc_set_timing(h, enable: bool) -> None:
    _check(lib().cc_set_timing(h, 1 if enable else 0), "cc_set_timing")


def cc_get_timing(h, cap: int = 64):
    names = ctypes.create_string_buffer(48 * cap)
    ms = np.zeros(cap, dtype=np.float64)
    cnt = np.zeros(cap, dtype=np.int64)
    n = lib().cc_get_timing(h, names, _ptr(ms, ctypes.c_double), _ptr(cnt, ctypes.c_int64), cap)
    if n < 0:
        raise CCError(n, "cc_get_timing")
    out = {}
    for i in range(min(n, cap)):
        nm = names.raw[48 * i:48 * (i + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (float(ms[i]), int(cnt[i]))
    return out


def cc_kernel_launches(h) -> int:
    out = ctypes.c_uint64(0)
    _check(lib().cc_kernel_launches(h, ctypes.byref(out)), "cc_kernel_launches")
    return int(out.value)


def cc_reset_timing(h) -> None:
    _check(lib().cc_reset_timing(h), "cc_reset_timing")


def cc_count_cycle_noalloc(device: int, stream: int | None, L: int, n: int, d_row_ptr: int, d_col: int,
                           d_colors: int) -> int:
    """Plain-cycle colourful count with no device allocation by the library.

    For callers that cannot let a library allocate GPU memory: inputs are
    device addresses (sorted CSR rows, colours) the caller owns; the
    library's working memory is a fixed 64 MiB static device array.  Calls
    that overlap on the GPU share that array and race."""
    out = ctypes.c_uint64(0)
    _check(lib().cc_count_cycle_noalloc(device, ctypes.c_void_p(stream or 0), L, n, ctypes.c_void_p(d_row_ptr),
                                        ctypes.c_void_p(d_col), ctypes.c_void_p(d_colors), ctypes.byref(out)),
           "cc_count_cycle_noalloc")
    return out.value


def cc_count_batch(h, requests):
    """requests: list of (graph_id, query_id, first_trial, trials).
    Returns (list of uint64 arrays, one per request; list of status codes)."""
    reqs = (cc_request * len(requests))(*[cc_request(*r) for r in requests])
    total = sum(r[3] for r in requests)
    out = np.zeros(max(total, 1), dtype=np.uint64)
    st = (ctypes.c_int * len(requests))()
    _check(lib().cc_count_batch(h, reqs, len(requests), _ptr(out, ctypes.c_uint64), st), "cc_count_batch")
    res, i = [], 0
    for r in requests:
        res.append(out[i:i + r[3]].copy())
        i += r[3]
    return res, [int(x) for x in st]


def cc_set_graph_capture(h, enable: bool) -> None:
    _check(lib().cc_set_graph_capture(h, 1 if enable else 0), "cc_set_graph_capture")


def cc_set_batch_lanes(h, lanes: int) -> None:
    _check(lib().cc_set_batch_lanes(h, lanes), "cc_set_batch_lanes")


def cc_autotune_plan(h, gid: int, qid: int) -> int:
    """Time every supported decomposition tree on the graph and keep the
    fastest; returns its index among the supported trees."""
    i = ctypes.c_int(0)
    _check(lib().cc_autotune_plan(h, gid, qid, ctypes.byref(i)), "cc_autotune_plan")
    return i.value


def cc_autotune(h, gid: int, qid: int) -> int:
    hd = ctypes.c_int(0)
    _check(lib().cc_autotune(h, gid, qid, ctypes.byref(hd)), "cc_autotune")
    return hd.value


class Server:
    """The library's serving loop (cc_server_*): graphs and queries resident,
    requests admitted by table memory as workers and memory free up."""

    def __init__(self, device: int = 0, workers: int = 4, memory_budget: int = 0):
        self.h = ctypes.c_void_p()
        _check(lib().cc_server_create(ctypes.byref(self.h), device, workers, memory_budget), "cc_server_create")
        self._bufs = {}
        self.n_of = {}

    def close(self):
        if self.h:
            lib().cc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_graph(self, g) -> int:
        rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
        cl = np.ascontiguousarray(g.col, dtype=np.int32)
        if cl.size == 0:
            cl = np.zeros(1, dtype=np.int32)
        gid = ctypes.c_int32(0)
        _check(lib().cc_server_load_csr(self.h, g.n, _ptr(rp, ctypes.c_int64), _ptr(cl, ctypes.c_int32),
                                        int(rp[-1]), ctypes.byref(gid)), "cc_server_load_csr")
        self.n_of[gid.value] = g.n
        return gid.value

    def set_query(self, k: int, edges) -> int:
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
        qid = ctypes.c_int32(0)
        _check(lib().cc_server_set_query(self.h, k, int(e.shape[0]), _ptr(e, ctypes.c_int32), ctypes.byref(qid)),
               "cc_server_set_query")
        return qid.value

    def set_seed(self, seed: int) -> None:
        _check(lib().cc_server_set_coloring_seed(self.h, seed), "cc_server_set_coloring_seed")

    def submit(self, gid: int, qid: int, first_trial: int, trials: int) -> int:
        buf = np.zeros(trials, dtype=np.uint64)
        t = ctypes.c_int64(0)
        _check(lib().cc_server_submit(self.h, gid, qid, first_trial, trials, _ptr(buf, ctypes.c_uint64),
                                      ctypes.byref(t)), "cc_server_submit")
        self._bufs[t.value] = buf
        return t.value

    def poll(self, cap: int = 256, timeout_ms: int = 0):
        out = (cc_server_result * cap)()
        n = lib().cc_server_poll(self.h, out, cap, timeout_ms)
        if n < 0:
            raise CCError(n, "cc_server_poll")
        res = []
        for r in out[:n]:
            res.append({"ticket": r.ticket, "status": r.status, "trials": r.trials, "submit_s": r.submit_s,
                        "admit_s": r.admit_s, "done_s": r.done_s, "colorful": self._bufs.pop(r.ticket)})
        return res

    def stats(self):
        p, r = ctypes.c_int64(), ctypes.c_int64()
        b = ctypes.c_size_t()
        _check(lib().cc_server_stats(self.h, ctypes.byref(p), ctypes.byref(r), ctypes.byref(b)), "cc_server_stats")
        return {"waiting": p.value, "running": r.value, "bytes_in_flight": b.value}


def cc_strerror(code: int) -> str:
    return lib().cc_strerror(code).decode()


# --------------------------- convenience wrapper ---------------------------
class Context:
    """A library context on one CUDA device, on torch's current stream, with
    torch's caching allocator behind the library's device allocations."""

    def __init__(self, device: int = 0, torch_allocator: bool = True, budget_bytes: int = 0):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("paper_1602_04478_gb300 needs a CUDA device (no CPU fallback)")
        self.device = device
        with torch.cuda.device(device):
            self.stream = torch.cuda.current_stream(device)
            self.h = cc_create(device, self.stream.cuda_stream)
        self._keep = []
        if torch_allocator:
            dev, stream = device, self.stream

            def _alloc(nbytes, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
                except Exception:  # out of memory: the library reports CC_ERR_OOM
                    return None

            def _free(ptr, nbytes, user):
                torch.cuda.caching_allocator_delete(ptr)

            a, f = ALLOC_FN(_alloc), FREE_FN(_free)
            self._keep = [a, f]
            cc_set_allocator(self.h, a, f, None)
        if budget_bytes:
            cc_set_memory_budget(self.h, budget_bytes)
        self.n_of = {}

    def close(self):
        if self.h:
            cc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_graph(self, g) -> int:
        gid = cc_load_csr(self.h, g.n, g.row_ptr, g.col)
        self.n_of[gid] = g.n
        return gid

    def free_graph(self, gid: int) -> None:
        cc_free_graph(self.h, gid)
        self.n_of.pop(gid, None)

    def set_query(self, k: int, edges) -> int:
        return cc_set_query(self.h, k, edges)

    def count(self, gid: int, qid: int, first_trial: int = 0, T: int = 1, allow_overflow: bool = False):
        return cc_count(self.h, gid, qid, first_trial, T, allow_overflow)

    def count_per_vertex(self, gid: int, qid: int, trial: int = 0):
        return cc_count_per_vertex(self.h, gid, qid, self.n_of[gid], trial)
