"""Compile the CUDA library (libcc.so) in place for sm_103a.

Each translation unit is compiled by nvcc in parallel into ``_build/`` and
linked into ``paper_1602_04478_gb300/libcc.so`` (shared CUDA runtime).

Test builds: ``VARIANTS`` names libraries that are the same library with a
compile-time switch set in the translation units that read it (the other
objects are shared with libcc.so).  Only tests load them.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libcc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
SOURCES = ["api.cu", "graph.cu", "join.cu", "triangle.cu", "cycle.cu", "cycle_heavy.cu", "cycle_plain.cu", "noalloc.cu", "batch.cu", "serve.cu", "pair.cu", "plan.cpp"]
# name -> (translation units that read the switch, extra flags)
VARIANTS = {
    # the per-CTA push's bounded wait gives up on its first entry
    "libcc_waittest.so": (("cycle_plain.cu", "noalloc.cu"), ("-DCC_TEST_WAIT_EXPIRES",)),
    # data-dependent indices checked against their arrays (status flag, access skipped)
    "libcc_boundscheck.so": (("cycle_plain.cu", "triangle.cu", "join.cu", "cycle.cu"), ("-DCC_BOUNDS_CHECK",)),
}
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-strict-aliasing",
         "-I" + os.path.join(ROOT, "include")]


def _digest(paths, extra=()):
    h = hashlib.sha1()
    for p in paths:
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(ARCH + FLAGS + list(extra)).encode())
    return h.hexdigest()


def _headers():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))) + \
        [os.path.join(ROOT, "include", "cc.h")]


def _compile(src: str, extra=()) -> str:
    path = os.path.join(CSRC, src)
    tag = _digest([path] + _headers(), extra)[:16]
    obj = os.path.join(BUILD, f"{src}.{tag}.o")
    if not os.path.exists(obj):
        tmp = obj + ".tmp%d" % os.getpid()
        cmd = [NVCC] + ARCH + FLAGS + list(extra) + ["-c", path, "-o", tmp]
        if src.endswith(".cpp"):
            cmd = [NVCC] + FLAGS + list(extra) + ["-x", "c++", "-c", path, "-o", tmp]
        subprocess.check_call(cmd)
        os.replace(tmp, obj)
    return obj


def _link(lib: str, objs) -> None:
    tmp = lib + ".tmp%d" % os.getpid()
    subprocess.check_call([NVCC] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + list(objs))
    os.replace(tmp, lib)


def _fresh(lib: str, tag: str) -> bool:
    stamp = lib + ".stamp"
    return os.path.exists(lib) and os.path.exists(stamp) and open(stamp).read() == tag


def _stamp(lib: str, tag: str) -> None:
    with open(lib + ".stamp", "w") as f:
        f.write(tag)


def variant_path(name: str) -> str:
    return os.path.join(HERE, name)


def build(force: bool = False, verbose: bool = False) -> str:
    """Build libcc.so and the test variants; returns libcc.so's path."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    jobs = []  # (library, tag, [(source, extra flags)])
    tag = _digest(srcs + _headers())
    if force or not _fresh(LIB, tag):
        jobs.append((LIB, tag, [(s, ()) for s in SOURCES]))
    for name, (units, extra) in VARIANTS.items():
        vtag = _digest(srcs + _headers(), extra)
        if force or not _fresh(variant_path(name), vtag):
            jobs.append((variant_path(name), vtag, [(s, extra if s in units else ()) for s in SOURCES]))
    if not jobs:
        return LIB
    todo = sorted({u for _, _, us in jobs for u in us})
    with cf.ThreadPoolExecutor(max_workers=len(todo)) as ex:
        objs = dict(zip(todo, ex.map(lambda u: _compile(*u), todo)))
    for lib, t, units in jobs:
        _link(lib, [objs[u] for u in units])
        _stamp(lib, t)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
