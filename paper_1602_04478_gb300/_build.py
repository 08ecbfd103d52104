"""Compile the CUDA library (libcc.so) in place for sm_103a.

Each translation unit is compiled by nvcc in parallel into ``_build/`` and
linked into ``paper_1602_04478_gb300/libcc.so`` (shared CUDA runtime).
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
SOURCES = ["api.cu", "graph.cu", "join.cu", "triangle.cu", "cycle.cu", "cycle_heavy.cu", "cycle_plain.cu", "noalloc.cu", "batch.cu", "serve.cu", "plan.cpp"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-strict-aliasing",
         "-I" + os.path.join(ROOT, "include")]


def _digest(paths):
    h = hashlib.sha1()
    for p in paths:
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


def _headers():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))) + \
        [os.path.join(ROOT, "include", "cc.h")]


def _compile(src: str) -> str:
    path = os.path.join(CSRC, src)
    tag = _digest([path] + _headers())[:16]
    obj = os.path.join(BUILD, f"{src}.{tag}.o")
    if not os.path.exists(obj):
        tmp = obj + ".tmp%d" % os.getpid()
        cmd = [NVCC] + ARCH + FLAGS + ["-c", path, "-o", tmp]
        if src.endswith(".cpp"):
            cmd = [NVCC] + FLAGS + ["-x", "c++", "-c", path, "-o", tmp]
        subprocess.check_call(cmd)
        os.replace(tmp, obj)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    tag = _digest(srcs + _headers())
    stamp = LIB + ".stamp"
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == tag:
        return LIB
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call([NVCC] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(tag)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
