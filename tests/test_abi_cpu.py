"""CPU-side checks of the boundary: the library builds, loads and exports every
entry point that include/cc.h declares (no compute call needs a GPU here)."""
import os
import re
import subprocess

import paper_1602_04478_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(cc_[a-z_]+)\s*\(", src)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_library_exports_every_declared_symbol():
    path = P.build()
    out = subprocess.check_output(["nm", "-D", "--defined-only", path]).decode()
    exported = set(line.split()[-1] for line in out.splitlines() if " T " in line)
    declared = declared_functions()
    assert declared, "no declarations found"
    missing = [n for n in declared if n not in exported]
    assert not missing, missing
    assert sorted(declared) == sorted(P.EXPORTED)


def test_library_loads_and_reports_errors_without_gpu():
    L = P.lib()
    assert P.cc_strerror(-3).startswith("query has no block decomposition")
    assert P.cc_strerror(0) == "ok"
    for name in P.EXPORTED:
        assert hasattr(L, name)


def test_error_table_matches_header():
    src = open(os.path.join(ROOT, "include", "cc.h")).read()
    codes = dict((int(v), k) for k, v in re.findall(r"#define (CC_ERR_[A-Z0-9_]+) \((-?\d+)\)", src))
    assert codes == P.ERRORS


def test_test_builds_export_the_same_symbols():
    # the test variants (same sources, one compile-time switch) keep the boundary
    from paper_1602_04478_gb300 import _build
    P.build()
    for name in _build.VARIANTS:
        path = _build.variant_path(name)
        out = subprocess.check_output(["nm", "-D", "--defined-only", path]).decode()
        exported = set(line.split()[-1] for line in out.splitlines() if " T " in line)
        assert not [n for n in declared_functions() if n not in exported], name
