"""Reader of the stored expected values in tests/golden/ (written by
tests/golden/make_golden.py from the CPU oracle only)."""
from __future__ import annotations

import hashlib
import os

import numpy as np

import graphgen as gg

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def fingerprint(g) -> str:
    h = hashlib.sha1()
    h.update(np.ascontiguousarray(g.row_ptr, dtype="<i8").tobytes())
    h.update(np.ascontiguousarray(g.col, dtype="<i4").tobytes())
    return h.hexdigest()


def _fields(parts):
    return dict(p.split("=", 1) for p in parts if "=" in p)


class Golden:
    def __init__(self, name: str):
        self.graph_spec, self.graph_sha = {}, {}
        self.counts, self.filtered, self.sources, self.requests = {}, {}, {}, []
        with open(os.path.join(GOLDEN, f"{name}.txt")) as f:
            for line in f:
                if not line.strip() or line.startswith("#"):
                    continue
                parts = line.split()
                kw = _fields(parts)
                if parts[0] == "graph":
                    self.graph_spec[parts[1]] = parts[2]
                    self.graph_sha[parts[1]] = kw["sha1"]
                elif parts[0] == "request":
                    self.requests.append((parts[2], parts[3], int(kw["first"]), int(kw["trials"])))
                else:
                    key = (parts[1], parts[2], int(kw["seed"]), int(kw["trial"]))
                    if parts[0] == "count":
                        self.counts[key] = (int(kw["value"]), kw["overflow"] == "1")
                    elif parts[0] == "filtered":
                        srcs = tuple(int(x) for x in kw["sources"].split(","))
                        self.filtered[key + (srcs,)] = (int(kw["value"]), kw["overflow"] == "1")
                    elif parts[0] == "source":
                        self.sources.setdefault(key, {})[int(kw["vertex"])] = int(kw["value"])
        self._graphs = {}

    def graph(self, name: str):
        """The graph regenerated from its recorded generator call, checked
        against the recorded fingerprint."""
        if name not in self._graphs:
            g = eval(self.graph_spec[name], {"gg": gg})
            assert fingerprint(g) == self.graph_sha[name], f"graph {name} differs from the one the values were made on"
            self._graphs[name] = g
        return self._graphs[name]


_cache = {}


def load(name: str) -> Golden:
    if name not in _cache:
        _cache[name] = Golden(name)
    return _cache[name]
