"""The C-ABI library loads and exports every entry point declared in
include/rbfib.h (no GPU needed; nothing is called)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"\b(rbfib_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    import paper_1901_06427_gb300.binding as B
    if not os.path.exists(B.LIB_PATH):
        from paper_1901_06427_gb300 import build
        build.build()
    import ctypes
    L = ctypes.CDLL(B.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, f"missing exports: {missing}"
    assert len(_declared()) >= 16


def test_binding_covers_declared_symbols():
    import paper_1901_06427_gb300.binding as B
    B.lib()
    src = open(B.__file__).read()
    for n in _declared():
        assert f'"{n}"' in src, n


def test_binding_argument_counts_match_header():
    """Every ctypes signature of the binding has as many arguments as the
    header declares (a swapped or missing argument would crash the host)."""
    import paper_1901_06427_gb300.binding as B
    L = B.lib()
    hdr = "".join(open(os.path.join(ROOT, "include", f)).read()
                  for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))
    decl = {}
    for m in re.finditer(r"\b(?:int|void|const char\*|uint64_t|int64_t|rbfib_grid\*)\s+(rbfib_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", hdr):
        args = [a for a in m.group(2).split(",") if a.strip() and a.strip() != "void"]
        decl[m.group(1)] = len(args)
    assert set(decl) == set(_declared())
    for name, k in decl.items():
        assert len(getattr(L, name).argtypes) == k, name
