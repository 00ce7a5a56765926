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
