"""Independent FP64 CPU oracle for the RB-FIB mobility solve.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of what the paper computes (Sec. III discrete operators, Sec. IV
Split-Euler-Maruyama scheme, Algorithm 1), written in numpy/scipy in float64.
Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library and never
imports it; the product path must never call into it.

Parity unpinned: none.  Every function here is pinned by a ``-m "not gpu"``
test against a closed form, an identity the paper states, a library routine or
brute force (see tests/test_oracle_*.py).
"""
from .grid import Grid

from . import operators, kernel, ib, rigid, saddle, solve, philox, noise, forces, sem, binning, adjoint

__all__ = ["Grid", "operators", "kernel", "ib", "rigid", "saddle", "solve",
           "philox", "noise", "forces", "sem", "binning", "adjoint"]
