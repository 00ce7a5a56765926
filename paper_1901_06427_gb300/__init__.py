"""GB300-native RB-FIB mobility solve (Sprinkle, Donev, Bhalla, Patankar,
Brownian dynamics of fully confined suspensions of rigid particles without
Green's functions): a C-ABI CUDA library (librbfib.so, include/rbfib.h) and a
thin ctypes binding.  PyTorch supplies device memory and streams only; every
step of the solve runs in the library's kernels.  There is no CPU fallback:
if the library is missing, importing ``paper_1901_06427_gb300.binding``
raises.
"""
__all__ = ["binding"]
