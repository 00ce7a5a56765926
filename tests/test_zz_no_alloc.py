"""The allocation-free fluid forcing entry point.

Some callers cannot call cudaMalloc: code that runs inside a custom device
allocator or memory pool (a nested allocation would re-enter it) and
applications that plan all of their device memory up front.  For them the
library offers rbfib_stochastic_forcing_static, which needs no grid object and
keeps its stress-field scratch in a fixed array of the library's device
image.  This file checks, through the C ABI, that it reproduces the
grid-based rbfib_stochastic_forcing on two calls in a row, and that it
rejects grids whose stress field does not fit its scratch.  It is collected
last so that a run stopping at the first failure has run everything else."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_1901_06427_gb300.binding as binding
    binding.lib()
    return binding


def _static(B, desc, kT, dt, seed, step, out):
    err = ctypes.create_string_buffer(256)
    st = B.lib().rbfib_stochastic_forcing_static(ctypes.byref(desc), kT, dt, seed, step, 0,
                                                 ctypes.c_void_p(out.data_ptr() if out is not None else 1),
                                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                                 err, len(err))
    return st, err.value.decode()


@pytest.mark.parametrize("make", [lambda: workloads.two_sphere_cavity(steps=1),
                                  lambda: workloads.small_case(n=(16, 10, 9), periodic=(True, False, False)),
                                  lambda: workloads.small_case(n=(16, 10, 9), periodic=(True, False, False),
                                                               free_slip=(False, False, True, False, False, True))])
def test_static_forcing_matches_grid_entry_point(B, make):
    w = make()
    g = B.grid_for(w)
    nf = g.layout()[3]
    out = torch.full((nf,), float("nan"), dtype=torch.float64, device="cuda")
    for step in (0, 1):                       # two calls in a row share the scratch
        ref = g.stochastic_forcing(1.0, 0.05, 4242, step).cpu().numpy()
        st, msg = _static(B, g.desc, 1.0, 0.05, 4242, step, out)
        torch.cuda.synchronize()
        assert st == B.OK, msg
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) <= 1e-15 * np.max(np.abs(ref))


def test_static_forcing_rejects_oversized_grid(B):
    d = B.GridDesc()
    d.n[0], d.n[1], d.n[2] = 128, 128, 64
    d.h, d.eta, d.kernel, d.restart, d.max_iter, d.rtol = 1.0, 1.0, 3, 30, 100, 1e-8
    st, msg = _static(B, d, 1.0, 0.05, 1, 0, None)
    assert st == B.EINVAL
    assert "exceeds the static scratch" in msg
