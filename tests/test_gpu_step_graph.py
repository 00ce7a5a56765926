"""The device-driven SEM step (the whole step of Algorithm 1 as one CUDA graph:
restart cycles and refinement sweeps in WHILE nodes, the body block's
warm-start choice in an IF/ELSE node, the rejection test on the device)
against the host-orchestrated step of the same grid and against the oracle,
over several consecutive steps, in FP64 and FP32-refined mode; and the
rejection path."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import sem  # noqa: E402
from gpu_common import case, assert_close, SEM_STEP  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_1901_06427_gb300.binding as binding
    binding.lib()
    return binding


def dev(x):
    return torch.tensor(np.asarray(x).ravel(), dtype=torch.float64, device="cuda")


def _grid(B, w, host, **kw):
    """A grid whose steps are host-orchestrated (host=True) or device-driven;
    the choice is read from the environment when the grid is created."""
    old = os.environ.get("RBFIB_NO_STEP_GRAPH")
    os.environ["RBFIB_NO_STEP_GRAPH"] = "1" if host else "0"
    try:
        return B.grid_for(w, **kw)
    finally:
        if old is None:
            del os.environ["RBFIB_NO_STEP_GRAPH"]
        else:
            os.environ["RBFIB_NO_STEP_GRAPH"] = old


@pytest.mark.parametrize("name,precision", [("walls", "fp64"), ("ragged42", "fp64"), ("xper_moving", "refined")])
def test_step_graph_matches_host_steps(B, name, precision):
    w, og, ob = case(name)
    prec = B.FP64 if precision == "fp64" else B.FP32_REFINED
    gh = _grid(B, w, True, precision=prec, rtol=1e-11)
    gd = _grid(B, w, False, precision=prec, rtol=1e-11)
    p = B.sem_params(w.potentials, dt=0.05, kT=1.0)
    qh, quath = dev(w.q), dev(w.quat)
    qd, quatd = dev(w.q), dev(w.quat)
    for k in range(4):                     # the graph is captured once and relaunched
        sh, ih = gh.sem_step(p, 21, k, 0, qh, quath)
        sd, idv = gd.sem_step(p, 21, k, 0, qd, quatd)
        assert sh == sd == 0
        assert gh.step_mode() == 0 and gd.step_mode() == 1
        for key in ("solve_rfd", "solve_stokes", "solve_main"):
            assert idv[key]["rel_residual"] <= 1e-11
            # same kernels in the same order, but FP32 atomics in the spreading
            # sum in another order: the FP32-refined counts may drift a little
            assert abs(idv[key]["iterations"] - ih[key]["iterations"]) <= 2 + 0.15 * ih[key]["iterations"]
        assert_close(qd.cpu().numpy(), qh.cpu().numpy(), (1e-9, 1e-9), f"q after step {k}")
        assert_close(quatd.cpu().numpy(), quath.cpu().numpy(), (1e-9, 1e-9), f"quat after step {k}")
    it, passes = gd.krylov_stats()
    assert it > 0 and passes >= 0


def test_step_graph_against_oracle(B):
    w, og, ob = case("walls")
    g = _grid(B, w, False, rtol=1e-12)
    q, quat = dev(w.q), dev(w.quat)
    st, info = g.sem_step(B.sem_params(w.potentials, dt=0.05, kT=1.0), 11, 2, 1, q, quat)
    ref = sem.sem_step(og, ob, w.eta, 1.0, 0.05, w.potentials, seed=11, step=2, attempt=1)
    assert st == 0 and info["rejected"] == 0 and g.step_mode() == 1
    assert_close(q.cpu().numpy().reshape(-1, 3) - w.q, ref["q"] - w.q, SEM_STEP, "device-driven SEM displacement")


def test_step_graph_rejection_leaves_configuration(B):
    """A huge force pushes a body through the bottom wall: the device-side
    test rejects the step and q, quat stay as they were; the next attempt
    with a normal force is accepted."""
    w, og, ob = case("walls")
    g = _grid(B, w, False, rtol=1e-10)
    fext = np.zeros((w.n_bodies, 6))
    fext[:, 2] = -1e5
    q, quat = dev(w.q), dev(w.quat)
    st, info = g.sem_step(B.sem_params(w.potentials, dt=0.05, kT=1.0, force_ext=dev(fext)), 1, 0, 0, q, quat)
    assert st == B.EREJECT and info["rejected"] == 1 and g.step_mode() == 1
    assert np.array_equal(q.cpu().numpy(), w.q.ravel())
    assert np.array_equal(quat.cpu().numpy(), w.quat.ravel())
    st, info = g.sem_step(B.sem_params(w.potentials, dt=0.05, kT=1.0), 1, 0, 1, q, quat)
    assert st == 0 and info["rejected"] == 0
    assert not np.array_equal(q.cpu().numpy(), w.q.ravel())
