"""The driven monolayer of Sec. V.B at reduced size, against the oracle:
eight 12-blob spheres (R = 1h) one radius above the bottom wall of a
24x12x12 channel periodic in x, no-slip side and bottom walls and a top wall
moving at (U, 0, 0) with U = 0.5; Yukawa pair repulsion (Eq. YukawaPot),
per-blob soft wall repulsion (Eq. Usoft) and the commensurate substrate
potential of amplitude 4kT.  Mobility solve and SEM step (Algorithm 1) in
FP64 and with FP32 kernels inside FP64 refinement, gated element by element."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import saddle, solve, sem, forces  # noqa: E402
import workloads  # noqa: E402
from gpu_common import assert_close, SOLVED, SEM_STEP, F64_OP  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_1901_06427_gb300.binding as binding
    binding.lib()
    return binding


@pytest.fixture(scope="module")
def case():
    w = workloads.driven_monolayer(wall_speed=0.5, cols=4, rows=2, nz=12, z=2.0)
    og = oracle.Grid(w.n, periodic=w.periodic, wall_vel=w.wall_vel)
    ob = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
    ref = sem.sem_step(og, ob, w.eta, w.kT, w.dt, w.potentials, seed=5, step=3)
    assert not ref["reject"]
    return w, og, ob, ref


def dev(x):
    return torch.tensor(np.asarray(x).ravel(), dtype=torch.float64, device="cuda")


def test_monolayer_forces(B, case):
    w, og, ob, ref = case
    g = B.grid_for(w)
    F = g.body_forces(B.sem_params(w.potentials)).cpu().numpy()
    assert_close(F, forces.body_forces(og, ob, w.potentials).ravel(), F64_OP, "monolayer forces")


@pytest.mark.parametrize("precision", ["fp64", "refined"])
def test_monolayer_mobility_solve(B, case, precision):
    """Forces and torques of the potentials with the moving top wall."""
    w, og, ob, ref = case
    prec = B.FP64 if precision == "fp64" else B.FP32_REFINED
    g = B.grid_for(w, precision=prec, rtol=1e-12 if precision == "fp64" else 1e-11)
    F = forces.body_forces(og, ob, w.potentials)
    U, info = g.mobility_solve(dev(F))
    x0 = solve.constrained(og, ob, w.eta, saddle.rhs(og, ob, w.eta, F=F))
    gate = SOLVED if precision == "fp64" else (1e-7, 1e-8)
    assert_close(U.cpu().numpy(), x0[-6 * w.n_bodies:], gate, f"monolayer U ({precision})")


@pytest.mark.parametrize("precision", ["fp64", "refined"])
def test_monolayer_sem_step(B, case, precision):
    w, og, ob, ref = case
    prec = B.FP64 if precision == "fp64" else B.FP32_REFINED
    g = B.grid_for(w, precision=prec, rtol=1e-12 if precision == "fp64" else 1e-11)
    q, quat = dev(w.q), dev(w.quat)
    st, info = g.sem_step(B.sem_params(w.potentials, dt=w.dt, kT=w.kT), 5, 3, 0, q, quat)
    assert st == 0
    dq = q.cpu().numpy().reshape(-1, 3) - w.q
    gate = SEM_STEP if precision == "fp64" else (1e-6, 1e-6)
    assert_close(dq, ref["q"] - w.q, gate, f"monolayer SEM displacement ({precision})")
    assert_close(quat.cpu().numpy() - w.quat.ravel(), ref["quat"].ravel() - w.quat.ravel(), gate,
                 f"monolayer SEM orientation increment ({precision})")
