"""The confined boomerang of App. A on the GPU against the oracle, in a
reduced slit (20h x 20h x 12h, x and y periodic, six-point kernel): the body
forces with the buoyant weight of every blob and the blob-wall repulsion, one
SEM step (Algorithm 1) of the L-shaped body tilted towards the bottom wall,
and the same step without the RFD drift (the naive Euler-Maruyama scheme of
App. A's biased curve)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import saddle, forces, sem  # noqa: E402
import workloads  # noqa: E402
from gpu_common import assert_close, F64_OP, SEM_STEP  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_1901_06427_gb300.binding as binding
    binding.lib()
    return binding


def reduced(dtau=0.14):
    w = workloads.boomerang_slit(dtau, n=(20, 20, 12))
    ang = np.deg2rad(25.0)                    # tilted: the arms rise from the cross point near the wall
    axis = np.array([1.0, -1.0, 0.0]) / np.sqrt(2.0)
    w.bodies[0].quat = np.concatenate([[np.cos(ang / 2)], np.sin(ang / 2) * axis])
    w.bodies[0].q = np.array([6.0, 5.0, 2.0])
    og = oracle.Grid(w.n, periodic=w.periodic, kernel=6)
    ob = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
    assert ob.positions()[:, 2].min() > 0.5
    return w, og, ob


def dev(x):
    return torch.tensor(np.asarray(x).ravel(), dtype=torch.float64, device="cuda")


def test_boomerang_forces(B):
    w, og, ob = reduced()
    pot = dict(w.potentials)
    pot["blob_gravity"] = 0.35                # larger than the physical weight, to weigh in the comparison
    g = B.grid_for(w)
    F = g.body_forces(B.sem_params(pot)).cpu().numpy()
    F0 = forces.body_forces(og, ob, pot).ravel()
    assert np.abs(F0[3:]).max() > 0.1         # the weight's torque about the cross point
    assert_close(F, F0, F64_OP, "boomerang forces")


@pytest.mark.parametrize("rfd", [True, False])
def test_boomerang_sem_step(B, rfd):
    w, og, ob = reduced()
    g = B.grid_for(w, rtol=1e-12)
    q, quat = dev(w.q), dev(w.quat)
    st, info = g.sem_step(B.sem_params(w.potentials, dt=w.dt, kT=1.0, rfd=rfd), 17, 3, 0, q, quat)
    ref = sem.sem_step(og, ob, w.eta, 1.0, w.dt, w.potentials, seed=17, step=3, attempt=0, rfd=rfd)
    assert st == 0 and not ref["reject"]
    if not rfd:
        assert info["solve_rfd"]["iterations"] == 0 and info["solve_stokes"]["iterations"] == 0
    assert_close(q.cpu().numpy().reshape(-1, 3) - w.q, ref["q"] - w.q, SEM_STEP, f"displacement (rfd={rfd})")
    assert_close(quat.cpu().numpy() - w.quat.ravel(), ref["quat"].ravel() - w.quat.ravel(), SEM_STEP,
                 f"orientation increment (rfd={rfd})")
