"""The coupled body block of the preconditioner after SEM steps (C ABI
rbfib_sem_step, rbfib_body_block_info): its inverse RPY matrix, updated from
the previous configuration's inverse (rotated with each body's rotation,
then Newton-Schulz steps) or rebuilt by Gauss-Jordan, matches a Gauss-Jordan
inverse built from scratch for the same configuration.  The two grids'
preconditioner outputs agree to the FP32 accuracy of the inverse."""
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


def _grid(B, w, q, quat):
    g = B.Grid(w.n, h=w.h, eta=w.eta, periodic=w.periodic, wall_vel=w.wall_vel, precision=B.FP64, rtol=1e-8)
    g.set_bodies(w.blob_offsets, w.ref_blobs, q, quat)
    return g


def test_body_block_after_sem_steps_matches_fresh_build(B):
    w = workloads.small_case(n=(16, 16, 16), n_bodies=3, blobs=12, seed=53)
    q0 = np.asarray(w.q, dtype=np.float64).reshape(-1, 3)
    quat0 = np.asarray(w.quat, dtype=np.float64).reshape(-1, 4)
    ga = _grid(B, w, q0, quat0)                 # Gauss-Jordan at the first configuration
    dense, warm0 = ga.body_block_info()
    assert dense
    p = B.sem_params(w.potentials, dt=0.05, kT=1.0)
    q = torch.tensor(q0.ravel(), device="cuda")
    quat = torch.tensor(quat0.ravel(), device="cuda")
    st, _ = ga.sem_step(p, w.seed, 0, 0, q, quat)   # rebuilds at the same configuration
    assert st == 0
    _, warm1 = ga.body_block_info()
    assert warm1 == warm0 + 1                   # an unchanged configuration always starts warm
    q1, quat1 = q.clone(), quat.clone()
    st, _ = ga.sem_step(p, w.seed, 1, 0, q, quat)   # rebuilds at (q1, quat1), then moves on
    assert st == 0
    gb = _grid(B, w, q1.cpu().numpy().reshape(-1, 3), quat1.cpu().numpy().reshape(-1, 4))
    n = ga.n_total
    gen = torch.Generator(device="cuda").manual_seed(7)
    r = torch.randn(n, dtype=torch.float64, device="cuda", generator=gen)
    za = ga.apply_preconditioner(r)
    zb = gb.apply_preconditioner(r)
    torch.cuda.synchronize()
    rel = (torch.linalg.norm(za - zb) / torch.linalg.norm(zb)).item()
    assert rel < 2e-3, rel
    ga.close()
    gb.close()
