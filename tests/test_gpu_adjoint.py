"""Hand-written adjoint of the mobility solve (GPU) against the oracle's
adjoint gradient and central finite differences, and through the
torch.autograd.Function."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import saddle, adjoint  # noqa: E402
import workloads  # noqa: E402
from gpu_common import rel  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_1901_06427_gb300.binding as binding
    binding.lib()
    return binding


def dev(x):
    return torch.tensor(np.asarray(x).ravel(), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("blobs,radius,n", [(12, 1.0, (12, 10, 9)), (42, 2.5, (17, 15, 13))])
def test_adjoint_matches_oracle(B, blobs, radius, n):
    w = workloads.small_case(n=n, n_bodies=2, blobs=blobs, radius=radius, seed=9, near_wall=True)
    og = oracle.Grid(w.n)
    ob = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
    r = ob.positions() + 0.05 * np.random.default_rng(2).standard_normal((w.n_blobs, 3))
    obr = ob.with_positions(r)
    x0, U0 = adjoint.forward(og, obr, w.eta, w.slip.ravel(), w.force_torque)
    dr0, ds0 = adjoint.gradient(og, obr, w.eta, x0, 2.0 * U0)
    g = B.grid_for(w, rtol=1e-12)
    g.set_blob_positions(dev(r))
    U, info, x = g.mobility_solve(dev(w.force_torque), slip=dev(w.slip), return_x=True)
    assert rel(U.cpu().numpy(), U0) < 1e-8
    dr, ds, ainfo = g.mobility_solve_adjoint(2.0 * U, x)
    assert ainfo["rel_residual"] <= 1e-12
    assert rel(dr.cpu().numpy(), dr0) < 1e-7
    assert rel(ds.cpu().numpy(), ds0) < 1e-7


def test_autograd_function(B):
    from paper_1901_06427_gb300.autograd import MobilitySolve
    w = workloads.small_case(n=(12, 10, 9), n_bodies=2, blobs=12, seed=4)
    ob = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
    g = B.grid_for(w, rtol=1e-12)
    r = dev(ob.positions()).requires_grad_(True)
    slip = dev(w.slip).requires_grad_(True)
    U = MobilitySolve.apply(r, slip, g, dev(w.force_torque))
    L = (U ** 2).sum()
    L.backward()
    x0, U0 = adjoint.forward(oracle.Grid(w.n), ob.with_positions(ob.positions()), w.eta, w.slip.ravel(),
                             w.force_torque)
    dr0, ds0 = adjoint.gradient(oracle.Grid(w.n), ob.with_positions(ob.positions()), w.eta, x0, 2.0 * U0)
    assert rel(r.grad.cpu().numpy(), dr0) < 1e-7
    assert rel(slip.grad.cpu().numpy(), ds0) < 1e-7


@pytest.mark.slow
def test_adjoint_fullsize_finite_differences(B):
    """The 128x128x64 suspension of 64 spheres with active slip: FP32-refined
    forward and backward; sampled gradient components against central
    differences (step 1e-5) of FP64 forward solves."""
    w = workloads.adjoint_suspension()
    ob = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
    r0 = ob.positions()
    FT = dev(np.zeros((w.n_bodies, 6)))
    g = B.grid_for(w, precision=B.FP32_REFINED, rtol=1e-10)
    g.set_blob_positions(dev(r0))
    U, info, x = g.mobility_solve(FT, slip=dev(w.slip), return_x=True)
    dr, ds, ainfo = g.mobility_solve_adjoint(2.0 * U, x)
    dr = dr.cpu().numpy().reshape(-1, 3)
    ds = ds.cpu().numpy()
    gf = B.grid_for(w, precision=B.FP64, rtol=1e-11)

    def L_of(rr, ss):
        gf.set_blob_positions(dev(rr))
        Uf, _ = gf.mobility_solve(FT, slip=dev(ss))
        return float((Uf ** 2).sum())

    eps = 1e-5
    scale = max(np.abs(dr).max(), np.abs(ds).max())
    rng = np.random.default_rng(5)
    for _ in range(2):
        i, c = int(rng.integers(w.n_blobs)), int(rng.integers(3))
        rp, rm = r0.copy(), r0.copy()
        rp[i, c] += eps
        rm[i, c] -= eps
        fd = (L_of(rp, w.slip) - L_of(rm, w.slip)) / (2 * eps)
        assert abs(fd - dr[i, c]) < 1e-4 * scale
    for _ in range(2):
        k = int(rng.integers(ds.size))
        sp, sm = w.slip.ravel().copy(), w.slip.ravel().copy()
        sp[k] += eps
        sm[k] -= eps
        fd = (L_of(r0, sp) - L_of(r0, sm)) / (2 * eps)
        assert abs(fd - ds[k]) < 1e-4 * scale
