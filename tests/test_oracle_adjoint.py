"""Pin of the oracle's adjoint gradients against central finite differences
of the oracle's own forward map (blob positions as independent inputs)."""
import numpy as np

import workloads
from oracle import Grid, saddle, adjoint, solve


def test_adjoint_gradient_matches_finite_differences():
    w = workloads.small_case(n=(9, 8, 7), n_bodies=2, blobs=12, seed=3, near_wall=True)
    g = Grid(w.n)
    b0 = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
    r0 = b0.positions().copy()
    b = b0.with_positions(r0)
    eta = 1.3
    slip = w.slip.ravel()
    F = w.force_torque
    op = solve.StokesOperator(g, eta)
    x, U = adjoint.forward(g, b, eta, slip, F, op=op)
    dr, dslip = adjoint.gradient(g, b, eta, x, 2.0 * U, op=op)
    rng = np.random.default_rng(0)
    eps = 1e-5
    scale = max(np.abs(dr).max(), np.abs(dslip).max())
    for _ in range(5):
        i, c = int(rng.integers(w.n_blobs)), int(rng.integers(3))
        rp, rm = r0.copy(), r0.copy()
        rp[i, c] += eps
        rm[i, c] -= eps
        Lp = adjoint.loss(adjoint.forward(g, b0.with_positions(rp), eta, slip, F, op=op)[1])
        Lm = adjoint.loss(adjoint.forward(g, b0.with_positions(rm), eta, slip, F, op=op)[1])
        assert abs((Lp - Lm) / (2 * eps) - dr[i, c]) < 1e-6 * scale
    for _ in range(5):
        k = int(rng.integers(slip.size))
        sp, sm = slip.copy(), slip.copy()
        sp[k] += eps
        sm[k] -= eps
        Lp = adjoint.loss(adjoint.forward(g, b, eta, sp, F, op=op)[1])
        Lm = adjoint.loss(adjoint.forward(g, b, eta, sm, F, op=op)[1])
        assert abs((Lp - Lm) / (2 * eps) - dslip[k]) < 1e-6 * scale


def test_stencil_gradient_is_derivative_of_weights():
    g = Grid((7, 6, 5), periodic=(True, False, False))
    from oracle import ib
    rng = np.random.default_rng(1)
    r = np.concatenate([rng.uniform(0.05, 1.0, (4, 3)), rng.uniform(1.5, 4.0, (4, 3))])
    e = 1e-6
    for a in range(3):
        idx, coef, dcoef = ib.stencil_grad(g, r, a)
        for bdir in range(3):
            rp, rm = r.copy(), r.copy()
            rp[:, bdir] += e
            rm[:, bdir] -= e
            ip, cp, _ = ib.stencil_grad(g, rp, a)
            im, cm, _ = ib.stencil_grad(g, rm, a)
            ok = np.all(ip == idx, axis=1) & np.all(im == idx, axis=1)   # same kernel points
            fd = (cp - cm) / (2 * e)
            assert np.abs(fd[ok] - dcoef[ok, :, bdir]).max() < 1e-6
