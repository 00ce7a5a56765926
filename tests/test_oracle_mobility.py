"""Pins of the oracle's constrained solve and mobility matrices: SPD blob and
body mobilities (Sec. III.C), the reduced form of Eq. (incompleteN) against a
direct sparse solve, isotropy forced by symmetry, discrete fluctuation-
dissipation balance (Eqs. LangevinM1, incompleteN) deterministically and by
sampling the oracle's own noise, and the drift expectation of Eq. (DriDef)
against finite differences of N."""
import numpy as np
import pytest

import workloads
from oracle import Grid, saddle, solve, rigid, ib, operators, noise, sem


def _setup(n=(8, 7, 6), per=(False, False, False), n_bodies=2, blobs=12, radius=1.0, seed=7,
           wall_speed=0.0, near_wall=False):
    w = workloads.small_case(n=n, periodic=per, n_bodies=n_bodies, blobs=blobs, radius=radius,
                             seed=seed, wall_speed=wall_speed, near_wall=near_wall)
    g = Grid(w.n, periodic=w.periodic, wall_vel=w.wall_vel)
    b = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
    return w, g, b


@pytest.mark.parametrize("per,ws", [((False, False, False), 0.0), ((True, False, False), 0.4),
                                    ((False, True, False), 0.0)])
def test_reduced_solve_matches_direct(per, ws):
    w, g, b = _setup(per=per, wall_speed=ws, near_wall=True)
    f = saddle.rhs(g, b, 1.3, F=w.force_torque, slip=w.slip,
                   f_fluid=np.random.default_rng(1).standard_normal(g.N_f))
    x_dir = solve.direct(g, b, 1.3, f)
    x_red = solve.constrained(g, b, 1.3, f)
    np.testing.assert_allclose(x_red, x_dir, rtol=0, atol=1e-11 * np.abs(x_dir).max())
    r = saddle.apply(g, b, 1.3, x_red) - f
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(f)
    A = saddle.assemble(g, b, 1.3)
    np.testing.assert_allclose(A @ x_red, saddle.apply(g, b, 1.3, x_red), atol=1e-12)


def test_weighted_saddle_matrix_is_symmetric():
    w, g, b = _setup(per=(True, False, False), near_wall=True)
    A = saddle.assemble(g, b, 0.9).toarray()
    WA = saddle.weights(g, b)[:, None] * A
    np.testing.assert_allclose(WA, WA.T, atol=1e-14)


def test_mobility_spd_and_reduced_formula():
    w, g, b = _setup(near_wall=True)
    eta = 1.0
    M = solve.blob_mobility(g, b, eta)
    assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0
    K = rigid.K_matrix(b.ref, b.offsets, b.quat)
    N = solve.body_mobility(M, K)
    assert np.abs(N - N.T).max() <= 1e-11 * np.abs(N).max()
    assert np.linalg.eigvalsh(0.5 * (N + N.T)).min() > 0
    # U = N F - N K^T M^-1 slip  (Eq. incompleteN without noise)
    f = saddle.rhs(g, b, eta, F=w.force_torque, slip=w.slip, walls=False)
    U = solve.direct(g, b, eta, f)[-6 * b.n_bodies:]
    expect = N @ w.force_torque.ravel() - N @ K.T @ np.linalg.solve(M, w.slip.ravel())
    np.testing.assert_allclose(U, expect, rtol=0, atol=1e-11 * np.abs(expect).max())


@pytest.mark.parametrize("blobs,radius,n", [(12, 1.0, 10), (42, 2.5, 12)])
def test_isotropy_of_centred_shell(blobs, radius, n):
    """A T_h-symmetric shell at the centre of a cubic no-slip box: the cube's
    symmetries force N_tt = mu_t I, N_rr = mu_r I, N_tr = 0."""
    g = Grid((n, n, n))
    shell = workloads.icosahedral_shell(blobs, radius)
    b = saddle.Bodies(shell, [0, blobs], [[n / 2, n / 2, n / 2]], [[1, 0, 0, 0]])
    M = solve.blob_mobility(g, b, 1.0)
    N = solve.body_mobility(M, rigid.K_matrix(b.ref, b.offsets, b.quat))
    mt, mr = N[0, 0], N[3, 3]
    np.testing.assert_allclose(N[:3, :3], mt * np.eye(3), atol=1e-11 * mt)
    np.testing.assert_allclose(N[3:, 3:], mr * np.eye(3), atol=1e-11 * mr)
    assert np.abs(N[:3, 3:]).max() < 1e-11 * mt


def _dense_stokes_inverse(g, eta):
    op = solve.StokesOperator(g, eta)
    V, _ = op.solve(np.eye(g.N_f))
    return V.T          # column j = L^{-1} e_j


def test_fluctuation_dissipation_deterministic():
    """c^2 J L^-1 DD DD^T L^-1 J^T = (2 kT/dt) M, c^2 = 2 eta kT/(dV dt), and the
    same for N through N^{1/2} = N K^T M^-1 M^{1/2} (Sec. III.C)."""
    w, g, b = _setup(n=(6, 5, 5), n_bodies=1, near_wall=True)
    eta, kT, dt = 1.3, 0.7, 0.05
    Linv = _dense_stokes_inverse(g, eta)
    DD = operators.tensor_divergence(g).toarray()
    J = ib.J_matrix(g, b.positions()).toarray()
    c2 = 2 * eta * kT / (g.dV * dt)
    B = J @ Linv @ DD
    M = solve.blob_mobility(g, b, eta)
    np.testing.assert_allclose(c2 * B @ B.T, 2 * kT / dt * M, rtol=0, atol=1e-11 * np.abs(M).max() * 2 * kT / dt)
    K = rigid.K_matrix(b.ref, b.offsets, b.quat)
    N = solve.body_mobility(M, K)
    Nh = N @ K.T @ np.linalg.solve(M, B)
    np.testing.assert_allclose(c2 * Nh @ Nh.T, 2 * kT / dt * N, rtol=0, atol=1e-10 * np.abs(N).max() * 2 * kT / dt)


def test_fluctuation_dissipation_sampled_from_oracle_noise():
    """Body velocities driven by the oracle's Philox stress alone have sample
    covariance (2 kT/dt) N within sampling error."""
    w, g, b = _setup(n=(6, 5, 5), n_bodies=1, near_wall=True)
    eta, kT, dt = 1.0, 1.0, 0.1
    Linv = _dense_stokes_inverse(g, eta)
    J = ib.J_matrix(g, b.positions()).toarray()
    M = solve.blob_mobility(g, b, eta)
    K = rigid.K_matrix(b.ref, b.offsets, b.quat)
    N = solve.body_mobility(M, K)
    T = N @ K.T @ np.linalg.solve(M, J @ Linv)      # U = T f_fluid
    DD = operators.tensor_divergence(g)
    n_s = 4000
    U = np.empty((n_s, 6))
    for s in range(n_s):
        f = noise.fluid_forcing(g, eta, kT, dt, seed=1234, step=s, DD=DD)
        U[s] = T @ f
    C = U.T @ U / n_s
    target = 2 * kT / dt * N
    sd = np.sqrt((np.outer(np.diag(target), np.diag(target)) + target ** 2) / n_s)
    assert np.all(np.abs(C - target) < 5 * sd)


def _N_of(g, b, eta):
    M = solve.blob_mobility(g, b, eta)
    return solve.body_mobility(M, rigid.K_matrix(b.ref, b.offsets, b.quat))


_DRIFT = {}


def _drift_case():
    """Two 12-blob shells in an 8x7x7 walled box, their blob mobility, and
    kT div_Q N from central differences of N in positions and lab-frame
    rotation angles (computed once per test session)."""
    if _DRIFT:
        return _DRIFT
    n = (8, 7, 7)
    g = Grid(n)
    shell = workloads.icosahedral_shell(12, 1.0)
    q = np.array([[2.2, 3.1, 2.0], [5.3, 3.9, 4.6]])
    quat = np.array([[0.9, 0.1, -0.3, 0.2], [0.6, -0.5, 0.4, 0.1]])
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    b = saddle.Bodies(np.vstack([shell, shell]), [0, 12, 24], q, quat)
    eta, kT = 1.0, 1.0
    op = solve.StokesOperator(g, eta)
    M = solve.blob_mobility(g, b, eta, op=op)
    nb = b.n_bodies
    eps = 1e-4
    div = np.zeros(6 * nb)
    for p in range(nb):
        for c in range(6):
            k = 6 * p + c
            qp, qm = q.copy(), q.copy()
            tp, tm = quat.copy(), quat.copy()
            if c < 3:
                qp[p, c] += eps; qm[p, c] -= eps
            else:
                e = np.zeros((nb, 3)); e[p, c - 3] = eps
                tp = rigid.rotate(quat, e); tm = rigid.rotate(quat, -e)
            Np = _N_of(g, b.moved(qp, tp), eta)
            Nm = _N_of(g, b.moved(qm, tm), eta)
            div += (Np[:, k] - Nm[:, k]) / (2 * eps)
    div *= kT
    _DRIFT.update(g=g, b=b, eta=eta, kT=kT, op=op, M=M, nb=nb, div=div, q=q, quat=quat)
    return _DRIFT


@pytest.mark.slow
def test_drift_expectation_by_basis_enumeration():
    """<U_drift> = sum_k U_drift(xi = e_k) equals kT div_Q N from central
    differences of N in positions and lab-frame rotation angles (Eq. DriDef,
    App. B); with the RFD terms dropped the drift would vanish."""
    c = _drift_case()
    g, b, eta, kT, op, M, nb, div = (c[k] for k in ("g", "b", "eta", "kT", "op", "M", "nb", "div"))
    Lp = rigid.body_length(b.ref, b.offsets)
    drift = np.zeros(6 * nb)
    for k in range(6 * nb):
        xi = np.zeros((nb, 6)); xi.flat[k] = 1.0
        t = sem.rfd_terms(g, b, eta, kT, xi[:, :3], xi[:, 3:], Lp, M=M, op=op)
        f = saddle.rhs(g, b, eta, F=-t["D_KT"], slip=t["D_K"] - t["D_J"] - t["D_S"], walls=False)
        drift += solve.constrained(g, b, eta, f, M=M, op=op)[-6 * nb:]
    assert np.linalg.norm(div) > 1e-3       # a real drift, which plain EM would miss
    np.testing.assert_allclose(drift, div, rtol=0, atol=2e-6 * np.linalg.norm(div))


@pytest.mark.slow
def test_sem_step_mean_drift_by_basis_enumeration():
    """The same expectation through oracle.sem.sem_step itself: with no
    forces, no fluid noise and the body normals injected as xi = e_k, the
    step's body velocity is the drift alone (its step-6 solve with force
    F - D^{K^T} and slip D^K - D^J - D^S), so sum_k U(e_k) = kT div_Q N
    (Eq. DriDef, App. B), and the step moves every body by dt U.  A sign slip
    in the step-6 assembly or a dropped RFD term fails this."""
    c = _drift_case()
    g, b, eta, kT, op, M, nb, div = (c[k] for k in ("g", "b", "eta", "kT", "op", "M", "nb", "div"))
    dt = 0.01
    mean_U = np.zeros(6 * nb)
    for k in range(6 * nb):
        xi = np.zeros((nb, 6)); xi.flat[k] = 1.0
        out = sem.sem_step(g, b, eta, kT, dt, {}, seed=0, step=0, normals=(xi[:, :3], xi[:, 3:]),
                           fluid_noise=False, op=op, M=M)
        np.testing.assert_allclose(out["q"] - b.q, dt * out["U"][:, :3], rtol=0, atol=1e-15)
        mean_U += out["U"].ravel()
    np.testing.assert_allclose(mean_U, div, rtol=0, atol=2e-6 * np.linalg.norm(div))
