"""Pins of the six-point kernel of Sec. III.B (oracle/kernel.py: phi6, dphi6)
and of spreading and interpolation with it.

The kernel's closed form in the oracle comes from our own solution of its
defining conditions.  Here the conditions are imposed directly: at random
shifts r the six weights are re-solved numerically from the five linear
conditions (even and odd sums 1/2, moments 1 and 3 zero, moment 2 equal to
K = 59/60 - sqrt(29)/20) and the quadratic one (sum of squares C), with
numpy's least squares and null space, not the closed form.  Independently
of any formula: the kernel is even, vanishes with its first three
derivatives at |x| = 3, and has three continuous derivatives at the
integers (the property K is chosen for); J = dV S^T holds near walls; linear
fields are interpolated exactly."""
import itertools

import numpy as np
import pytest

from oracle import Grid, kernel, ib

K = 59.0 / 60.0 - np.sqrt(29.0) / 20.0
J6 = np.arange(-2, 4)


def _candidates(r, C):
    """Both solutions of the defining conditions at shift r (the six weights
    phi(r - j), j = -2..3)."""
    d = r - J6
    A = np.array([(J6 % 2 == 0).astype(float), (J6 % 2 != 0).astype(float), d, d ** 2, d ** 3])
    b = np.array([0.5, 0.5, 0.0, K, 0.0])
    p = np.linalg.lstsq(A, b, rcond=None)[0]
    n = np.linalg.svd(A)[2][-1]
    qa, qb, qc = n @ n, 2 * p @ n, p @ p - C
    roots = (-qb + np.array([-1.0, 1.0]) * np.sqrt(max(qb * qb - 4 * qa * qc, 0.0))) / (2 * qa)
    return [p + t * n for t in roots]


def _solve_conditions(r, C, steps=400):
    """The branch through phi(-3) = 0 at r = 0, followed continuously: start at
    r = 0 with the solution whose phi(-3) vanishes, then at each small step in
    r take the solution nearest the previous one."""
    w = min(_candidates(0.0, C), key=lambda c: abs(c[5]))
    for rr in np.linspace(0.0, r, steps + 1)[1:]:
        w = min(_candidates(rr, C), key=lambda c: np.abs(c - w).max())
    return w


def test_constant_c_makes_the_support_close():
    """At r = 0 the conditions with C6 give phi(-3) = 0, phi even about 0."""
    w = _solve_conditions(0.0, kernel.C6)
    assert abs(w[5]) < 1e-12
    np.testing.assert_allclose(w[:5], w[4::-1], atol=1e-13)


def test_closed_form_solves_the_defining_conditions():
    rng = np.random.default_rng(3)
    for r in np.concatenate([rng.uniform(0, 1, 40), [0.0, 0.5, 1 - 1e-9]]):
        w = _solve_conditions(r, kernel.C6)
        got = kernel.phi6(r - J6)
        np.testing.assert_allclose(got, w, rtol=0, atol=2e-13)
        d = r - J6
        assert abs(got[J6 % 2 == 0].sum() - 0.5) < 1e-14 and abs(got[J6 % 2 != 0].sum() - 0.5) < 1e-14
        assert abs((d * got).sum()) < 1e-14 and abs((d ** 3 * got).sum()) < 1e-13
        assert abs((d ** 2 * got).sum() - K) < 1e-14 and abs((got ** 2).sum() - kernel.C6) < 1e-14


def test_even_support_and_smoothness():
    x = np.random.default_rng(4).uniform(-3.5, 3.5, 5000)
    np.testing.assert_allclose(kernel.phi6(x), kernel.phi6(-x), atol=1e-14)
    assert np.all(kernel.phi6(np.array([3.0, -3.0, 3.2, -4.0])) == 0.0)
    # one-sided derivatives 0..3 by quartic fits on either side of every
    # integer: they agree (three continuous derivatives); at |x| = 3 they are 0
    h = 1e-3
    xs = h * np.arange(1, 6)
    for m in range(-3, 4):
        cl = np.polyfit(-xs, kernel.phi6(m - xs), 4)
        cr = np.polyfit(xs, kernel.phi6(m + xs), 4)
        for q, tol in ((0, 1e-12), (1, 1e-9), (2, 2e-6), (3, 2e-3)):
            dl = np.polyval(np.polyder(cl, q), 0.0)
            dr = np.polyval(np.polyder(cr, q), 0.0)
            assert abs(dl - dr) < tol, (m, q, dl, dr)
            if abs(m) == 3:
                assert abs(dl) < tol and abs(dr) < tol


def test_derivative_against_finite_differences():
    x = np.random.default_rng(6).uniform(-2.99, 2.99, 3000)
    x = x[np.abs(x - np.round(x)) > 1e-4]
    e = 1e-6
    fd = (kernel.phi6(x + e) - kernel.phi6(x - e)) / (2 * e)
    np.testing.assert_allclose(kernel.dphi6(x), fd, atol=2e-9)


BCS = [p for p in itertools.product([False, True], repeat=3) if not all(p)]


@pytest.mark.parametrize("per", BCS)
def test_adjointness_near_walls_six_point(per):
    g = Grid((9, 8, 7), h=0.8, periodic=per, kernel=6)
    rng = np.random.default_rng(8)
    L = g.length()
    r = np.concatenate([rng.uniform(0, 0.9, (5, 3)), L - rng.uniform(0, 0.9, (5, 3)),
                        rng.uniform(0, L, (6, 3))])
    v = rng.standard_normal(g.N_f)
    lam = rng.standard_normal(3 * r.shape[0])
    lhs = np.dot(ib.interpolate(g, r, v), lam)
    rhs = g.dV * np.dot(v, ib.spread(g, r, lam))
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + np.linalg.norm(v) * np.linalg.norm(lam))


def test_six_point_interpolates_linear_and_cubic_fields_in_the_interior():
    """Away from walls the six-point kernel reproduces polynomials up to the
    third degree minus its (constant) second-moment correction: linear and
    odd-cubic fields about the blob exactly, a quadratic with the offset K h^2."""
    g = Grid((20, 20, 20), periodic=(True, True, False), kernel=6)
    rng = np.random.default_rng(11)
    r = np.column_stack([rng.uniform(0, 20, 30), rng.uniform(0, 20, 30), rng.uniform(6, 14, 30)])
    # v_z field (component 2 lives on z-faces at (i + 1/2, j + 1/2, k) h)
    e = g.face_ext(2)
    i, j, k = np.meshgrid(np.arange(e[0]), np.arange(e[1]), np.arange(e[2]), indexing="ij")
    zk = (k + 1.0) * g.h                         # compact index k -> physical face k + 1
    for c0, c1 in ((0.3, 1.7), (-2.0, 0.25)):
        vz = np.zeros(g.N_f)
        vz[g.face_offset(2):] = (c0 + c1 * zk).transpose(2, 1, 0).ravel()
        u = ib.interpolate(g, r, vz).reshape(-1, 3)[:, 2]
        np.testing.assert_allclose(u, c0 + c1 * r[:, 2], atol=1e-12)
    vz = np.zeros(g.N_f)
    vz[g.face_offset(2):] = (zk ** 2).transpose(2, 1, 0).ravel()
    u = ib.interpolate(g, r, vz).reshape(-1, 3)[:, 2]
    np.testing.assert_allclose(u, r[:, 2] ** 2 + K * g.h ** 2, atol=1e-11)
