"""Pins of the three-point kernel (moment conditions), of spreading and
interpolation (adjointness J = dV S^T near walls and corners, exact
interpolation of linear fields through the ghost treatment) and of binning."""
import itertools

import numpy as np
import pytest

from oracle import Grid, kernel, ib, binning


def test_kernel_moment_conditions():
    s = np.random.default_rng(0).uniform(-3, 3, 10000)
    j = np.arange(-6, 7)
    P = kernel.phi(s[:, None] - j[None, :])
    np.testing.assert_allclose(P.sum(axis=1), 1.0, atol=1e-15)
    np.testing.assert_allclose((P * (s[:, None] - j[None, :])).sum(axis=1), 0.0, atol=2e-15)
    np.testing.assert_allclose((P ** 2).sum(axis=1), 0.5, atol=1e-15)
    assert np.all(kernel.phi(np.array([1.5, -1.5, 2.0])) == 0.0)


def test_kernel_c1_and_derivative():
    for x0 in (0.5, 1.5, -0.5):
        e = 1e-7
        left = (kernel.phi(x0) - kernel.phi(x0 - e)) / e
        right = (kernel.phi(x0 + e) - kernel.phi(x0)) / e
        assert abs(left - right) < 1e-5
    np.testing.assert_allclose(kernel.dphi(np.array([0.5, 1.5, -0.5])), [-1.0, 0.0, 1.0], atol=1e-12)
    x = np.random.default_rng(2).uniform(-1.49, 1.49, 2000)
    x = x[(np.abs(np.abs(x) - 0.5) > 1e-3)]
    e = 1e-6
    fd = (kernel.phi(x + e) - kernel.phi(x - e)) / (2 * e)
    np.testing.assert_allclose(kernel.dphi(x), fd, atol=1e-7)


BCS = [p for p in itertools.product([False, True], repeat=3) if not all(p)]


@pytest.mark.parametrize("per", BCS)
def test_adjointness_near_walls_and_corners(per):
    wv = np.zeros((6, 3))
    g = Grid((7, 6, 5), h=0.8, periodic=per, wall_vel=wv)
    rng = np.random.default_rng(5)
    L = g.length()
    # blobs hugging walls, edges and corners, plus interior ones
    r = np.concatenate([rng.uniform(0, 0.9, (6, 3)), L - rng.uniform(0, 0.9, (6, 3)),
                        rng.uniform(0, L, (8, 3))])
    v = rng.standard_normal(g.N_f)
    lam = rng.standard_normal(3 * r.shape[0])
    lhs = np.dot(ib.interpolate(g, r, v), lam)
    rhs = g.dV * np.dot(v, ib.spread(g, r, lam))
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + np.linalg.norm(v) * np.linalg.norm(lam))


def test_interpolation_exact_for_linear_fields_with_moving_walls():
    """A linear velocity field that satisfies the wall conditions (tangential
    Couette-like shear matching moving walls, normal component vanishing on
    the walls' planes) is interpolated exactly, also within 1.5h of a wall:
    the kernel reproduces linear functions and the ghost treatment extends
    them linearly."""
    Lz = 6.0
    U = 0.8
    wv = np.zeros((6, 3)); wv[5, 0] = U; wv[4, 1] = -0.3    # top moves +x, bottom moves -y
    g = Grid((5, 4, 6), h=1.0, periodic=(True, True, False), wall_vel=wv)
    X = [g.face_coords(a) for a in range(3)]
    v = np.zeros(g.N_f)
    # v_x = U z/Lz ; v_y = -0.3 (1 - z/Lz) ; v_z = 0
    v[:g.n_face(0)] = U * X[0][:, 2] / Lz
    v[g.face_offset(1):g.face_offset(1) + g.n_face(1)] = -0.3 * (1 - X[1][:, 2] / Lz)
    rng = np.random.default_rng(9)
    r = np.concatenate([rng.uniform([0, 0, 0], [5, 4, 1.2], (10, 3)),
                        rng.uniform([0, 0, 4.8], [5, 4, 6], (10, 3))])
    Jv = ib.interpolate(g, r, v, with_walls=True).reshape(-1, 3)
    np.testing.assert_allclose(Jv[:, 0], U * r[:, 2] / Lz, atol=1e-14)
    np.testing.assert_allclose(Jv[:, 1], -0.3 * (1 - r[:, 2] / Lz), atol=1e-14)
    np.testing.assert_allclose(Jv[:, 2], 0.0, atol=1e-14)


def test_interpolation_exact_for_normal_linear_field():
    """v_z = c z (zero on the bottom wall plane) is reproduced near z = 0 by the
    odd reflection of the normal component."""
    g = Grid((4, 4, 8), h=1.0, periodic=(True, True, False))
    v = np.zeros(g.N_f)
    s = slice(g.face_offset(2), g.face_offset(2) + g.n_face(2))
    v[s] = 0.7 * g.face_coords(2)[:, 2]
    r = np.random.default_rng(4).uniform([0, 0, 0], [4, 4, 1.4], (12, 3))
    Jv = ib.interpolate(g, r, v).reshape(-1, 3)
    np.testing.assert_allclose(Jv[:, 2], 0.7 * r[:, 2], atol=1e-14)


def test_interpolation_reproduces_linear_interior_fields():
    g = Grid((9, 8, 7), h=0.5)
    rng = np.random.default_rng(1)
    coef = rng.standard_normal((3, 4))
    v = np.zeros(g.N_f)
    for a in range(3):
        X = g.face_coords(a)
        v[g.face_offset(a):g.face_offset(a) + g.n_face(a)] = coef[a, 0] + X @ coef[a, 1:]
    L = g.length()
    r = rng.uniform(1.6 * g.h, L - 1.6 * g.h, (20, 3))
    Jv = ib.interpolate(g, r, v).reshape(-1, 3)
    for a in range(3):
        np.testing.assert_allclose(Jv[:, a], coef[a, 0] + r @ coef[a, 1:], atol=1e-13)


def test_spread_total_force_and_sum_of_squares():
    """Away from walls S conserves force (partition of unity) and the
    spread weights of one blob satisfy sum w^2 = (1/2)^3 (kernel condition)."""
    g = Grid((10, 9, 8), h=1.0)
    rng = np.random.default_rng(11)
    r = rng.uniform(2.0, 6.0, (5, 3))
    lam = rng.standard_normal((5, 3))
    f = ib.spread(g, r, lam.ravel())
    for a in range(3):
        s = slice(g.face_offset(a), g.face_offset(a) + g.n_face(a))
        np.testing.assert_allclose(f[s].sum() * g.dV, lam[:, a].sum(), atol=1e-13)
    for a in range(3):
        _, coef, _ = ib.stencil(g, r[:1], a)
        np.testing.assert_allclose((coef ** 2).sum(), 0.125, atol=1e-15)


def test_binning_brute_force():
    g = Grid((5, 4, 3), h=1.5, periodic=(True, False, False))
    rng = np.random.default_rng(3)
    r = rng.uniform(-2, 9, (200, 3))
    r[:20] = np.floor(r[:20])         # exact cell boundaries
    perm, off = binning.counting_sort(g, r)
    assert off[0] == 0 and off[-1] == 200
    keys = binning.cell_keys(g, r)
    # brute force: cell c holds exactly the blobs with key c, in increasing id
    for c in range(g.N_c):
        assert list(perm[off[c]:off[c + 1]]) == [i for i in range(200) if keys[i] == c]
    for i in range(200):
        cx = int(np.floor(r[i, 0] / 1.5)) % 5
        cy = min(max(int(np.floor(r[i, 1] / 1.5)), 0), 3)
        cz = min(max(int(np.floor(r[i, 2] / 1.5)), 0), 2)
        assert keys[i] == cx + 5 * (cy + 4 * cz)
