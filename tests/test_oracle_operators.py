"""Pins of the oracle's fluid operators (Sec. III.A) against independent
loop-based stencils, exact discrete identities and analytic channel flows."""
import itertools

import numpy as np
import pytest

from oracle import Grid, operators, solve, saddle

BCS = list(itertools.product([False, True], repeat=3))[:-1]   # at least one wall axis


def _loop_gradient(g):
    """(G pi)_face = (pi_right - pi_left)/h on unknown faces, by loops."""
    rows = []
    for a in range(3):
        ext = g.face_ext(a)
        for k in range(ext[2]):
            for j in range(ext[1]):
                for i in range(ext[0]):
                    c = [i, j, k]
                    p = g.face_phys(a, c[a])
                    right = list(c); right[a] = p % g.n[a]
                    left = list(c); left[a] = (p - 1) % g.n[a]
                    row = np.zeros(g.N_c)
                    row[g.flat(g.n, *right)] += 1.0 / g.h
                    row[g.flat(g.n, *left)] -= 1.0 / g.h
                    rows.append(row)
    return np.array(rows)


def _loop_laplacian(g):
    """Ghost-reflection vector Laplacian, component by component, by loops:
    Dirichlet zero at wall-normal boundary faces, ghost u_{-1} = -u_0 across
    walls along tangential axes, wrap on periodic axes."""
    L = np.zeros((g.N_f, g.N_f))
    for a in range(3):
        ext = g.face_ext(a)
        off = g.face_offset(a)
        for k in range(ext[2]):
            for j in range(ext[1]):
                for i in range(ext[0]):
                    c = [i, j, k]
                    me = off + g.flat(ext, *c)
                    for ax in range(3):
                        L[me, me] -= 2.0 / g.h ** 2
                        for s in (-1, 1):
                            nb = list(c); nb[ax] += s
                            if g.periodic[ax]:
                                nb[ax] %= ext[ax]
                                L[me, off + g.flat(ext, *nb)] += 1.0 / g.h ** 2
                            elif 0 <= nb[ax] < ext[ax]:
                                L[me, off + g.flat(ext, *nb)] += 1.0 / g.h ** 2
                            elif ax != a:
                                L[me, me] -= 1.0 / g.h ** 2    # ghost = -self
                            # ax == a at a boundary face: Dirichlet zero
    return L


@pytest.mark.parametrize("per", BCS)
def test_gradient_is_minus_divergence_transpose(per):
    g = Grid((4, 3, 5), h=0.7, periodic=per)
    G = operators.gradient(g).toarray()
    np.testing.assert_allclose(G, _loop_gradient(g), atol=1e-14)
    D = operators.divergence(g).toarray()
    np.testing.assert_array_equal(G, -D.T)


@pytest.mark.parametrize("per", BCS)
def test_vector_laplacian_is_ghost_reflection_stencil(per):
    g = Grid((4, 5, 3), h=1.3, periodic=per)
    L = operators.vector_laplacian(g).toarray()
    np.testing.assert_allclose(L, _loop_laplacian(g), atol=1e-13)
    assert np.abs(L - L.T).max() == 0.0
    assert np.linalg.eigvalsh(L).max() < 0.0


def test_scalar_laplacian_is_neumann_7pt():
    g = Grid((4, 3, 5), periodic=(True, False, False))
    DG = (operators.divergence(g) @ operators.gradient(g)).toarray()
    ref = np.zeros_like(DG)
    for k in range(5):
        for j in range(3):
            for i in range(4):
                me = g.flat(g.n, i, j, k)
                for ax in range(3):
                    for s in (-1, 1):
                        nb = [i, j, k]; nb[ax] += s
                        if g.periodic[ax]:
                            nb[ax] %= g.n[ax]
                        elif not (0 <= nb[ax] < g.n[ax]):
                            continue       # zero flux through walls
                        ref[me, me] -= 1.0
                        ref[me, g.flat(g.n, *nb)] += 1.0
    np.testing.assert_allclose(DG, ref, atol=1e-14)


@pytest.mark.parametrize("per", [(False, False, False), (True, False, False), (True, True, False)])
def test_divergence_of_discrete_curl_vanishes(per):
    """v = curl A with A on edges (tangential A vanishing on walls) is exactly
    divergence free."""
    g = Grid((5, 4, 6), h=0.9, periodic=per)
    L = g.length()

    freq = (1.3, 0.7, 0.9)
    phase = (0.4, -0.2, 1.1)

    def A(c, x):
        val = 0.3 * (c + 1)
        for b in range(3):
            # periodic axes: functions of period L_b; wall axes: arbitrary
            k = 2 * np.pi / L[b] if per[b] else freq[b]
            val = val * (1.2 + np.sin(k * x[..., b] + phase[b] + c))
            if b != c and not per[b]:
                val = val * np.sin(np.pi * x[..., b] / L[b])   # tangential A vanishes on walls
        return val

    h = g.h
    v = np.zeros(g.N_f)
    for a in range(3):
        b1, b2 = (a + 1) % 3, (a + 2) % 3
        X = g.face_coords(a)
        # v_a = d_b1 A_b2 - d_b2 A_b1 with A_b2 on edges at +-h/2 along b1
        e1 = np.zeros(3); e1[b1] = h / 2
        e2 = np.zeros(3); e2[b2] = h / 2
        va = (A(b2, X + e1) - A(b2, X - e1)) / h - (A(b1, X + e2) - A(b1, X - e2)) / h
        v[g.face_offset(a):g.face_offset(a) + g.n_face(a)] = va
    Dv = operators.divergence(g) @ v
    assert np.abs(Dv).max() < 1e-13 * max(1.0, np.abs(v).max())


def test_couette_is_exact():
    """x,y periodic, z walls, top wall moving at U along x: v_x = U z / L_z at
    z = (k + 1/2) h and constant pressure solve the discrete system exactly."""
    U, eta = 0.75, 1.7
    wv = np.zeros((6, 3)); wv[5, 0] = U
    g = Grid((6, 5, 8), h=0.5, periodic=(True, True, False), wall_vel=wv)
    b = saddle.Bodies(np.zeros((0, 3)), [0], np.zeros((0, 3)), np.zeros((0, 4)))
    x = np.zeros(g.N_f + g.N_c)
    z = g.face_coords(0)[:, 2]
    x[:g.n_face(0)] = U * z / g.length()[2]
    f = saddle.rhs(g, b, eta)
    r = saddle.apply(g, b, eta, x) - f
    assert np.abs(r).max() < 1e-12
    v, pi = solve.stokes(g, eta, f[:g.N_f])
    np.testing.assert_allclose(v[:g.n_face(0)], x[:g.n_face(0)], atol=1e-12)
    assert np.abs(v[g.n_face(0):]).max() < 1e-12


def test_poiseuille_closed_form():
    """Static walls in z, periodic x, y, body force g along x:
    v_x = g z (L - z)/(2 eta) + g h^2/(8 eta) at z = (k + 1/2) h."""
    gx, eta = 0.3, 1.3
    g = Grid((4, 3, 10), h=0.6, periodic=(True, True, False))
    f = np.zeros(g.N_f); f[:g.n_face(0)] = gx
    v, pi = solve.stokes(g, eta, f)
    z = g.face_coords(0)[:, 2]
    Lz = g.length()[2]
    exact = gx * z * (Lz - z) / (2 * eta) + gx * g.h ** 2 / (8 * eta)
    np.testing.assert_allclose(v[:g.n_face(0)], exact, rtol=1e-12, atol=1e-13)
    D = operators.divergence(g)
    assert np.abs(D @ v).max() < 1e-13


@pytest.mark.parametrize("per", [(False, False, False), (True, False, False), (False, True, True)])
def test_stokes_solver_matches_direct_and_is_divergence_free(per):
    g = Grid((6, 5, 4), h=0.8, periodic=per)
    rng = np.random.default_rng(3)
    f = rng.standard_normal(g.N_f)
    fp = rng.standard_normal(g.N_c); fp -= fp.mean()
    b = saddle.Bodies(np.zeros((0, 3)), [0], np.zeros((0, 3)), np.zeros((0, 4)))
    x_dir = solve.direct(g, b, 1.4, np.concatenate([f, fp]))
    v, pi = solve.stokes(g, 1.4, f, fp)
    np.testing.assert_allclose(np.concatenate([v, pi]), x_dir, rtol=0, atol=1e-12 * np.abs(x_dir).max())
    np.testing.assert_allclose(-(operators.divergence(g) @ v), fp, atol=1e-12)


@pytest.mark.parametrize("per", BCS)
def test_exact_laplacian_inverse(per):
    g = Grid((5, 4, 6), h=1.1, periodic=per)
    L = operators.vector_laplacian(g)
    rng = np.random.default_rng(1)
    for a in range(3):
        s = slice(g.face_offset(a), g.face_offset(a) + g.n_face(a))
        f = rng.standard_normal(g.n_face(a))
        u = solve.laplacian_solve(g, a, f)
        np.testing.assert_allclose((L[s, s] @ u), f, atol=1e-12)
