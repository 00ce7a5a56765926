"""Pins of the oracle's free-slip walls (the Introduction's boundary conditions:
any combination of periodic, no-slip and free-slip walls along the axes).

Independently of the free-slip code:
  * the vector Laplacian equals a loop-built stencil whose ghost across a
    free-slip wall is +self (zero normal derivative of the tangential
    velocity) and -self across a no-slip wall;
  * the transform-based inverse inverts the assembled operator;
  * a channel with one free-slip wall carries the half-Poiseuille profile
    g z (2 L - z) / (2 eta) plus the ghost-reflection offset g h^2 / (8 eta)
    of the no-slip wall, exactly at the faces;
  * mirror images: a free-slip wall is a plane of mirror symmetry, so a body
    next to it moves exactly as the same body with its mirror image in a box
    doubled across that wall (periodic across two free-slip walls, no-slip at
    the far walls otherwise).  The doubled box uses only the periodic and
    no-slip code; the comparison covers the operators, the kernel folding,
    the moving-wall terms and the constrained solve;
  * spreading and interpolation stay adjoint (J = dV S^T) and interpolate a
    constant tangential field exactly next to a free-slip wall."""
import numpy as np
import pytest

from oracle import Grid, operators, solve, saddle, ib

T, F = True, False
# (periodic, free_slip) combinations with no velocity null mode
FS_CASES = [
    ((F, F, F), (T, T, F, F, F, F)),
    ((F, F, F), (F, T, T, F, F, T)),
    ((T, F, F), (F, F, T, T, F, T)),
    ((T, T, F), (F, F, F, F, T, F)),
    ((F, T, T), (T, F, F, F, F, F)),
]


def _loop_laplacian_fs(g):
    """Vector Laplacian by loops: Dirichlet zero at wall-normal boundary faces,
    ghost -self across a no-slip wall and +self across a free-slip wall along
    tangential axes, wrap on periodic axes."""
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
                                free = g.free_slip[2 * ax + (s > 0)]
                                L[me, me] += (1.0 if free else -1.0) / g.h ** 2
    return L


@pytest.mark.parametrize("per,fs", FS_CASES)
def test_vector_laplacian_free_slip_stencil(per, fs):
    g = Grid((4, 5, 3), h=1.3, periodic=per, free_slip=fs)
    L = operators.vector_laplacian(g).toarray()
    np.testing.assert_allclose(L, _loop_laplacian_fs(g), atol=1e-13)
    assert np.abs(L - L.T).max() == 0.0
    assert np.linalg.eigvalsh(L).max() < 0.0


def test_velocity_null_mode_is_rejected():
    with pytest.raises(ValueError):
        Grid((4, 4, 4), periodic=(F, T, T), free_slip=(T, T, F, F, F, F))
    with pytest.raises(ValueError):
        Grid((4, 4, 4), periodic=(T, T, F), free_slip=(F, F, F, F, T, T))
    with pytest.raises(ValueError):                       # a free-slip wall cannot move
        wv = np.zeros((6, 3)); wv[5, 0] = 1.0
        Grid((4, 4, 4), periodic=(T, T, F), free_slip=(F, F, F, F, F, T), wall_vel=wv)


@pytest.mark.parametrize("per,fs", FS_CASES)
def test_exact_laplacian_inverse_free_slip(per, fs):
    g = Grid((5, 4, 6), h=1.1, periodic=per, free_slip=fs)
    L = operators.vector_laplacian(g)
    rng = np.random.default_rng(1)
    for a in range(3):
        s = slice(g.face_offset(a), g.face_offset(a) + g.n_face(a))
        f = rng.standard_normal(g.n_face(a))
        u = solve.laplacian_solve(g, a, f)
        np.testing.assert_allclose(L[s, s] @ u, f, atol=1e-12)


@pytest.mark.parametrize("top_free", [True, False])
def test_half_poiseuille_closed_form(top_free):
    """Body force g along x between a no-slip and a free-slip wall (z):
    v_x = g z (2 L - z) / (2 eta) + g h^2 / (8 eta), z measured from the
    no-slip wall, exact at the faces (z = (k + 1/2) h).  The profile is even
    about the free-slip wall, so its even ghost is exact there; the constant
    is the offset that makes the no-slip ghost (odd about the wall) exact for
    a quadratic, as in plane Poiseuille flow.  y walls free-slip on both
    sides leave the flow uniform in y."""
    gx, eta = 0.3, 1.3
    fs = (F, F, T, T, not top_free, top_free)
    g = Grid((4, 3, 9), h=0.6, periodic=(T, F, F), free_slip=fs)
    f = np.zeros(g.N_f); f[:g.n_face(0)] = gx
    v, pi = solve.stokes(g, eta, f)
    z = g.face_coords(0)[:, 2]
    Lz = g.length()[2]
    zz = z if top_free else Lz - z            # distance from the no-slip wall
    exact = gx * zz * (2 * Lz - zz) / (2 * eta) + gx * g.h ** 2 / (8 * eta)
    np.testing.assert_allclose(v[:g.n_face(0)], exact, rtol=1e-12, atol=1e-13)
    assert np.abs(v[g.n_face(0):]).max() < 1e-12


def _shell12(R):
    gr = (1 + 5 ** 0.5) / 2
    v = []
    for s1 in (-1, 1):
        for s2 in (-1, 1):
            v += [(0, s1, s2 * gr), (s1, s2 * gr, 0), (s2 * gr, 0, s1)]
    v = np.array(v, dtype=np.float64)
    return R * v / np.linalg.norm(v, axis=1, keepdims=True)


class _BodyResponse:
    """Body velocities (n_b * 6) for forces/torques FT, bodies given by lab
    frame blob offsets (identity orientation); the blob mobility is formed
    once per system."""

    def __init__(self, g, ref_list, q_list, eta):
        ref = np.concatenate(ref_list)
        offs = np.concatenate([[0], np.cumsum([r.shape[0] for r in ref_list])])
        quat = np.tile([1.0, 0, 0, 0], (len(q_list), 1))
        self.g, self.eta, self.nb = g, eta, len(q_list)
        self.b = saddle.Bodies(ref, offs, np.array(q_list), quat)
        self.op = solve.StokesOperator(g, eta)
        self.M = solve.blob_mobility(g, self.b, eta, op=self.op)

    def __call__(self, FT):
        f = saddle.rhs(self.g, self.b, self.eta, F=FT)
        x = solve.constrained(self.g, self.b, self.eta, f, M=self.M, op=self.op)
        return x[-6 * self.nb:]


@pytest.mark.parametrize("ax,both,kernel", [(2, True, 3), (2, False, 3), (1, False, 3), (2, False, 6)])
def test_free_slip_wall_equals_mirror_image(ax, both, kernel):
    eta = 1.1
    n = [7, 6, 6] if kernel == 3 else [12, 12, 10]
    per = [True, False, False]
    per[ax] = False
    H = n[ax] * 1.0
    fs = [F] * 6
    fs[2 * ax] = True
    fs[2 * ax + 1] = both
    wv = np.zeros((6, 3))
    if not both:
        t = (ax + 1) % 3                        # the far (no-slip) wall moves tangentially
        wv[2 * ax + 1, t] = 0.4
    g = Grid(n, periodic=per, free_slip=fs, wall_vel=wv, kernel=kernel)
    R = 1.0 if kernel == 3 else 2.0
    ref = _shell12(R)
    q = np.array([3.4, 2.9, 3.1]) if kernel == 3 else np.array([6.2, 5.7, 5.3])
    q[ax] = 1.55 if kernel == 3 else 2.6      # kernel points reach across the free-slip wall
    Mr = np.ones(3); Mr[ax] = -1.0
    # doubled box across the free-slip wall
    n2 = list(n); n2[ax] = 2 * n[ax]
    per2 = list(per)
    wv2 = np.zeros((6, 3))
    shift = 0.0
    if both:
        per2[ax] = True
    else:
        shift = H                               # the original half is the upper one
        wv2[2 * ax + 1] = wv[2 * ax + 1]
        wv2[2 * ax] = wv[2 * ax + 1]            # tangential wall velocity is even
    g2 = Grid(n2, periodic=per2, wall_vel=wv2, kernel=kernel)
    q_orig = q.copy(); q_orig[ax] += shift
    q_img = q.copy(); q_img[ax] = shift - q[ax]
    if both:
        q_img[ax] %= 2 * H
    ref_img = ref * Mr
    resp = _BodyResponse(g, [ref], [q], eta)
    resp2 = _BodyResponse(g2, [ref, ref_img], [q_orig, q_img], eta)
    for k in range(7):
        FT = np.zeros(6)
        if k < 6:
            FT[k] = 1.0
        FT_img = np.concatenate([Mr * FT[:3], -Mr * FT[3:]])
        U = resp(FT)
        U2 = resp2(np.concatenate([FT, FT_img]))
        scale = np.abs(U2).max()
        np.testing.assert_allclose(U, U2[:6], rtol=0, atol=1e-10 * scale)
        np.testing.assert_allclose(U2[6:9], Mr * U2[:3], rtol=0, atol=1e-10 * scale)
        np.testing.assert_allclose(U2[9:], -Mr * U2[3:6], rtol=0, atol=1e-10 * scale)


@pytest.mark.parametrize("kernel", [3, 6])
@pytest.mark.parametrize("per,fs", FS_CASES)
def test_adjointness_near_free_slip_walls(per, fs, kernel):
    g = Grid((9, 8, 7), h=0.8, periodic=per, free_slip=fs, kernel=kernel)
    rng = np.random.default_rng(8)
    L = g.length()
    r = np.concatenate([rng.uniform(0, 0.9, (5, 3)), L - rng.uniform(0, 0.9, (5, 3)),
                        rng.uniform(0, L, (6, 3))])
    v = rng.standard_normal(g.N_f)
    lam = rng.standard_normal(3 * r.shape[0])
    lhs = np.dot(ib.interpolate(g, r, v), lam)
    rhs = g.dV * np.dot(v, ib.spread(g, r, lam))
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + np.linalg.norm(v) * np.linalg.norm(lam))


@pytest.mark.parametrize("kernel", [3, 6])
def test_constant_tangential_field_next_to_free_slip_wall(kernel):
    """Partition of unity survives the even mirror: a constant tangential
    velocity is interpolated exactly right next to a free-slip wall (the odd
    mirror of a no-slip wall would not)."""
    g = Grid((10, 10, 12), periodic=(T, T, F), free_slip=(F, F, F, F, T, F), kernel=kernel)
    rng = np.random.default_rng(5)
    r = np.column_stack([rng.uniform(0, 10, 20), rng.uniform(0, 10, 20), rng.uniform(0.0, 1.0, 20)])
    for a, c in ((0, 0.7), (1, -1.3)):
        v = np.zeros(g.N_f)
        v[g.face_offset(a):g.face_offset(a) + g.n_face(a)] = c
        u = ib.interpolate(g, r, v).reshape(-1, 3)
        np.testing.assert_allclose(u[:, a], c, atol=1e-13)
    gn = Grid((10, 10, 12), periodic=(T, T, F), kernel=kernel)
    v = np.zeros(gn.N_f); v[:gn.n_face(0)] = 0.7
    assert np.abs(ib.interpolate(gn, r, v).reshape(-1, 3)[:, 0] - 0.7).max() > 0.05
