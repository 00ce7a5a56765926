"""Immersed-boundary spreading S and interpolation J of Sec. III.B with the
three-point or the six-point kernel (Grid.kernel), including the wall
treatment.

  (J v)_i = sum_alpha delta_h(x_alpha - r_i) v(x_alpha) dV      (= sum w v)
  (S l)_alpha = (1/dV) sum_i delta_h(x_alpha - r_i) l_i dV     (= sum w l / dV)

with w = phi(dx/h) phi(dy/h) phi(dz/h).  For velocity component a the kernel
points along each axis are the 3 (or 6) grid points nearest to the blob on
that component's staggered grid (faces along a, cell centres otherwise).

Walls (our reading of the ghost-point treatment the paper cites): a point on a
wall-normal boundary face holds the prescribed normal velocity (zero) and is
dropped; a point beyond a wall is a ghost that mirrors onto the interior point
reflected about the wall with coefficient -1; a tangential ghost also carries
the affine part 2 u_w of the ghost-reflection boundary condition.  Across a
free-slip wall a tangential ghost mirrors with coefficient +1 (the tangential
velocity is even about the wall) and carries no affine part; the normal
component stays odd.  When a
point is a ghost along several axes the reflections are applied in x, y, z
order.  A point whose mirror is not an unknown is dropped.  S and J use the
same folded weights, so J = dV S^T exactly (Sec. III.B).
"""
import numpy as np

from .grid import Grid
from .kernel import kernel


def _axis_points(g: Grid, a, ax, x, deriv=False):
    """For coordinates x (N,) along axis ax of component a: the kernel's
    candidate points per blob -> (index p (N,k), weight (N,k)) and, with
    deriv, the weights' derivative with respect to x."""
    phi, dphi, k, first = kernel(g.kernel)
    o = 0.0 if ax == a else 0.5
    s = x / g.h - o
    p = first(s)[:, None] + np.arange(k)[None, :]
    w = phi(s[:, None] - p)
    if deriv:
        return p, w, dphi(s[:, None] - p) / g.h
    return p, w


def _fold(g: Grid, a, ax, p):
    """Map physical index p along ax to (compact index, sign, tangential-ghost
    wall id or -1, keep mask)."""
    n = g.n[ax]
    if g.periodic[ax]:
        return np.mod(p, n), np.ones(p.shape), np.full(p.shape, -1), np.ones(p.shape, dtype=bool)
    if ax == a:                       # normal component along its own axis: faces 0..n
        comp = p - 1
        sign = np.ones(p.shape)
        keep = (p >= 1) & (p <= n - 1)
        lo = p < 0
        hi = p > n
        m_lo = -p
        m_hi = 2 * n - p
        comp = np.where(lo, m_lo - 1, np.where(hi, m_hi - 1, comp))
        sign = np.where(lo | hi, -1.0, sign)
        keep = keep | (lo & (m_lo >= 1) & (m_lo <= n - 1)) | (hi & (m_hi >= 1) & (m_hi <= n - 1))
        return comp, sign, np.full(p.shape, -1), keep
    # tangential: cell-centred points 0..n-1, ghosts reflect about the wall
    # (odd at a no-slip wall, even at a free-slip wall)
    lo = p < 0
    hi = p > n - 1
    comp = np.where(lo, -1 - p, np.where(hi, 2 * n - 1 - p, p))
    s_lo = 1.0 if g.free_slip[2 * ax] else -1.0
    s_hi = 1.0 if g.free_slip[2 * ax + 1] else -1.0
    sign = np.where(lo, s_lo, np.where(hi, s_hi, 1.0))
    wall = np.where(lo & (s_lo < 0), 2 * ax, np.where(hi & (s_hi < 0), 2 * ax + 1, -1))
    keep = (comp >= 0) & (comp <= n - 1)
    return comp, sign, wall, keep


def stencil(g: Grid, r, a):
    """Folded k^3-point stencils (k = Grid.kernel) of blobs r (N,3) for
    velocity component a.

    Returns (idx (N,k^3) flat index within the component, coef (N,k^3) folded
    weight, affine (N,k^3) ghost boundary value times weight)."""
    r = np.asarray(r, dtype=np.float64).reshape(-1, 3)
    N = r.shape[0]
    ext = g.face_ext(a)
    k = g.kernel
    per_axis = []
    for ax in range(3):
        p, w = _axis_points(g, a, ax, r[:, ax])
        comp, sign, wall, keep = _fold(g, a, ax, p)
        per_axis.append((comp, sign, wall, keep, w))
    idx = np.zeros((N, k ** 3), dtype=np.int64)
    coef = np.zeros((N, k ** 3))
    aff = np.zeros((N, k ** 3))
    t = 0
    for dz in range(k):
        for dy in range(k):
            for dx in range(k):
                d = (dx, dy, dz)
                comps = [per_axis[ax][0][:, d[ax]] for ax in range(3)]
                keep = np.ones(N, dtype=bool)
                w = np.ones(N)
                sgn = np.ones(N)
                affv = np.zeros(N)
                for ax in range(3):
                    comp, sign, wall, kp, ww = per_axis[ax]
                    keep &= kp[:, d[ax]]
                    w = w * ww[:, d[ax]]
                    folded = sign[:, d[ax]] < 0
                    wid = wall[:, d[ax]]
                    uw = np.where(wid >= 0, g.wall_vel[np.maximum(wid, 0), a], 0.0)
                    affv = affv + np.where(folded, sgn * 2.0 * uw, 0.0)
                    sgn = np.where(folded, -sgn, sgn)
                idx[:, t] = np.where(keep, g.flat(ext, *comps), 0)
                coef[:, t] = np.where(keep, w * sgn, 0.0)
                aff[:, t] = np.where(keep, w * affv, 0.0)
                t += 1
    return idx, coef, aff


def interpolate(g: Grid, r, v, with_walls=False):
    """J v: (N_bl*3,) blob velocities from face velocities v (N_f,).  With
    ``with_walls`` the affine ghost values of moving walls are included."""
    r = np.asarray(r).reshape(-1, 3)
    out = np.zeros((r.shape[0], 3))
    for a in range(3):
        idx, coef, aff = stencil(g, r, a)
        va = v[g.face_offset(a):g.face_offset(a) + g.n_face(a)]
        out[:, a] = np.sum(coef * va[idx], axis=1)
        if with_walls:
            out[:, a] += np.sum(aff, axis=1)
    return out.ravel()


def interpolate_wall_part(g: Grid, r):
    """The affine part of J: blob velocities induced by moving-wall ghosts."""
    r = np.asarray(r).reshape(-1, 3)
    out = np.zeros((r.shape[0], 3))
    for a in range(3):
        _, _, aff = stencil(g, r, a)
        out[:, a] = np.sum(aff, axis=1)
    return out.ravel()


def spread(g: Grid, r, lam):
    """S lambda: face force densities (N_f,) from blob forces lambda (N_bl*3,)."""
    r = np.asarray(r).reshape(-1, 3)
    lam = np.asarray(lam).reshape(-1, 3)
    out = np.zeros(g.N_f)
    for a in range(3):
        idx, coef, _ = stencil(g, r, a)
        part = np.zeros(g.n_face(a))
        np.add.at(part, idx.ravel(), (coef * lam[:, a:a + 1]).ravel() / g.dV)
        out[g.face_offset(a):g.face_offset(a) + g.n_face(a)] = part
    return out


def J_matrix(g: Grid, r):
    """J as a dense (3 N_bl, N_f) array (tiny problems only)."""
    import scipy.sparse as sp
    r = np.asarray(r).reshape(-1, 3)
    rows, cols, vals = [], [], []
    for a in range(3):
        idx, coef, _ = stencil(g, r, a)
        rr = np.repeat(3 * np.arange(r.shape[0]) + a, g.kernel ** 3)
        rows.append(rr); cols.append(idx.ravel() + g.face_offset(a)); vals.append(coef.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(3 * r.shape[0], g.N_f))


def S_matrix(g: Grid, r):
    """S = J^T / dV as a sparse (N_f, 3 N_bl) matrix, built by spreading unit
    blob forces one at a time."""
    import scipy.sparse as sp
    r = np.asarray(r).reshape(-1, 3)
    cols = []
    for c in range(3 * r.shape[0]):
        e = np.zeros(3 * r.shape[0]); e[c] = 1.0
        cols.append(sp.csr_matrix(spread(g, r, e)).T)
    return sp.hstack(cols).tocsr() if cols else sp.csr_matrix((g.N_f, 0))


def stencil_grad(g: Grid, r, a):
    """Derivatives of the folded weights of component a with respect to the
    blob position: (idx (N,k^3), coef (N,k^3), dcoef (N,k^3,3)) where
    dcoef[..., b] = d coef / d r_b = phi'(s_b - p_b)/h * prod_{c != b} phi * sign."""
    r = np.asarray(r, dtype=np.float64).reshape(-1, 3)
    N = r.shape[0]
    ext = g.face_ext(a)
    k = g.kernel
    per_axis = []
    for ax in range(3):
        p, w, dw = _axis_points(g, a, ax, r[:, ax], deriv=True)
        comp, sign, wall, keep = _fold(g, a, ax, p)
        per_axis.append((comp, sign, keep, w, dw))
    idx = np.zeros((N, k ** 3), dtype=np.int64)
    coef = np.zeros((N, k ** 3))
    dcoef = np.zeros((N, k ** 3, 3))
    t = 0
    for dz in range(k):
        for dy in range(k):
            for dx in range(k):
                d = (dx, dy, dz)
                comps = [per_axis[ax][0][:, d[ax]] for ax in range(3)]
                keep = np.ones(N, dtype=bool)
                sgn = np.ones(N)
                ws = [per_axis[ax][3][:, d[ax]] for ax in range(3)]
                dws = [per_axis[ax][4][:, d[ax]] for ax in range(3)]
                for ax in range(3):
                    keep &= per_axis[ax][2][:, d[ax]]
                    sgn = sgn * per_axis[ax][1][:, d[ax]]
                idx[:, t] = np.where(keep, g.flat(ext, *comps), 0)
                coef[:, t] = np.where(keep, ws[0] * ws[1] * ws[2] * sgn, 0.0)
                for b in range(3):
                    prod = dws[b] * ws[(b + 1) % 3] * ws[(b + 2) % 3]
                    dcoef[:, t, b] = np.where(keep, prod * sgn, 0.0)
                t += 1
    return idx, coef, dcoef


def interpolate_derivative(g: Grid, r, f):
    """D(f)[i, a, b] = sum over the kernel points of d w_a / d r_{i,b} * f_a:
    the derivative of (J f)_{ia} with respect to blob position r_i."""
    r = np.asarray(r).reshape(-1, 3)
    out = np.zeros((r.shape[0], 3, 3))
    for a in range(3):
        idx, _, dcoef = stencil_grad(g, r, a)
        fa = f[g.face_offset(a):g.face_offset(a) + g.n_face(a)]
        out[:, a, :] = np.einsum("ntb,nt->nb", dcoef, fa[idx])
    return out
