"""Solutions of the discrete Stokes and constrained systems.

The method's Krylov solve reaches (to its tolerance) the exact solution of
Eqs. (LangevinD1-D4), so the oracle computes that solution by other means:

  * ``direct``: sparse LU of the saddle matrix bordered by the pressure gauge
    sum(pi) = 0 (tiny grids only);
  * ``stokes``: the discrete Stokes solution operator of Sec. III.A.  The
    vector Laplacian acts on each velocity component separately and is
    diagonalised by sine and cosine transforms (DST-I along the component's own
    wall axis; along a tangential wall axis DST-II between no-slip walls, DCT-II
    between free-slip walls, DST-IV / DCT-IV with one of each) and Fourier
    transforms on periodic axes,
    so (-eta LL)^{-1} is applied exactly; the pressure then solves the Schur
    complement G^T (-eta LL)^{-1} G pi = ... by conjugate gradients to 1e-14;
  * ``constrained``: the reduced form of Sec. III.C, Eq. (incompleteN),
    with the blob mobility M = J L^{-1} S and N = (K^T M^{-1} K)^{-1} formed
    densely, column by column, from Stokes solves.
"""
import numpy as np
import scipy.fft as sfft
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .grid import Grid
from . import operators, ib, rigid, saddle


# ---------------------------------------------------------------- direct
def direct(g: Grid, b, eta, f):
    A = saddle.assemble(g, b, eta).tocsc()
    o = saddle.layout(g, b)
    n = A.shape[0]
    e = np.zeros((n, 1)); e[o[3]:o[4], 0] = 1.0
    B = sp.bmat([[A, sp.csc_matrix(e)], [sp.csc_matrix(e.T), None]], format="csc")
    rhs = np.concatenate([f, [0.0]])
    x = spla.spsolve(B, rhs)
    return x[:n]


# ------------------------------------------------- exact Laplacian inverse
def _axis_modes(g: Grid, a, ax):
    """Transform kind and eigenvalues of the 1D second difference of component
    a along axis ax.  Along a tangential wall axis the ghost is odd at a
    no-slip wall and even at a free-slip wall."""
    n, h = g.n[ax], g.h
    if g.periodic[ax]:
        k = np.arange(n)
        return "fft", -4.0 * np.sin(np.pi * k / n) ** 2 / h ** 2
    if ax == a:
        k = np.arange(1, n)
        return "dst1", -4.0 * np.sin(np.pi * k / (2 * n)) ** 2 / h ** 2
    even_lo, even_hi = g.free_slip[2 * ax], g.free_slip[2 * ax + 1]
    if not even_lo and not even_hi:
        k = np.arange(1, n + 1)
        return "dst2", -4.0 * np.sin(np.pi * k / (2 * n)) ** 2 / h ** 2
    if even_lo and even_hi:
        k = np.arange(n)
        return "dct2", -4.0 * np.sin(np.pi * k / (2 * n)) ** 2 / h ** 2
    k = np.arange(n) + 0.5
    return ("dst4" if even_hi else "dct4"), -4.0 * np.sin(np.pi * k / (2 * n)) ** 2 / h ** 2


_FWD = {"dst1": (sfft.dst, 1), "dst2": (sfft.dst, 2), "dst4": (sfft.dst, 4),
        "dct2": (sfft.dct, 2), "dct4": (sfft.dct, 4)}
_INV = {"dst1": (sfft.idst, 1), "dst2": (sfft.idst, 2), "dst4": (sfft.idst, 4),
        "dct2": (sfft.idct, 2), "dct4": (sfft.idct, 4)}


def laplacian_solve(g: Grid, a, f):
    """Solve LL_a u = f for component a; f has shape (..., n_face(a))."""
    ext = g.face_ext(a)
    lead = f.shape[:-1]
    arr = f.reshape(lead + (ext[2], ext[1], ext[0]))
    nd = arr.ndim
    axis_of = {0: nd - 1, 1: nd - 2, 2: nd - 3}
    kinds, eig = [], 0.0
    for ax in range(3):
        kind, lam = _axis_modes(g, a, ax)
        kinds.append(kind)
        shape = [1] * 3
        shape[2 - ax] = lam.size
        eig = eig + lam.reshape(shape)
    t = arr.astype(np.float64)
    for ax in range(3):
        if kinds[ax] in _FWD:
            fn, typ = _FWD[kinds[ax]]
            t = fn(t, type=typ, axis=axis_of[ax], norm="ortho")
    per = [ax for ax in range(3) if kinds[ax] == "fft"]
    if per:
        t = sfft.fftn(t, axes=[axis_of[ax] for ax in per])
    t = t / eig
    if per:
        t = sfft.ifftn(t, axes=[axis_of[ax] for ax in per]).real
    for ax in range(3):
        if kinds[ax] in _INV:
            fn, typ = _INV[kinds[ax]]
            t = fn(t, type=typ, axis=axis_of[ax], norm="ortho")
    return t.reshape(lead + (g.n_face(a),))


def viscous_solve(g: Grid, eta, f):
    """(-eta LL)^{-1} f for f of shape (m, N_f)."""
    out = np.empty_like(f)
    for a in range(3):
        s = slice(g.face_offset(a), g.face_offset(a) + g.n_face(a))
        out[..., s] = -laplacian_solve(g, a, f[..., s]) / eta
    return out


# ------------------------------------------------------------ Stokes solve
class StokesOperator:
    def __init__(self, g: Grid, eta):
        self.g, self.eta = g, eta
        self.G = operators.gradient(g)
        self.GT = self.G.T.tocsr()

    def solve(self, f_v, f_pi=None, tol=1e-14, maxiter=5000):
        """(v, pi) with -eta LL v + G pi = f_v, -D v = f_pi, mean(pi) = 0.
        f_v: (N_f,) or (m, N_f)."""
        g, eta = self.g, self.eta
        single = f_v.ndim == 1
        fv = np.atleast_2d(f_v)
        m = fv.shape[0]
        fp = np.zeros((m, g.N_c)) if f_pi is None else np.atleast_2d(f_pi)
        fp = fp - fp.mean(axis=1, keepdims=True)
        Ainv_f = viscous_solve(g, eta, fv)
        rhs = (self.GT @ Ainv_f.T).T - fp
        rhs -= rhs.mean(axis=1, keepdims=True)
        pi = np.zeros((m, g.N_c))
        r = rhs.copy()
        z = eta * r
        p = z.copy()
        rz = np.sum(r * z, axis=1)
        nb = np.linalg.norm(rhs, axis=1)
        active = nb > 0
        for _ in range(maxiter):
            if not np.any(active):
                break
            Sp = (self.GT @ viscous_solve(g, eta, (self.G @ p.T).T).T).T
            Sp -= Sp.mean(axis=1, keepdims=True)
            pSp = np.sum(p * Sp, axis=1)
            alpha = np.where(active, rz / np.where(pSp != 0, pSp, 1.0), 0.0)
            pi += alpha[:, None] * p
            r -= alpha[:, None] * Sp
            active = active & (np.linalg.norm(r, axis=1) > tol * nb)
            z = eta * r
            rz_new = np.sum(r * z, axis=1)
            beta = np.where(active, rz_new / np.where(rz != 0, rz, 1.0), 0.0)
            p = z + beta[:, None] * p
            rz = rz_new
        pi -= pi.mean(axis=1, keepdims=True)
        v = Ainv_f - viscous_solve(g, eta, (self.G @ pi.T).T)
        if single:
            return v[0], pi[0]
        return v, pi


def stokes(g: Grid, eta, f_v, f_pi=None, tol=1e-14):
    return StokesOperator(g, eta).solve(f_v, f_pi, tol=tol)


# ------------------------------------------------------- mobility matrices
def blob_mobility(g: Grid, b, eta, chunk=48, op=None):
    """M = J L^{-1} S, dense (3 N_bl, 3 N_bl)."""
    op = op or StokesOperator(g, eta)
    r = b.positions()
    n = 3 * b.n_blobs
    M = np.zeros((n, n))
    for c0 in range(0, n, chunk):
        cols = range(c0, min(n, c0 + chunk))
        F = np.zeros((len(cols), g.N_f))
        for t, c in enumerate(cols):
            e = np.zeros(n); e[c] = 1.0
            F[t] = ib.spread(g, r, e)
        v, _ = op.solve(F)
        for t, c in enumerate(cols):
            M[:, c] = ib.interpolate(g, r, v[t])
    return M


def body_mobility(M, K):
    """N = (K^T M^{-1} K)^{-1}."""
    cf = sla.cho_factor(M)
    return np.linalg.inv(K.T @ sla.cho_solve(cf, K))


def constrained(g: Grid, b, eta, f, M=None, op=None):
    """Solution of the saddle system A x = f (pi with zero mean) by the
    reduced form of Eq. (incompleteN)."""
    op = op or StokesOperator(g, eta)
    o = saddle.layout(g, b)
    fv, fp, fl, fU = f[o[0]:o[3]], f[o[3]:o[4]], f[o[4]:o[5]], f[o[5]:o[6]]
    r = b.positions()
    v0, p0 = op.solve(fv, fp)
    if b.n_bodies == 0:
        return np.concatenate([v0, p0])
    if M is None:
        M = blob_mobility(g, b, eta, op=op)
    K = b.K_matrix()
    cf = sla.cho_factor(M)
    N = np.linalg.inv(K.T @ sla.cho_solve(cf, K))
    s = fl + ib.interpolate(g, r, v0)
    U = N @ (fU + K.T @ sla.cho_solve(cf, s))
    lam = sla.cho_solve(cf, K @ U - s)
    v1, p1 = op.solve(ib.spread(g, r, lam))
    return np.concatenate([v0 + v1, p0 + p1, lam, U])
