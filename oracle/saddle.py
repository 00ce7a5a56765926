"""The constrained saddle-point system of Sec. III.C, Eqs. (LangevinD1-D4).

Sign convention (our reading; the matrices printed in Algorithm 1 steps 2 and
6 carry -K and -K^T, which contradicts Eq. (LangevinD3)):

  [ -eta LL   G   -S   0 ] [v  ]   [f_v]      f_v = g + noise + eta * wall terms
  [   -D      0    0   0 ] [pi ] = [f_pi]     f_pi = 0
  [   -J      0    0   K ] [lam]   [f_lam]    f_lam = -slip + J wall part
  [    0      0   K^T  0 ] [U  ]   [f_U]      f_U = F

W A is symmetric for W = diag(dV I, dV I, I, I).  Vector layout:
[v_x | v_y | v_z | pi | lambda (N_bl x 3) | U (N_b x 6: u, w)].
"""
import numpy as np
import scipy.sparse as sp

from .grid import Grid
from . import operators, ib, rigid


class Bodies:
    """Blob shells, body placements and orientations.  With ``r`` given, the
    blob positions are taken as independent inputs (arms r_i - q_p), as the
    adjoint's gradient with respect to blob positions requires."""

    def __init__(self, ref, offsets, q, quat, r=None):
        self.ref = np.asarray(ref, dtype=np.float64).reshape(-1, 3)
        self.offsets = np.asarray(offsets, dtype=np.int64)
        self.q = np.asarray(q, dtype=np.float64).reshape(-1, 3)
        self.quat = np.asarray(quat, dtype=np.float64).reshape(-1, 4)
        self.r = None if r is None else np.asarray(r, dtype=np.float64).reshape(-1, 3)

    @property
    def n_blobs(self):
        return self.ref.shape[0]

    @property
    def n_bodies(self):
        return self.q.shape[0]

    def positions(self):
        if self.r is not None:
            return self.r
        return rigid.blob_positions(self.ref, self.offsets, self.q, self.quat)

    def arms(self):
        if self.r is not None:
            return self.r - self.q[rigid.body_of_blob(self.offsets)]
        return rigid.arms(self.ref, self.offsets, self.quat)

    def K_matrix(self):
        return rigid.K_matrix_arms(self.arms(), self.offsets)

    def K_apply(self, U):
        return rigid.K_apply_arms(self.arms(), self.offsets, U)

    def KT_apply(self, lam):
        return rigid.KT_apply_arms(self.arms(), self.offsets, lam)

    def moved(self, q, quat):
        return Bodies(self.ref, self.offsets, q, quat)

    def with_positions(self, r):
        return Bodies(self.ref, self.offsets, self.q, self.quat, r=r)


def layout(g: Grid, b: Bodies):
    """Offsets of the blocks [vx, vy, vz, pi, lambda, U, end]."""
    o = [0, g.n_face(0), g.n_face(0) + g.n_face(1), g.N_f, g.N_f + g.N_c]
    o.append(o[-1] + 3 * b.n_blobs)
    o.append(o[-1] + 6 * b.n_bodies)
    return o


def assemble(g: Grid, b: Bodies, eta):
    """Sparse saddle matrix A (tiny and medium problems)."""
    L = operators.vector_laplacian(g)
    D = operators.divergence(g)
    G = operators.gradient(g)
    r = b.positions()
    J = ib.J_matrix(g, r)
    S = (J.T / g.dV).tocsr()
    K = sp.csr_matrix(b.K_matrix())
    nl, nU = 3 * b.n_blobs, 6 * b.n_bodies
    blocks = [[-eta * L, G, -S, None],
              [-D, None, None, None],
              [-J, None, None, K],
              [None, None, K.T, None]]
    # explicit zero blocks keep bmat's shape inference happy for empty bodies
    blocks[1][1] = sp.csr_matrix((g.N_c, g.N_c))
    blocks[3][3] = sp.csr_matrix((nU, nU))
    blocks[2][2] = sp.csr_matrix((nl, nl))
    return sp.bmat(blocks, format="csr")


def apply(g: Grid, b: Bodies, eta, x, L=None, D=None, G=None):
    """y = A x computed block by block from the operator definitions."""
    if L is None:
        L = operators.vector_laplacian(g)
    if D is None:
        D = operators.divergence(g)
    if G is None:
        G = operators.gradient(g)
    o = layout(g, b)
    v, pi, lam, U = x[o[0]:o[3]], x[o[3]:o[4]], x[o[4]:o[5]], x[o[5]:o[6]]
    r = b.positions()
    y = np.zeros_like(x)
    y[o[0]:o[3]] = -eta * (L @ v) + G @ pi - ib.spread(g, r, lam)
    y[o[3]:o[4]] = -(D @ v)
    y[o[4]:o[5]] = -ib.interpolate(g, r, v) + b.K_apply(U)
    y[o[5]:o[6]] = b.KT_apply(lam)
    return y


def rhs(g: Grid, b: Bodies, eta, F=None, slip=None, f_fluid=None, walls=True):
    """Right-hand side for forces/torques F (N_b,6), active slip (N_bl,3),
    fluid forcing f_fluid (N_f,) and, with ``walls``, the moving-wall terms."""
    o = layout(g, b)
    out = np.zeros(o[-1])
    if f_fluid is not None:
        out[o[0]:o[3]] += f_fluid
    if walls:
        out[o[0]:o[3]] += operators.wall_velocity_rhs(g, eta)
        out[o[4]:o[5]] += ib.interpolate_wall_part(g, b.positions())
    if slip is not None:
        out[o[4]:o[5]] -= np.asarray(slip).ravel()
    if F is not None:
        out[o[5]:o[6]] += np.asarray(F).ravel()
    return out


def weights(g: Grid, b: Bodies):
    """Diagonal of W: the inner product in which A is self-adjoint."""
    o = layout(g, b)
    w = np.ones(o[-1])
    w[o[0]:o[4]] = g.dV
    return w
