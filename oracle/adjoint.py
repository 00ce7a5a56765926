"""Adjoint of the mobility solve: gradients of a loss of the body velocities
with respect to blob positions and active slip (an extension of the method;
the paper's Eqs. LangevinD1-D4 define the forward map).

Forward: A(r) x = b(slip), x = [v, pi, lambda, U], b = [0, 0, -slip, F]
(static walls).  For L(U):
  * W A is symmetric (W = diag(dV, dV, 1, 1)), so A^T y = dL/dx is solved as
    A z = W^{-1} dL/dx = [0, 0, 0, dL/dU] and y = W z;
  * dL/dslip = y_lambda^T d b/d slip = -z_lambda;
  * dL/dr_i = -y^T (dA/dr_i) x, with the r-dependent blocks -S, -J, K, K^T:
      dL/dr_i = sum_a lambda_ia D(z_v)_ia + sum_a z_lambda,ia D(v)_ia
                - z_lambda,i x w_p - lambda_i x tau_p,
    D(f)_ia = d (J f)_ia / d r_i and tau_p the rotational part of z_U.
Blob positions are independent inputs (arms r_i - q_p).
"""
import numpy as np

from . import saddle, solve, ib


def forward(g, b, eta, slip, F=None, op=None):
    """x and U of the constrained solve with slip and force F (default 0)."""
    nb = b.n_bodies
    F = np.zeros((nb, 6)) if F is None else np.asarray(F).reshape(nb, 6)
    f = saddle.rhs(g, b, eta, F=F, slip=slip, walls=False)
    x = solve.constrained(g, b, eta, f, op=op)
    return x, x[-6 * nb:]


def loss(U):
    return float(np.sum(np.asarray(U) ** 2))


def gradient(g, b, eta, x, dL_dU, op=None):
    """(dL/dr (N_bl,3), dL/dslip (N_bl*3,)) at the forward solution x."""
    o = saddle.layout(g, b)
    nb = b.n_bodies
    f = saddle.rhs(g, b, eta, F=np.asarray(dL_dU).reshape(nb, 6), walls=False)
    z = solve.constrained(g, b, eta, f, op=op)
    v, lam, U = x[o[0]:o[3]], x[o[4]:o[5]].reshape(-1, 3), x[o[5]:o[6]].reshape(-1, 6)
    zv, zl, zU = z[o[0]:o[3]], z[o[4]:o[5]].reshape(-1, 3), z[o[5]:o[6]].reshape(-1, 6)
    r = b.positions()
    Dz = ib.interpolate_derivative(g, r, zv)
    Dv = ib.interpolate_derivative(g, r, v)
    bb = np.repeat(np.arange(nb), np.diff(b.offsets))
    dr = (np.einsum("na,nab->nb", lam, Dz) + np.einsum("na,nab->nb", zl, Dv)
          - np.cross(zl, U[bb, 3:]) - np.cross(lam, zU[bb, 3:]))
    return dr, -zl.ravel()
