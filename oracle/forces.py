"""External forces and torques on the bodies from the potentials of Sec. V:
the soft repulsion of Eq. (Usoft) between body centres and between centres or
blobs and the walls, the Yukawa pair repulsion of Eq. (YukawaPot), the
commensurate substrate potential of Sec. V.B.1, gravity on every body
("gravity") and on every blob ("blob_gravity": the buoyant weight of the
boomerang blobs of App. A, with its torque about the tracking point).

  Usoft:  Phi(r) = Phi0 (1 + (d - r)/b) for r < d, Phi0 exp((d - r)/b) for r >= d
          -dPhi/dr = (Phi0/b) * (1 if r < d else exp((d - r)/b))
  Yukawa: U(r) = U0 exp((D_H - r)/lambda_D) / (r / D_H)
          -dU/dr = U0 D_H exp((D_H - r)/lambda_D) (1/(lambda_D r) + 1/r^2)
  substrate: U = (U0/2) {3 - cos((k1 - k2).X) - cos(k1.X) - cos(k2.X)},
          X = (x, y - L_y/2), k1,2 = 4pi/(sqrt(3) s) (-sqrt(3)/2, -+1/2)
Pair distances use the minimum image along periodic axes.  Returns (N_b, 6).
"""
import numpy as np

from . import rigid


def _soft(r, phi0, b, d):
    return (phi0 / b) * np.where(r < d, 1.0, np.exp((d - r) / b))


def _pair_vectors(g, q):
    d = q[:, None, :] - q[None, :, :]
    L = g.length()
    for a in range(3):
        if g.periodic[a]:
            d[:, :, a] -= L[a] * np.round(d[:, :, a] / L[a])
    r = np.linalg.norm(d, axis=2)
    np.fill_diagonal(r, np.inf)
    return d, r


def body_forces(g, b, potentials):
    nb = b.n_bodies
    F = np.zeros((nb, 6))
    if nb == 0:
        return F
    q = b.q
    L = g.length()
    if "gravity" in potentials:
        F[:, 2] -= potentials["gravity"]
    if "pair_soft" in potentials and nb > 1:
        p = potentials["pair_soft"]
        d, r = _pair_vectors(g, q)
        mag = np.where(np.isfinite(r), _soft(np.where(np.isfinite(r), r, 1.0), p["phi0"], p["b"], p["d"]), 0.0)
        F[:, :3] += np.sum(mag[:, :, None] * d / np.where(np.isfinite(r), r, 1.0)[:, :, None], axis=1)
    if "yukawa" in potentials and nb > 1:
        p = potentials["yukawa"]
        d, r = _pair_vectors(g, q)
        rr = np.where(np.isfinite(r), r, 1.0)
        mag = p["u0"] * p["d_h"] * np.exp((p["d_h"] - rr) / p["lambda_d"]) * (1.0 / (p["lambda_d"] * rr) + 1.0 / rr ** 2)
        mag = np.where(np.isfinite(r), mag, 0.0)
        F[:, :3] += np.sum(mag[:, :, None] * d / rr[:, :, None], axis=1)
    if "wall_soft" in potentials:
        p = potentials["wall_soft"]
        for a in range(3):
            if g.periodic[a]:
                continue
            F[:, a] += _soft(q[:, a], p["phi0"], p["b"], p["d"])
            F[:, a] -= _soft(L[a] - q[:, a], p["phi0"], p["b"], p["d"])
    if "blob_gravity" in potentials:
        arm = rigid.arms(b.ref, b.offsets, b.quat)
        f = np.zeros_like(arm)
        f[:, 2] = -potentials["blob_gravity"]
        bb = rigid.body_of_blob(b.offsets)
        np.add.at(F[:, :3], bb, f)
        np.add.at(F[:, 3:], bb, np.cross(arm, f))
    if "blob_wall_soft" in potentials:
        p = potentials["blob_wall_soft"]
        r = b.positions()
        arm = rigid.arms(b.ref, b.offsets, b.quat)
        f = np.zeros_like(r)
        for a in range(3):
            if g.periodic[a]:
                continue
            f[:, a] += _soft(r[:, a], p["phi0"], p["b"], p["d"])
            f[:, a] -= _soft(L[a] - r[:, a], p["phi0"], p["b"], p["d"])
        bb = rigid.body_of_blob(b.offsets)
        np.add.at(F[:, :3], bb, f)
        np.add.at(F[:, 3:], bb, np.cross(arm, f))
    if "substrate" in potentials:
        p = potentials["substrate"]
        s = p["s_lattice"]
        c = 4.0 * np.pi / (np.sqrt(3.0) * s)
        k1 = c * np.array([-np.sqrt(3.0) / 2.0, -0.5])
        k2 = c * np.array([-np.sqrt(3.0) / 2.0, 0.5])
        X = np.stack([q[:, 0], q[:, 1] - L[1] / 2.0], axis=1)
        grad = np.zeros((nb, 2))
        for k in (k1 - k2, k1, k2):
            grad += np.sin(X @ k)[:, None] * k[None, :]
        F[:, :2] -= 0.5 * p["u0"] * grad
    return F
