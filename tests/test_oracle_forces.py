"""Pin of the oracle's body forces and torques (oracle/forces.py) against
central finite differences of the potential ENERGIES, written out here from
the paper: the soft repulsion of Eq. (Usoft) (between body centres, between
centres and walls, and between blobs and walls), the Yukawa pair repulsion of
Eq. (YukawaPot), the commensurate substrate potential of Sec. V.B.1, gravity
on the bodies and on every blob (App. A).  The force on body p is -dE/dq_p; the torque is -dE/dphi_p, with
phi_p a lab-frame rotation angle applied to body p's arms (blob positions
q_p + R(phi_p) R(quat_p) r_ref), computed with scipy's rotations rather than
the oracle's quaternion code.  Pair distances use the minimum image along
periodic axes.  A dropped term, a sign slip or a wrong derivative anywhere in
the oracle changes the force or torque at O(1) against these energies."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import workloads
from oracle import Grid, saddle, forces


def usoft(r, phi0, b, d):
    """Eq. (Usoft): Phi0 (1 + (d - r)/b) inside d, Phi0 exp((d - r)/b) outside."""
    r = np.asarray(r, dtype=float)
    return phi0 * np.where(r < d, 1.0 + (d - r) / b, np.exp((d - r) / b))


def yukawa(r, u0, dh, lam):
    """Eq. (YukawaPot): U0 exp((D_H - r)/lambda_D) / (r / D_H)."""
    return u0 * np.exp((dh - r) / lam) / (r / dh)


def substrate(x, y, ly, u0, s):
    """Sec. V.B.1: (U0/2) {3 - cos((k1 - k2).X) - cos(k1.X) - cos(k2.X)} with
    X = (x, y - L_y/2), k1,2 = 4 pi / (sqrt(3) s) (-sqrt(3)/2, -+1/2)."""
    c = 4.0 * np.pi / (np.sqrt(3.0) * s)
    k1 = c * np.array([-np.sqrt(3.0) / 2.0, -0.5])
    k2 = c * np.array([-np.sqrt(3.0) / 2.0, 0.5])
    X = np.array([x, y - ly / 2.0])
    return 0.5 * u0 * (3.0 - np.cos((k1 - k2) @ X) - np.cos(k1 @ X) - np.cos(k2 @ X))


def min_image(dv, L, per):
    dv = dv.copy()
    for a in range(3):
        if per[a]:
            dv[a] -= L[a] * np.round(dv[a] / L[a])
    return dv


def energy(L, per, q, arms, pot):
    """Total potential energy of bodies at centres q with lab-frame arms."""
    nb = len(q)
    E = 0.0
    if "gravity" in pot:
        E += pot["gravity"] * np.sum(q[:, 2])
    if "blob_gravity" in pot:                     # weight of every blob at its height
        E += pot["blob_gravity"] * sum(np.sum(q[p, 2] + arms[p][:, 2]) for p in range(nb))
    for p in range(nb):
        for s in range(p + 1, nb):
            r = np.linalg.norm(min_image(q[p] - q[s], L, per))
            if "pair_soft" in pot:
                c = pot["pair_soft"]
                E += usoft(r, c["phi0"], c["b"], c["d"])
            if "yukawa" in pot:
                c = pot["yukawa"]
                E += yukawa(r, c["u0"], c["d_h"], c["lambda_d"])
    for a in range(3):
        if per[a]:
            continue
        if "wall_soft" in pot:
            c = pot["wall_soft"]
            E += np.sum(usoft(q[:, a], c["phi0"], c["b"], c["d"]) + usoft(L[a] - q[:, a], c["phi0"], c["b"], c["d"]))
        if "blob_wall_soft" in pot:
            c = pot["blob_wall_soft"]
            for p in range(nb):
                r = q[p][None, :] + arms[p]
                E += np.sum(usoft(r[:, a], c["phi0"], c["b"], c["d"])
                            + usoft(L[a] - r[:, a], c["phi0"], c["b"], c["d"]))
    if "substrate" in pot:
        c = pot["substrate"]
        for p in range(nb):
            E += substrate(q[p, 0], q[p, 1], L[1], c["u0"], c["s_lattice"])
    return E


def fd_forces(L, per, q, arms, pot, h=1e-6):
    nb = len(q)
    F = np.zeros((nb, 6))
    for p in range(nb):
        for c in range(3):
            qp, qm = q.copy(), q.copy()
            qp[p, c] += h
            qm[p, c] -= h
            F[p, c] = -(energy(L, per, qp, arms, pot) - energy(L, per, qm, arms, pot)) / (2 * h)
        for c in range(3):
            phi = np.zeros(3)
            phi[c] = h
            ap, am = list(arms), list(arms)
            ap[p] = Rotation.from_rotvec(phi).apply(arms[p])
            am[p] = Rotation.from_rotvec(-phi).apply(arms[p])
            F[p, 3 + c] = -(energy(L, per, q, ap, pot) - energy(L, per, q, am, pot)) / (2 * h)
    return F


def lab_arms(ref, offsets, quat):
    """Arms R(quat_p) r_ref from scipy (quaternions stored w first here)."""
    out = []
    for p in range(len(offsets) - 1):
        R = Rotation.from_quat(np.roll(quat[p], -1))      # scipy wants (x, y, z, w)
        out.append(R.apply(ref[offsets[p]:offsets[p + 1]]))
    return out


ALL = {
    "gravity": 1.3,
    "pair_soft": {"phi0": 4.0, "b": 0.25, "d": 2.6},
    "yukawa": {"u0": 20.0, "d_h": 2.0, "lambda_d": 0.45},
    "wall_soft": {"phi0": 4.0, "b": 0.25, "d": 1.6},
    "blob_wall_soft": {"phi0": 4.0, "b": 0.2, "d": 1.0},
    "substrate": {"u0": 4.0, "s_lattice": 6.0},
}


def _bodies(n, per, q):
    """Three 12-blob shells of radius 1.0 with seeded orientations."""
    rng = np.random.default_rng(17)
    shell = workloads.icosahedral_shell(12, 1.0)
    nb = len(q)
    quat = rng.standard_normal((nb, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    ref = np.vstack([shell] * nb)
    off = [12 * p for p in range(nb + 1)]
    g = Grid(n, periodic=per)
    b = saddle.Bodies(ref, off, np.asarray(q, dtype=float), quat)
    return g, b


# Bodies placed so that the pair and wall terms sit on both branches of
# Eq. (Usoft) (inside and outside d) and blobs lie close to the walls.
GEOMS = {
    "walls": ((10, 9, 8), (False, False, False),
              [[1.5, 2.1, 1.2], [3.4, 3.0, 2.0], [6.5, 6.8, 5.9]]),
    # body 0 and body 2 interact only through the periodic image along x
    "xperiodic": ((12, 8, 7), (True, False, False),
                  [[0.6, 3.0, 1.4], [5.8, 4.4, 3.5], [11.1, 3.9, 2.1]]),
    "yzperiodic": ((9, 10, 11), (False, True, True),
                   [[1.3, 0.4, 9.8], [4.0, 9.4, 1.6], [7.6, 5.0, 5.5]]),
}


@pytest.mark.parametrize("geom", list(GEOMS))
@pytest.mark.parametrize("term", list(ALL) + ["all"])
def test_body_forces_are_minus_energy_gradient(geom, term):
    n, per, q = GEOMS[geom]
    g, b = _bodies(n, per, q)
    pot = dict(ALL) if term == "all" else {term: ALL[term]}
    L = np.asarray(g.length(), dtype=float)
    arms = lab_arms(b.ref, b.offsets, b.quat)
    F_fd = fd_forces(L, per, b.q, arms, pot)
    F = forces.body_forces(g, b, pot)
    scale = np.abs(F_fd).max()
    if term in ("pair_soft", "yukawa", "wall_soft", "blob_wall_soft", "substrate"):
        assert scale > 1e-3, "the geometry must exercise this potential"
    np.testing.assert_allclose(F, F_fd, rtol=0, atol=2e-7 * max(scale, 1.0))


def test_periodic_image_pair_force():
    """Two bodies 1.5 apart only across the periodic x boundary repel along
    -x / +x with the Usoft slope Phi0/b (inside d), and feel nothing from the
    direct (long) separation."""
    g, b = _bodies((12, 8, 8), (True, False, False), [[0.4, 4.0, 4.0], [10.9, 4.0, 4.0]])
    pot = {"pair_soft": {"phi0": 4.0, "b": 0.5, "d": 2.0}}
    F = forces.body_forces(g, b, pot)
    np.testing.assert_allclose(F[0], [4.0 / 0.5, 0, 0, 0, 0, 0], atol=1e-12)
    np.testing.assert_allclose(F[1], [-4.0 / 0.5, 0, 0, 0, 0, 0], atol=1e-12)


def test_blob_gravity_force_and_torque():
    """Gravity on every blob of bodies whose tracking point is off the blob
    centroid (an L-shaped arm, as the boomerang of App. A): the force is the
    total weight and the torque is that of the weight at the centroid."""
    n, per = (10, 9, 8), (False, False, False)
    rng = np.random.default_rng(4)
    arm = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.5, 0.0], [0.0, 1.0, 0.0]])
    quat = rng.standard_normal((2, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    g = Grid(n, periodic=per)
    b = saddle.Bodies(np.vstack([arm, arm]), [0, 5, 10], np.array([[3.0, 3.0, 3.0], [6.0, 5.0, 4.0]]), quat)
    pot = {"blob_gravity": 0.7}
    L = np.asarray(g.length(), dtype=float)
    arms = lab_arms(b.ref, b.offsets, b.quat)
    F_fd = fd_forces(L, per, b.q, arms, pot)
    F = forces.body_forces(g, b, pot)
    np.testing.assert_allclose(F, F_fd, rtol=0, atol=2e-7)
    assert np.abs(F[:, 3:]).max() > 0.1              # the torque is exercised
    np.testing.assert_allclose(F[:, 2], -0.7 * 5, atol=1e-12)
