"""Samples of the Gibbs-Boltzmann distribution of the bodies' positions and
orientations, P(Q) ~ exp(-U(Q) / kT): the equilibrium distribution that the
SEM scheme reproduces to first order in dt (App. A, App. B), and the source of
the reference values of Sec. V.A (the long-time MSD asymptote, Eq. asymRef,
and the Gibbs-Boltzmann average of the mobility in Eq. SErel).

U is the potential energy whose negative gradient oracle/forces.py returns:
  * Eq. (Usoft) between body centres ("pair_soft"), between centres and walls
    ("wall_soft") and between blobs and walls ("blob_wall_soft"):
      Phi(r) = Phi0 (1 + (d - r)/b) for r < d, Phi0 exp((d - r)/b) for r >= d;
  * Eq. (YukawaPot) between body centres: U0 exp((D_H - r)/lambda_D) / (r/D_H);
  * the substrate potential of Sec. V.B.1:
      (U0/2) {3 - cos((k1 - k2).X) - cos(k1.X) - cos(k2.X)},
      X = (x, y - L_y/2), k1,2 = 4 pi / (sqrt(3) s) (-sqrt(3)/2, -+1/2);
  * gravity g z on every body ("gravity") and on every blob ("blob_gravity").
Pair distances use the minimum image along periodic axes.  A configuration
with a blob centre outside [0, L] along a wall axis has zero weight (the SEM
step rejects it, Sec. V).

Sampler: Metropolis random walk, one body per move, with a Gaussian
displacement of its tracking point and a lab-frame rotation by a Gaussian
angle vector (both proposals symmetric: the rotation increment is isotropic,
so the density of R' given R equals that of R given R'), accepted with
probability min(1, exp(-dU/kT)).

Test infrastructure: only tests/ and bench.py's reference legs use it.
"""
import numpy as np

from . import rigid


def _usoft(r, phi0, b, d):
    r = np.asarray(r, dtype=np.float64)
    return phi0 * np.where(r < d, 1.0 + (d - r) / b, np.exp((d - r) / b))


def energy(g, ref, offsets, q, quat, potentials):
    """U of bodies (tracking points q (N_b, 3), orientations quat (N_b, 4)),
    or +inf if a blob lies outside the domain along a wall axis."""
    q = np.asarray(q, dtype=np.float64).reshape(-1, 3)
    nb = q.shape[0]
    L = g.length()
    r = rigid.blob_positions(ref, offsets, q, quat)
    for a in range(3):
        if not g.periodic[a] and (np.any(r[:, a] < 0.0) or np.any(r[:, a] > L[a])):
            return np.inf
    U = 0.0
    if "gravity" in potentials:
        U += potentials["gravity"] * np.sum(q[:, 2])
    if "blob_gravity" in potentials:
        U += potentials["blob_gravity"] * np.sum(r[:, 2])
    if nb > 1 and ("pair_soft" in potentials or "yukawa" in potentials):
        iu, ju = np.triu_indices(nb, 1)
        dv = q[iu] - q[ju]
        for a in range(3):
            if g.periodic[a]:
                dv[:, a] -= L[a] * np.round(dv[:, a] / L[a])
        dist = np.linalg.norm(dv, axis=1)
        if "pair_soft" in potentials:
            p = potentials["pair_soft"]
            U += np.sum(_usoft(dist, p["phi0"], p["b"], p["d"]))
        if "yukawa" in potentials:
            p = potentials["yukawa"]
            U += np.sum(p["u0"] * np.exp((p["d_h"] - dist) / p["lambda_d"]) * p["d_h"] / dist)
    for a in range(3):
        if g.periodic[a]:
            continue
        if "wall_soft" in potentials:
            p = potentials["wall_soft"]
            U += np.sum(_usoft(q[:, a], p["phi0"], p["b"], p["d"]) + _usoft(L[a] - q[:, a], p["phi0"], p["b"], p["d"]))
        if "blob_wall_soft" in potentials:
            p = potentials["blob_wall_soft"]
            U += np.sum(_usoft(r[:, a], p["phi0"], p["b"], p["d"]) + _usoft(L[a] - r[:, a], p["phi0"], p["b"], p["d"]))
    if "substrate" in potentials:
        p = potentials["substrate"]
        c = 4.0 * np.pi / (np.sqrt(3.0) * p["s_lattice"])
        k1 = c * np.array([-np.sqrt(3.0) / 2.0, -0.5])
        k2 = c * np.array([-np.sqrt(3.0) / 2.0, 0.5])
        X = np.stack([q[:, 0], q[:, 1] - L[1] / 2.0], axis=1)
        U += 0.5 * p["u0"] * np.sum(3.0 - np.cos(X @ (k1 - k2)) - np.cos(X @ k1) - np.cos(X @ k2))
    return float(U)


def sample(g, ref, offsets, q0, quat0, potentials, kT, n_samples, thin=20, burn=2000,
           step_q=0.2, step_rot=0.1, seed=0):
    """Markov chain from (q0, quat0): ``burn`` sweeps discarded, then
    ``n_samples`` states recorded every ``thin`` sweeps (a sweep is one move
    per body).  Returns (q (n, N_b, 3), quat (n, N_b, 4), acceptance rate);
    positions along periodic axes are kept unwrapped."""
    rng = np.random.Generator(np.random.Philox(seed))
    q = np.array(q0, dtype=np.float64).reshape(-1, 3)
    quat = np.array(quat0, dtype=np.float64).reshape(-1, 4)
    nb = q.shape[0]
    U = energy(g, ref, offsets, q, quat, potentials)
    if not np.isfinite(U):
        raise ValueError("the initial configuration has zero weight")
    out_q = np.empty((n_samples, nb, 3))
    out_t = np.empty((n_samples, nb, 4))
    acc = tries = 0
    total = burn + n_samples * thin
    k = 0
    for sweep in range(total):
        for p in range(nb):
            qn, tn = q.copy(), quat.copy()
            qn[p] += step_q * rng.standard_normal(3)
            tn[p] = rigid.rotate(quat[p:p + 1], step_rot * rng.standard_normal(3))[0]
            Un = energy(g, ref, offsets, qn, tn, potentials)
            tries += 1
            if np.isfinite(Un) and (Un <= U or rng.random() < np.exp(-(Un - U) / kT)):
                q, quat, U = qn, tn, Un
                acc += 1
        if sweep >= burn and (sweep - burn) % thin == thin - 1:
            out_q[k], out_t[k] = q, quat
            k += 1
    return out_q, out_t, acc / max(tries, 1)
