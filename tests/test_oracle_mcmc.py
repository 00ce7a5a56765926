"""Pins of the Gibbs-Boltzmann sampler (oracle/mcmc.py).

  * its energy is the potential of oracle/forces.py: central differences of
    mcmc.energy in the tracking points and in lab-frame rotation angles equal
    the oracle's forces and torques, every potential on its own and together;
  * one blob under gravity between two soft walls: the sampled height has the
    mean and variance of the density exp(-U(z)/kT) on [0, L], computed here by
    quadrature;
  * a two-blob dumbbell under blob gravity far from the walls: the cosine of
    its axis with z has the mean -coth(beta) + 1/beta, beta = g a / kT (the
    Boltzmann factor exp(-beta cos) on the uniform sphere), so the rotation
    moves sample orientations with the Haar measure;
  * a body with no orientation-dependent energy has uniformly distributed
    orientations (every entry of the rotation matrix averages to zero)."""
import numpy as np
import pytest
from scipy.integrate import quad
from scipy.spatial.transform import Rotation

import workloads
from oracle import Grid, forces, mcmc, rigid, saddle

POT = {
    "gravity": 0.8,
    "blob_gravity": 0.3,
    "pair_soft": {"phi0": 4.0, "b": 0.25, "d": 2.6},
    "yukawa": {"u0": 20.0, "d_h": 2.0, "lambda_d": 0.45},
    "wall_soft": {"phi0": 4.0, "b": 0.25, "d": 1.6},
    "blob_wall_soft": {"phi0": 4.0, "b": 0.2, "d": 1.0},
    "substrate": {"u0": 4.0, "s_lattice": 6.0},
}


def _bodies():
    rng = np.random.default_rng(2)
    shell = workloads.icosahedral_shell(12, 1.0) + np.array([0.2, -0.1, 0.15])   # off-centre tracking point
    quat = rng.standard_normal((3, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    ref = np.vstack([shell] * 3)
    off = np.array([0, 12, 24, 36])
    q = np.array([[1.6, 2.3, 1.5], [3.6, 3.4, 2.2], [11.3, 4.1, 2.4]])
    return Grid((12, 8, 7), periodic=(True, False, False)), ref, off, q, quat


@pytest.mark.parametrize("term", list(POT) + ["all"])
def test_energy_gradient_is_the_oracle_force(term):
    g, ref, off, q, quat = _bodies()
    pot = dict(POT) if term == "all" else {term: POT[term]}
    F = forces.body_forces(g, saddle.Bodies(ref, off, q, quat), pot)
    h = 1e-6
    Ffd = np.zeros_like(F)
    for p in range(3):
        for c in range(3):
            qp, qm = q.copy(), q.copy()
            qp[p, c] += h
            qm[p, c] -= h
            Ffd[p, c] = -(mcmc.energy(g, ref, off, qp, quat, pot) - mcmc.energy(g, ref, off, qm, quat, pot)) / (2 * h)
            phi = np.zeros(3)
            phi[c] = h
            tp, tm = quat.copy(), quat.copy()
            # scipy rotations, (x, y, z, w) order
            tp[p] = np.roll((Rotation.from_rotvec(phi) * Rotation.from_quat(np.roll(quat[p], -1))).as_quat(), 1)
            tm[p] = np.roll((Rotation.from_rotvec(-phi) * Rotation.from_quat(np.roll(quat[p], -1))).as_quat(), 1)
            Ffd[p, 3 + c] = -(mcmc.energy(g, ref, off, q, tp, pot) - mcmc.energy(g, ref, off, q, tm, pot)) / (2 * h)
    scale = max(np.abs(Ffd).max(), 1.0)
    np.testing.assert_allclose(F, Ffd, rtol=0, atol=3e-7 * scale)


def test_outside_configuration_has_zero_weight():
    g, ref, off, q, quat = _bodies()
    q2 = q.copy()
    q2[0, 2] = 0.3                    # a blob below the bottom wall
    assert mcmc.energy(g, ref, off, q2, quat, {}) == np.inf


def test_height_of_one_blob_follows_boltzmann():
    g = Grid((6, 6, 10), periodic=(True, True, False))
    pot = {"gravity": 0.6, "wall_soft": {"phi0": 4.0, "b": 0.5, "d": 1.0}}
    ref, off = np.zeros((1, 3)), np.array([0, 1])
    qs, _, acc = mcmc.sample(g, ref, off, [[3.0, 3.0, 5.0]], [[1.0, 0, 0, 0]], pot, 1.0, n_samples=6000, thin=6,
                             burn=500, step_q=1.5, step_rot=0.0, seed=3)
    assert 0.2 < acc < 0.9
    z = qs[:, 0, 2]
    L = 10.0

    def U(x):
        return mcmc.energy(g, ref, off, [[3.0, 3.0, x]], [[1.0, 0, 0, 0]], pot)
    Z = quad(lambda x: np.exp(-U(x)), 0.0, L, limit=200)[0]
    m1 = quad(lambda x: x * np.exp(-U(x)), 0.0, L, limit=200)[0] / Z
    m2 = quad(lambda x: x * x * np.exp(-U(x)), 0.0, L, limit=200)[0] / Z
    var = m2 - m1 ** 2
    n_eff = z.size / 2.0             # thinned chain: allow a correlation time of two samples
    assert abs(z.mean() - m1) < 5 * np.sqrt(var / n_eff)
    assert abs(z.var() - var) < 5 * var * np.sqrt(2.0 / n_eff)


def test_dumbbell_orientation_under_blob_gravity():
    g = Grid((12, 12, 30), periodic=(True, True, False))
    a, gb = 2.0, 0.7
    pot = {"blob_gravity": gb, "wall_soft": {"phi0": 8.0, "b": 0.5, "d": 6.0}}
    ref, off = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, a]]), np.array([0, 2])
    qs, ts, acc = mcmc.sample(g, ref, off, [[6.0, 6.0, 15.0]], [[1.0, 0, 0, 0]], pot, 1.0, n_samples=6000, thin=4,
                              burn=500, step_q=1.0, step_rot=0.9, seed=5)
    R = rigid.quat_to_rot(ts[:, 0])
    cos = R[:, 2, 2]                  # z component of the rotated axis (0, 0, 1)
    beta = gb * a
    want = -(1.0 / np.tanh(beta) - 1.0 / beta)
    var = 1.0 - 2.0 * (1.0 / np.tanh(beta)) / beta + 2.0 / beta ** 2 - want ** 2
    assert abs(cos.mean() - want) < 5 * np.sqrt(var / (cos.size / 3.0))


def test_free_orientations_are_uniform():
    g = Grid((10, 10, 10), periodic=(True, True, False))
    ref, off = workloads.icosahedral_shell(12, 1.0), np.array([0, 12])
    pot = {"wall_soft": {"phi0": 4.0, "b": 0.5, "d": 2.5}}
    _, ts, _ = mcmc.sample(g, ref, off, [[5.0, 5.0, 5.0]], [[1.0, 0, 0, 0]], pot, 1.0, n_samples=3000, thin=4,
                           burn=300, step_q=0.5, step_rot=1.2, seed=7)
    R = rigid.quat_to_rot(ts[:, 0])
    # each entry of a Haar-random rotation has mean 0 and variance 1/3
    assert np.abs(R.mean(axis=0)).max() < 5 * np.sqrt(1.0 / 3.0 / (ts.shape[0] / 3.0))
