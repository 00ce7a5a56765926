"""Random draws of the SEM scheme (Algorithm 1 steps 1 and 6).

  * stochastic stress W: one standard normal per element of the nine
    independent stress blocks, in the global order of Grid.stress_blocks,
    purpose 1 of the Philox stream; the fluid forcing is
    sqrt(2 eta kT / (dV dt)) DD W  (Eq. LangevinD1);
  * body forces: W^f_p = normals 6p..6p+2 and W^tau_p = normals 6p+3..6p+5 of
    purpose 2, W^FT_p = kT [W^f_p / L_p ; W^tau_p]  (Sec. IV.B).
"""
import numpy as np

from . import philox, operators


def stress(g, seed, step, attempt=0):
    return philox.normals(seed, step, attempt, philox.PURPOSE_FLUID, g.N_w)


def fluid_forcing(g, eta, kT, dt, seed, step, attempt=0, W=None, DD=None):
    if W is None:
        W = stress(g, seed, step, attempt)
    if DD is None:
        DD = operators.tensor_divergence(g)
    return np.sqrt(2.0 * eta * kT / (g.dV * dt)) * (DD @ W)


def body_normals(n_bodies, seed, step, attempt=0):
    z = philox.normals(seed, step, attempt, philox.PURPOSE_BODY, 6 * n_bodies).reshape(n_bodies, 6)
    return z[:, :3], z[:, 3:]


def random_force_torque(Wf, Wt, L, kT):
    return np.concatenate([kT * Wf / L[:, None], kT * Wt], axis=1)
