"""One step of the Split-Euler-Maruyama scheme, Algorithm 1, in the paper's
order, with the readings below.

Readings:
  * RFD quantities come from the physical solve with F = W^FT, zero slip and a
    homogeneous fluid (no walls, no noise): U* = N W^FT, lambda* = M^{-1} K U*,
    v* = L^{-1} S lambda* (Eq. ulvRFD up to the printed signs).
  * D^{K^T}, D^K, D^J, D^S are the difference quotients of Eqs.
    (allDemBoysa-allDemBoys2b) with the "+" signs printed there.
  * Step 6 solves with force F^n - D^{K^T} and slip u_slip + D^K - D^J - D^S
    (Eq. DriDef; then the drift is dN : (W^FT dQ^T), whose mean is
    kT div_Q N).
  * delta = eps^(1/3), eps = 2^-52 (centred RFD, Sec. IV.A); displaced
    orientations are lab-frame rotations by +-(delta/2) W^tau.
  * A step is rejected when a blob of the new configuration lies outside the
    domain along a wall axis (Sec. V: unphysical configurations are rejected).
"""
import numpy as np

from .grid import Grid
from . import saddle, solve, ib, rigid, noise, forces, operators

DELTA = 6.0554544523933395e-06


def sem_step(g: Grid, b, eta, kT, dt, potentials, seed, step, attempt=0, delta=DELTA,
             F_ext=None, slip=None, op=None, parts=False, normals=None, fluid_noise=True, M=None, rfd=True):
    """One SEM step from configuration b.  The random draws are Philox
    normals of (seed, step, attempt) unless injected: ``normals`` = (W^f,
    W^tau), each (N_b, 3), replaces the body draw of step 1, and
    ``fluid_noise=False`` drops the stochastic stress of step 6 (the drift
    tests drive the step with basis vectors).  ``M`` may pass a precomputed
    blob mobility of b.  ``rfd=False`` skips steps 1-5 and sets the drift
    terms of step 6 to zero: the naive Euler-Maruyama scheme whose biased
    equilibrium App. A shows."""
    op = op or solve.StokesOperator(g, eta)
    nb, nbl = b.n_bodies, b.n_blobs
    o = saddle.layout(g, b)
    # forces F^n
    F = forces.body_forces(g, b, potentials)
    if F_ext is not None:
        F = F + np.asarray(F_ext).reshape(nb, 6)
    if M is None:
        M = solve.blob_mobility(g, b, eta, op=op)
    if rfd:
        # step 1: random forces and torques
        if normals is None:
            Wf, Wt = noise.body_normals(nb, seed, step, attempt)
        else:
            Wf, Wt = (np.asarray(x, dtype=float).reshape(nb, 3) for x in normals)
        Lp = rigid.body_length(b.ref, b.offsets)
        WFT = noise.random_force_torque(Wf, Wt, Lp, kT)
        terms = rfd_terms(g, b, eta, kT, Wf, Wt, Lp, delta, M=M, op=op)
        D_KT, D_K, D_J, D_S = terms["D_KT"], terms["D_K"], terms["D_J"], terms["D_S"]
    else:
        terms = {}
        D_KT, D_K, D_J, D_S = np.zeros(6 * nb), np.zeros(3 * nbl), np.zeros(3 * nbl), np.zeros(3 * nbl)
    # step 6: fluctuating constrained solve
    f_noise = noise.fluid_forcing(g, eta, kT, dt, seed, step, attempt) if fluid_noise else np.zeros(g.N_f)
    slip_tot = (np.zeros(3 * nbl) if slip is None else np.asarray(slip).ravel()) + D_K - D_J - D_S
    f2 = saddle.rhs(g, b, eta, F=F.ravel() - D_KT, slip=slip_tot, f_fluid=f_noise, walls=True)
    x2 = solve.constrained(g, b, eta, f2, M=M, op=op)
    U = x2[o[5]:o[6]].reshape(nb, 6)
    # step 7: update
    q_new = b.q + dt * U[:, :3]
    quat_new = rigid.rotate(b.quat, dt * U[:, 3:])
    r_new = rigid.blob_positions(b.ref, b.offsets, q_new, quat_new)
    L = g.length()
    reject = False
    for a in range(3):
        if not g.periodic[a] and (np.any(r_new[:, a] < 0.0) or np.any(r_new[:, a] > L[a])):
            reject = True
    out = {"q": q_new, "quat": quat_new, "U": U, "reject": reject}
    if parts:
        out.update(terms)
        out.update({"F": F, "x": x2, "f_noise": f_noise, "M": M})
        if rfd:
            out.update({"WFT": WFT, "Wf": Wf, "Wt": Wt, "Lp": Lp})
    return out


def rfd_terms(g: Grid, b, eta, kT, Wf, Wt, Lp, delta=DELTA, M=None, op=None):
    """Algorithm 1 steps 2-5 for given body normals: the RFD solve, the
    displaced configurations, the unconstrained Stokes solve and the four
    random finite differences."""
    op = op or solve.StokesOperator(g, eta)
    o = saddle.layout(g, b)
    WFT = noise.random_force_torque(Wf, Wt, Lp, kT)
    # step 2: constrained solve with W^FT (homogeneous)
    f1 = saddle.rhs(g, b, eta, F=WFT, walls=False)
    x1 = solve.constrained(g, b, eta, f1, M=M, op=op)
    v_rfd, lam_rfd, U_rfd = x1[o[0]:o[3]], x1[o[4]:o[5]], x1[o[5]:o[6]]
    # step 3: randomly displaced configurations
    dq = (0.5 * delta) * Lp[:, None] * Wf
    bp = b.moved(b.q + dq, rigid.rotate(b.quat, 0.5 * delta * Wt))
    bm = b.moved(b.q - dq, rigid.rotate(b.quat, -0.5 * delta * Wt))
    rp, rm = bp.positions(), bm.positions()
    # step 4: unconstrained Stokes solve
    f_sharp = (ib.spread(g, rp, lam_rfd) - ib.spread(g, rm, lam_rfd)) / delta
    v_sharp, _ = op.solve(f_sharp)
    # step 5: random finite differences
    D_KT = (rigid.KT_apply(bp.ref, bp.offsets, bp.quat, lam_rfd)
            - rigid.KT_apply(bm.ref, bm.offsets, bm.quat, lam_rfd)) / delta
    D_K = (rigid.K_apply(bp.ref, bp.offsets, bp.quat, U_rfd)
           - rigid.K_apply(bm.ref, bm.offsets, bm.quat, U_rfd)) / delta
    D_J = (ib.interpolate(g, rp, v_rfd) - ib.interpolate(g, rm, v_rfd)) / delta
    D_S = ib.interpolate(g, b.positions(), v_sharp)
    return {"x_rfd": x1, "q_plus": bp.q, "quat_plus": bp.quat, "q_minus": bm.q,
            "quat_minus": bm.quat, "f_sharp": f_sharp, "v_sharp": v_sharp,
            "D_KT": D_KT, "D_K": D_K, "D_J": D_J, "D_S": D_S}
