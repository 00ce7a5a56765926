"""Write the stored expected values under tests/golden/ with the FP64 oracle.

Every number here comes from oracle/ only (never from the CUDA path):
  single_sphere_32.json  body velocity of the 42-blob shell at the centre of
                         the 32^3 no-slip box under unit force x and unit
                         torque z (Eqs. LangevinD1-D4, reduced form Eq.
                         incompleteN);
  two_sphere_step0.json  one Split-Euler-Maruyama step (Algorithm 1) of the
                         two-sphere 48x48x32 workload, seed = workload seed,
                         step 0, attempt 0;
  gb_two_sphere_msd_{12,42,162}.json
                         Gibbs-Boltzmann samples (oracle.mcmc) of the tight
                         cavity of Sec. V.A: the covariance of the sphere
                         centres (the long-time MSD limit of Eq. asymRef is
                         twice it) with batch-means errors, and 64 equilibrium
                         configurations to start trajectories from and to
                         average the mobility over (Eq. SErel);
  gb_boomerang.json      Gibbs-Boltzmann samples of the boomerang slit of
                         App. A: densities of the cross-point height and of
                         the angle of its bisector with z, and 64 equilibrium
                         configurations.
Run: python tests/golden/make_golden.py [file names]   (all files: a few
minutes on one core)
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from oracle import saddle, solve, sem, mcmc, rigid  # noqa: E402
import workloads  # noqa: E402


def single_sphere():
    w = workloads.single_sphere_box()
    g = oracle.Grid(w.n, periodic=w.periodic, wall_vel=w.wall_vel)
    b = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
    f = saddle.rhs(g, b, w.eta, F=w.force_torque)
    x = solve.constrained(g, b, w.eta, f)
    U = x[-6:]
    res = np.linalg.norm(saddle.apply(g, b, w.eta, x) - f) / np.linalg.norm(f)
    return {"workload": w.name, "force_torque": w.force_torque.ravel().tolist(), "U": U.tolist(),
            "oracle_rel_residual": float(res),
            "source": "oracle.solve.constrained (dense M = J L^-1 S, N = (K^T M^-1 K)^-1)"}


def two_sphere_step():
    w = workloads.two_sphere_cavity(steps=1)
    g = oracle.Grid(w.n, periodic=w.periodic, wall_vel=w.wall_vel)
    b = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
    out = sem.sem_step(g, b, w.eta, w.kT, w.dt, w.potentials, seed=w.seed, step=0, attempt=0, parts=True)
    return {"workload": w.name, "seed": w.seed, "step": 0, "attempt": 0, "dt": w.dt, "kT": w.kT,
            "q0": w.q.ravel().tolist(), "quat0": w.quat.ravel().tolist(),
            "q": out["q"].ravel().tolist(), "quat": out["quat"].ravel().tolist(),
            "U": out["U"].ravel().tolist(), "U_rfd": out["x_rfd"][-12:].tolist(),
            "F": out["F"].ravel().tolist(), "D_KT": out["D_KT"].tolist(), "reject": bool(out["reject"]),
            "source": "oracle.sem.sem_step"}


def _gb_chain(w, n_samples, thin, step_q, step_rot, seed):
    g = oracle.Grid(w.n, periodic=w.periodic, wall_vel=w.wall_vel, kernel=w.kernel)
    return mcmc.sample(g, w.ref_blobs, w.blob_offsets, w.q, w.quat, w.potentials, w.kT, n_samples=n_samples,
                       thin=thin, burn=2000, step_q=step_q, step_rot=step_rot, seed=seed)


def _starts(qs, ts, count=64):
    idx = np.linspace(0, qs.shape[0] - 1, count).astype(int)
    return {"q": qs[idx].reshape(count, -1).tolist(), "quat": ts[idx].reshape(count, -1).tolist()}


def gb_two_sphere(blobs):
    w = workloads.two_sphere_msd(blobs)
    qs, ts, acc = _gb_chain(w, 40000, 5, 0.25 * w.hydrodynamic_radius / 3.0, 0.4, seed=11 + blobs)
    X = qs.reshape(qs.shape[0], 6)
    cov = np.cov(X.T)
    # batch means: 20 batches of consecutive samples
    nbat = 20
    covs = np.array([np.cov(B.T) for B in np.array_split(X, nbat)])
    err = covs.std(axis=0, ddof=1) / np.sqrt(nbat)
    return {"workload": w.name, "n_samples": int(X.shape[0]), "acceptance": acc,
            "mean_q": X.mean(axis=0).tolist(), "cov_q": cov.tolist(), "cov_q_err": err.tolist(),
            "starts": _starts(qs, ts), "source": "oracle.mcmc.sample (Metropolis, thin 5 sweeps)"}


def gb_boomerang():
    w = workloads.boomerang_slit()
    qs, ts, acc = _gb_chain(w, 100000, 5, 0.6, 0.25, seed=7)
    z = qs[:, 0, 2]
    R = rigid.quat_to_rot(ts[:, 0])
    p_body = -np.array([1.0, 1.0, 0.0]) / np.sqrt(2.0)     # bisector, pointing out of the cross point
    p_lab = R @ p_body
    theta = np.arccos(np.clip(p_lab[:, 2], -1.0, 1.0))
    hz, ez = np.histogram(z, bins=32, range=(0.0, 16.0), density=True)
    ht, et = np.histogram(theta, bins=30, range=(0.0, np.pi), density=True)
    return {"workload": w.name, "n_samples": int(z.size), "acceptance": acc,
            "height_edges": ez.tolist(), "height_density": hz.tolist(),
            "angle_edges": et.tolist(), "angle_density": ht.tolist(),
            "bisector_body_frame": p_body.tolist(), "starts": _starts(qs, ts),
            "source": "oracle.mcmc.sample (Metropolis, thin 5 sweeps)"}


FILES = {"single_sphere_32.json": single_sphere, "two_sphere_step0.json": two_sphere_step,
         "gb_two_sphere_msd_12.json": lambda: gb_two_sphere(12), "gb_two_sphere_msd_42.json": lambda: gb_two_sphere(42),
         "gb_two_sphere_msd_162.json": lambda: gb_two_sphere(162),
         "gb_boomerang.json": gb_boomerang}

if __name__ == "__main__":
    for name in (sys.argv[1:] or list(FILES)):
        t = time.time()
        data = FILES[name]()
        with open(os.path.join(HERE, name), "w") as fh:
            json.dump(data, fh, indent=1)
        print(name, f"{time.time() - t:.1f}s")
