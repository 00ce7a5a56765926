"""Write the stored expected values under tests/golden/ with the FP64 oracle.

Every number here comes from oracle/ only (never from the CUDA path):
  single_sphere_32.json  body velocity of the 42-blob shell at the centre of
                         the 32^3 no-slip box under unit force x and unit
                         torque z (Eqs. LangevinD1-D4, reduced form Eq.
                         incompleteN);
  two_sphere_step0.json  one Split-Euler-Maruyama step (Algorithm 1) of the
                         two-sphere 48x48x32 workload, seed = workload seed,
                         step 0, attempt 0.
Run: python tests/golden/make_golden.py   (a few minutes on one core)
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from oracle import saddle, solve, sem  # noqa: E402
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


if __name__ == "__main__":
    for name, fn in [("single_sphere_32.json", single_sphere), ("two_sphere_step0.json", two_sphere_step)]:
        t = time.time()
        data = fn()
        with open(os.path.join(HERE, name), "w") as fh:
            json.dump(data, fh, indent=1)
        print(name, f"{time.time() - t:.1f}s")
