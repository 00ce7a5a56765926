"""Helpers shared by the GPU parity tests: small seeded cases and the oracle
counterparts of their inputs."""
import numpy as np

import oracle
from oracle import saddle
import workloads

CASES = {
    "walls": dict(n=(13, 11, 9), periodic=(False, False, False), n_bodies=3, near_wall=True),
    "xper_moving": dict(n=(16, 10, 9), periodic=(True, False, False), n_bodies=3, near_wall=True, wall_speed=0.4),
    "yzper": dict(n=(9, 12, 14), periodic=(False, True, True), n_bodies=2, near_wall=False),
    "ragged42": dict(n=(17, 15, 11), periodic=(False, False, False), n_bodies=2, blobs=42, radius=2.5),
}


def case(name, seed=5):
    kw = dict(CASES[name])
    w = workloads.small_case(seed=seed, **kw)
    og = oracle.Grid(w.n, periodic=w.periodic, wall_vel=w.wall_vel)
    ob = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
    return w, og, ob


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
