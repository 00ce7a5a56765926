"""Helpers shared by the GPU parity tests: small seeded cases, the oracle
counterparts of their inputs, and the element-wise parity gate."""
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


# Element-wise gates |a_i - b_i| <= rtol |b_i| + floor ||b||_inf, applied per
# block of the saddle layout: every element must match to rtol relative to
# itself, except elements far below the block's largest one, whose rounding
# error is set by the magnitude of the terms summed into them (of the order
# of the block's largest value), not by their own magnitude.
F64_OP = (1e-12, 1e-14)        # single FP64 operators (spread, interpolation, forcing, forces)
F64_MATVEC = (1e-11, 1e-13)    # FP64 saddle matvec
F32_MATVEC = (1e-5, 1e-5)      # FP32 saddle matvec on the same FP32-rounded input
SOLVED = (1e-8, 1e-9)          # solved quantities (GPU to rel. residual 1e-12, oracle direct)
SEM_STEP = (1e-8, 1e-8)        # SEM displacements (three solves and the RFD difference quotients)


def elementwise_err(a, b, floor):
    """max_i |a_i - b_i| / (|b_i| + floor ||b||_inf): the smallest rtol the gate passes with."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    if b.size == 0:
        assert a.size == 0
        return 0.0
    assert a.shape == b.shape
    den = np.abs(b) + floor * np.abs(b).max()
    den = np.where(den > 0, den, 1.0)
    return float(np.max(np.abs(a - b) / den))


def assert_close(a, b, gate, what=""):
    """Element-wise gate = (rtol, atol_frac): |a_i - b_i| <= rtol |b_i| + atol_frac ||b||_inf."""
    rtol, atol_frac = gate
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    assert a.shape == b.shape, what
    assert np.all(np.isfinite(a)), f"{what}: non-finite values"
    lim = rtol * np.abs(b) + atol_frac * (np.abs(b).max() if b.size else 0.0)
    bad = np.abs(a - b) > lim
    if np.any(bad):
        i = int(np.argmax(np.abs(a - b) - lim))
        raise AssertionError(f"{what}: {int(bad.sum())} of {b.size} elements outside the gate "
                             f"(rtol {rtol:g}, floor {atol_frac:g} x max); worst index {i}: "
                             f"got {a[i]!r}, want {b[i]!r}")


def assert_close_blocks(a, b, layout, gate, what=""):
    """assert_close on each block of the saddle layout (offsets of length 7)."""
    names = ["v_x", "v_y", "v_z", "pi", "lambda", "U"]
    for i, nm in enumerate(names):
        assert_close(a[layout[i]:layout[i + 1]], b[layout[i]:layout[i + 1]], gate, f"{what} {nm}")
