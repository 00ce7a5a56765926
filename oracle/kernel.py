"""Immersed-boundary kernels phi (r in grid units) of the regularised delta
delta_h(x) = phi(x/h) phi(y/h) phi(z/h) / h^3 used by the spreading and
interpolation operators of Sec. III.B: the three-point Peskin kernel and the
six-point kernel with three continuous derivatives that the paper uses
(Sec. III.B, Sec. V).

Three-point kernel.

phi is the unique function supported on |r| < 3/2 with, for every shift s,
  sum_j phi(s - j) = 1,  sum_j (s - j) phi(s - j) = 0,  sum_j phi(s - j)^2 = 1/2.
Solving these gives the closed form below; it is C^1 (phi'(1/2) = -1 from
both sides, phi'(3/2) = 0).
"""
import numpy as np


def phi(r):
    r = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(r)
    inner = r <= 0.5
    outer = (r > 0.5) & (r < 1.5)
    out[inner] = (1.0 + np.sqrt(1.0 - 3.0 * r[inner] ** 2)) / 3.0
    ro = r[outer]
    out[outer] = (5.0 - 3.0 * ro - np.sqrt(1.0 - 3.0 * (1.0 - ro) ** 2)) / 6.0
    return out


def dphi(r):
    """Derivative phi'(r) (odd in r)."""
    r = np.asarray(r, dtype=np.float64)
    a = np.abs(r)
    s = np.sign(r)
    out = np.zeros_like(a)
    inner = a <= 0.5
    outer = (a > 0.5) & (a < 1.5)
    ai = a[inner]
    out[inner] = -ai / np.sqrt(1.0 - 3.0 * ai ** 2)
    ao = a[outer]
    out[outer] = (-3.0 - 3.0 * (1.0 - ao) / np.sqrt(1.0 - 3.0 * (1.0 - ao) ** 2)) / 6.0
    return s * out


# ---------------------------------------------------------------- six-point
# The six-point kernel (support |r| < 3) of the paper's Sec. III.B (its cited
# construction; the paper gives no formula).  It is defined by conditions on
# the six weights phi(r - j), j = -2..3, at every shift r in [0, 1):
#   sum over even j = sum over odd j = 1/2,
#   sum (r - j) phi = 0,  sum (r - j)^2 phi = K,  sum (r - j)^3 phi = 0,
#   sum phi^2 = C,
# with K = 59/60 - sqrt(29)/20 (the value that makes phi three times
# continuously differentiable) and C fixed by phi(+-3) = 0.  Solving the five
# linear conditions for the other weights in terms of t = phi(r - 3) (our
# derivation; the pins in tests/test_oracle_kernel6.py re-solve the system
# numerically and check the smoothness):
#   phi(r - 2) = r^3/12 + r^2/8 + (13 - sqrt29) r / 80 + 29/480 - sqrt29/160 - 3 t
#   phi(r - 1) = -r^3/6 + (7 + sqrt29) r / 40 + 1/4 + 2 t
#   phi(r)     = -r^2/4 + 91/240 + sqrt29/80 + 2 t
#   phi(r + 1) = r^3/6 - (7 + sqrt29) r / 40 + 1/4 - 3 t
#   phi(r + 2) = -r^3/12 + r^2/8 - (13 - sqrt29) r / 80 + 29/480 - sqrt29/160 + t
# and sum phi^2 = C becomes 28 t^2 + beta t + gamma = 0 with
#   beta  = -7 r^3/3 - 3 r^2/2 + (9 + 7 sqrt29) r / 20 + (31 + 3 sqrt29) / 40,
#   gamma = 5 r^6/72 + (1/32 - sqrt29/48) r^4,
# C = 5431/19200 + 51 sqrt29/6400; t is the root that vanishes at r = 0,
# t = -2 gamma / (beta + sqrt(beta^2 - 112 gamma)).
SQRT29 = np.sqrt(29.0)
K6 = 59.0 / 60.0 - SQRT29 / 20.0
C6 = 5431.0 / 19200.0 + 51.0 * SQRT29 / 6400.0


def _six_weights(r):
    """The six weights phi(r - j), j = -2..3, for r in [0, 1) (array (..., 6))
    and their derivatives with respect to r."""
    r = np.asarray(r, dtype=np.float64)
    beta = -7.0 * r ** 3 / 3.0 - 1.5 * r ** 2 + (9.0 + 7.0 * SQRT29) * r / 20.0 + (31.0 + 3.0 * SQRT29) / 40.0
    gamma = 5.0 * r ** 6 / 72.0 + (1.0 / 32.0 - SQRT29 / 48.0) * r ** 4
    root = np.sqrt(beta ** 2 - 112.0 * gamma)
    t = -2.0 * gamma / (beta + root)
    dbeta = -7.0 * r ** 2 - 3.0 * r + (9.0 + 7.0 * SQRT29) / 20.0
    dgamma = 5.0 * r ** 5 / 12.0 + 4.0 * (1.0 / 32.0 - SQRT29 / 48.0) * r ** 3
    dt = -(dbeta * t + dgamma) / (56.0 * t + beta)
    c1 = (13.0 - SQRT29) / 80.0
    c2 = (7.0 + SQRT29) / 40.0
    c0 = 29.0 / 480.0 - SQRT29 / 160.0
    w = np.stack([
        -r ** 3 / 12.0 + r ** 2 / 8.0 - c1 * r + c0 + t,          # phi(r + 2)
        r ** 3 / 6.0 - c2 * r + 0.25 - 3.0 * t,                   # phi(r + 1)
        -r ** 2 / 4.0 + 91.0 / 240.0 + SQRT29 / 80.0 + 2.0 * t,   # phi(r)
        -r ** 3 / 6.0 + c2 * r + 0.25 + 2.0 * t,                  # phi(r - 1)
        r ** 3 / 12.0 + r ** 2 / 8.0 + c1 * r + c0 - 3.0 * t,     # phi(r - 2)
        t,                                                        # phi(r - 3)
    ], axis=-1)
    dw = np.stack([
        -r ** 2 / 4.0 + r / 4.0 - c1 + dt,
        r ** 2 / 2.0 - c2 - 3.0 * dt,
        -r / 2.0 + 2.0 * dt,
        -r ** 2 / 2.0 + c2 + 2.0 * dt,
        r ** 2 / 4.0 + r / 4.0 + c1 - 3.0 * dt,
        dt,
    ], axis=-1)
    return w, dw


def phi6(x):
    """The six-point kernel at x (support |x| < 3)."""
    x = np.asarray(x, dtype=np.float64)
    fl = np.floor(x)
    r = x - fl                      # x = r - j with j = -fl
    j = (-fl).astype(np.int64)
    w, _ = _six_weights(r)
    inside = (j >= -2) & (j <= 3)
    col = np.clip(j + 2, 0, 5)
    out = np.take_along_axis(w, col[..., None], axis=-1)[..., 0]
    return np.where(inside, out, 0.0)


def dphi6(x):
    """phi6'(x)."""
    x = np.asarray(x, dtype=np.float64)
    fl = np.floor(x)
    r = x - fl
    j = (-fl).astype(np.int64)
    _, dw = _six_weights(r)
    inside = (j >= -2) & (j <= 3)
    col = np.clip(j + 2, 0, 5)
    out = np.take_along_axis(dw, col[..., None], axis=-1)[..., 0]
    return np.where(inside, out, 0.0)


def kernel(width):
    """(phi, phi', points per axis, first point offset) of a kernel width 3 or 6:
    the points of a coordinate s (grid units) are p = p0(s) + 0..width-1 with
    p0 = floor(s + 1/2) - 1 (three points) or floor(s) - 2 (six points)."""
    if width == 3:
        return phi, dphi, 3, lambda s: np.floor(s + 0.5).astype(np.int64) - 1
    if width == 6:
        return phi6, dphi6, 6, lambda s: np.floor(s).astype(np.int64) - 2
    raise ValueError("kernel width must be 3 or 6")
