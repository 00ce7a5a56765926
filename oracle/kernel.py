"""Three-point Peskin kernel phi (support |r| < 3/2, r in grid units), the
regularised delta delta_h(x) = phi(x/h) phi(y/h) phi(z/h) / h^3 used by the
spreading and interpolation operators of Sec. III.B.

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
