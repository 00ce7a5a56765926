"""Counter-based Philox4x64-10 generator (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC11), written from its published
definition with numpy uint64 arithmetic, plus the uniform and Box-Muller
normal conversions used for every random draw of the method.

Stream layout (shared interface with the CUDA library):
  key     = (seed, 0)
  counter = (block, step, (attempt << 32) | purpose, 0)
  normal number g of a stream is lane g % 4 of block g // 4; lanes (0, 1) and
  (2, 3) are Box-Muller pairs of the block's four uniforms.
  u = (2 (word >> 12) + 1) * 2^-53  (exact, in (0, 1));  (n0, n1) = sqrt(-2 ln u0) (cos 2pi u1, sin 2pi u1)
Purposes: 1 = fluid stochastic stress W, 2 = body RFD forces (W^f, W^tau).
"""
import numpy as np

M0 = np.uint64(0xD2E7470EE14C6C93)
M1 = np.uint64(0xCA5A826395121157)
W0 = np.uint64(0x9E3779B97F4A7C15)
W1 = np.uint64(0xBB67AE8584CAA73B)
MASK32 = np.uint64(0xFFFFFFFF)
S32 = np.uint64(32)

PURPOSE_FLUID = 1
PURPOSE_BODY = 2


def mulhilo(a, b):
    """Full 128-bit product of uint64 arrays: (hi, lo)."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    a0, a1 = a & MASK32, a >> S32
    b0, b1 = b & MASK32, b >> S32
    p00, p01, p10, p11 = a0 * b0, a0 * b1, a1 * b0, a1 * b1
    mid = (p00 >> S32) + (p01 & MASK32) + (p10 & MASK32)
    hi = p11 + (p01 >> S32) + (p10 >> S32) + (mid >> S32)
    with np.errstate(over="ignore"):
        lo = a * b
    return hi, lo


def philox4x64_10(ctr, key):
    """ctr: (N, 4) uint64, key: (2,) uint64 -> (N, 4) uint64 random words."""
    c = np.array(ctr, dtype=np.uint64).reshape(-1, 4).copy()
    k0 = np.uint64(key[0])
    k1 = np.uint64(key[1])
    with np.errstate(over="ignore"):
        for rnd in range(10):
            if rnd > 0:
                k0 = k0 + W0
                k1 = k1 + W1
            hi0, lo0 = mulhilo(M0, c[:, 0])
            hi1, lo1 = mulhilo(M1, c[:, 2])
            c = np.stack([hi1 ^ c[:, 1] ^ k0, lo1, hi0 ^ c[:, 3] ^ k1, lo0], axis=1)
    return c


def words(seed, step, attempt, purpose, n_blocks, first_block=0):
    blocks = np.arange(first_block, first_block + n_blocks, dtype=np.uint64)
    ctr = np.zeros((n_blocks, 4), dtype=np.uint64)
    ctr[:, 0] = blocks
    ctr[:, 1] = np.uint64(step)
    ctr[:, 2] = (np.uint64(attempt) << np.uint64(32)) | np.uint64(purpose)
    return philox4x64_10(ctr, (np.uint64(seed), np.uint64(0)))


def uniforms(w):
    """Odd multiples of 2^-53: every value is exact and lies in (0, 1)."""
    k = (w >> np.uint64(12)) * np.uint64(2) + np.uint64(1)
    return k.astype(np.float64) * (2.0 ** -53)


def normals(seed, step, attempt, purpose, count):
    """The first ``count`` standard normals of a stream."""
    nb = (count + 3) // 4
    u = uniforms(words(seed, step, attempt, purpose, nb))
    out = np.empty((nb, 4))
    for pa, pb in ((0, 1), (2, 3)):
        rad = np.sqrt(-2.0 * np.log(u[:, pa]))
        ang = 2.0 * np.pi * u[:, pb]
        out[:, pa] = rad * np.cos(ang)
        out[:, pb] = rad * np.sin(ang)
    return out.ravel()[:count]
