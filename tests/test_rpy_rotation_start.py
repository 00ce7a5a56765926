"""The facts behind the coupled body block's update from one configuration to
the next, checked on the CPU with an RPY mobility written out here.
- The RPY tensor is rotation-covariant: rotating a body's blobs rigidly about
  its centre by D turns its intra-body blocks into D M_ij D^T exactly.
- For a single body, D X D^T is then the exact inverse of the rotated M.
- On the two-sphere geometry (42-blob spheres of radius 2.5h, 6h apart)
  moved by one free-space SEM step (rotations of 0.016 rad and translations
  of 0.046 h per axis, the Brownian scales), rotating the previous inverse
  body by body cuts the start residual ||I - M X0||_F by at least a fifth.
  It is not zero, because the inter-body blocks change too.
- Eight Newton-Schulz steps from that start reach roundoff in every draw.
  That includes draws whose ||I - M X0||_F exceeds 1: the iteration needs
  only a spectral radius below 1.  The Frobenius bound of 0.95 that the
  update accepts is therefore conservative."""
import numpy as np
from scipy.spatial.transform import Rotation

import workloads


def rpy(r, a=0.91, eta=1.0):
    """Dense free-space RPY mobility of blobs at r (n x 3), radius a."""
    n = len(r)
    M = np.zeros((3 * n, 3 * n))
    c0 = 1.0 / (6.0 * np.pi * eta * a)
    for i in range(n):
        M[3 * i:3 * i + 3, 3 * i:3 * i + 3] = c0 * np.eye(3)
        for j in range(n):
            if i == j:
                continue
            d = r[i] - r[j]
            rr = np.linalg.norm(d)
            dd = np.outer(d, d) / rr ** 2
            if rr >= 2 * a:
                c = 1.0 / (8.0 * np.pi * eta * rr)
                blk = c * ((1 + 2 * a * a / (3 * rr * rr)) * np.eye(3) + (1 - 2 * a * a / (rr * rr)) * dd)
            else:
                blk = c0 * ((1 - 9 * rr / (32 * a)) * np.eye(3) + (3 * rr / (32 * a)) * dd)
            M[3 * i:3 * i + 3, 3 * j:3 * j + 3] = blk
    return M


def _bodies(rng, centres, blobs=12, radius=1.0):
    shell = workloads.icosahedral_shell(blobs, radius)
    R = [Rotation.random(random_state=rng).as_matrix() for _ in centres]
    return shell, R


def _positions(shell, centres, R):
    return np.concatenate([c + shell @ Rk.T for c, Rk in zip(centres, R)])


def _rotate_inverse(X, D, blobs):
    """X_ij <- D_b(i) X_ij D_b(j)^T for 3 x 3 blocks, b = body of the blob."""
    n = X.shape[0] // 3
    body = np.repeat(np.arange(len(D)), blobs)
    Y = X.copy()
    for i in range(n):
        for j in range(n):
            Y[3 * i:3 * i + 3, 3 * j:3 * j + 3] = D[body[i]] @ X[3 * i:3 * i + 3, 3 * j:3 * j + 3] @ D[body[j]].T
    return Y


def test_intra_body_blocks_are_rotation_covariant():
    rng = np.random.default_rng(3)
    shell, R = _bodies(rng, [np.zeros(3)])
    D = Rotation.from_rotvec(rng.normal(size=3) * 0.3).as_matrix()
    M0 = rpy(_positions(shell, [np.zeros(3)], R))
    M1 = rpy(_positions(shell, [np.zeros(3)], [D @ R[0]]))
    Q = np.kron(np.eye(len(shell)), D)
    assert np.abs(M1 - Q @ M0 @ Q.T).max() < 1e-14 * np.abs(M0).max()
    # one body: the rotated inverse is the inverse of the rotated matrix
    X1 = _rotate_inverse(np.linalg.inv(M0), [D], len(shell))
    assert np.abs(X1 @ M1 - np.eye(len(M1))).max() < 1e-10


def test_rotated_start_on_two_sphere_step_converges():
    rng = np.random.default_rng(1)
    shell = workloads.icosahedral_shell(42, 2.5)
    centres = [np.zeros(3), np.array([6.0, 0.0, 0.0])]
    R = [Rotation.random(random_state=rng).as_matrix() for _ in centres]
    M0 = rpy(_positions(shell, centres, R))
    X0 = np.linalg.inv(M0)
    for seed in range(4):
        mv = np.random.default_rng(10 + seed)
        D = [Rotation.from_rotvec(mv.normal(size=3) * 0.016).as_matrix() for _ in centres]
        moved = [c + mv.normal(size=3) * 0.046 for c in centres]
        M1 = rpy(_positions(shell, moved, [Dk @ Rk for Dk, Rk in zip(D, R)]))
        I = np.eye(len(M1))
        r_plain = np.linalg.norm(I - M1 @ X0)
        X = _rotate_inverse(X0, D, len(shell))
        r_rot = np.linalg.norm(I - M1 @ X)
        assert r_rot < 0.8 * r_plain, (seed, r_rot, r_plain)
        for _ in range(8):
            X = X + X @ (I - M1 @ X)
        assert np.linalg.norm(I - M1 @ X) < 1e-10, seed
