"""Rigid-body kinematics: body geometry, the geometric matrix K of Sec. III.B
and the quaternion rotation used for orientation updates (Algorithm 1 steps 3
and 7).

Reading: a rigid body with angular velocity w moves a point r at
u + w x (r - q).  K U = u + w x (r - q) is then the adjoint of the force/torque
map K^T lambda = [sum lambda; sum (r - q) x lambda] printed in Sec. III.B
(the printed (r - q) x w is taken as the same map written with reversed
cross-product order; only this form makes K and K^T transposes).
"""
import numpy as np


def quat_to_rot(quat):
    """Rotation matrices (N, 3, 3) of unit quaternions (N, 4), (w, x, y, z)."""
    q = np.asarray(quat, dtype=np.float64).reshape(-1, 4)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.empty((q.shape[0], 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z); R[:, 0, 1] = 2 * (x * y - w * z); R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z); R[:, 1, 1] = 1 - 2 * (x * x + z * z); R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y); R[:, 2, 1] = 2 * (y * z + w * x); R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def quat_mul(p, q):
    """Hamilton product p * q for (N, 4) arrays."""
    p = np.asarray(p, dtype=np.float64).reshape(-1, 4)
    q = np.asarray(q, dtype=np.float64).reshape(-1, 4)
    w1, x1, y1, z1 = p.T
    w2, x2, y2, z2 = q.T
    return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], axis=1)


def rotate(quat, angle_vec):
    """Rotate(theta, phi): the orientation after a lab-frame rotation by the
    oriented angle phi (|phi| radians about phi/|phi|), renormalised."""
    phi = np.asarray(angle_vec, dtype=np.float64).reshape(-1, 3)
    ang = np.linalg.norm(phi, axis=1)
    half = 0.5 * ang
    s = np.where(ang > 0, np.sin(half) / np.where(ang > 0, ang, 1.0), 0.5)
    dq = np.concatenate([np.cos(half)[:, None], s[:, None] * phi], axis=1)
    out = quat_mul(dq, quat)
    return out / np.linalg.norm(out, axis=1, keepdims=True)


def body_of_blob(offsets):
    off = np.asarray(offsets)
    return np.repeat(np.arange(off.size - 1), np.diff(off))


def blob_positions(ref, offsets, q, quat):
    """r_i = q_p + R(theta_p) r_i^ref for every blob i of body p."""
    R = quat_to_rot(quat)
    bb = body_of_blob(offsets)
    return np.asarray(q)[bb] + np.einsum("nij,nj->ni", R[bb], np.asarray(ref))


def arms(ref, offsets, quat):
    """r_i - q_p = R(theta_p) r_i^ref."""
    R = quat_to_rot(quat)
    bb = body_of_blob(offsets)
    return np.einsum("nij,nj->ni", R[bb], np.asarray(ref))


def body_length(ref, offsets):
    """L_p: maximum pairwise distance between the blobs of body p (Sec. IV.B)."""
    off = np.asarray(offsets)
    out = np.zeros(off.size - 1)
    for p in range(off.size - 1):
        r = np.asarray(ref)[off[p]:off[p + 1]]
        if r.shape[0] > 1:
            out[p] = np.max(np.linalg.norm(r[:, None, :] - r[None, :, :], axis=2))
    return out


def K_matrix(ref, offsets, quat):
    """K as a dense (3 N_bl, 6 N_b) array: (K U)_i = u_p + w_p x (r_i - q_p)."""
    return K_matrix_arms(arms(ref, offsets, quat), offsets)


def K_matrix_arms(d, offsets):
    bb = body_of_blob(offsets)
    nbl, nb = d.shape[0], len(offsets) - 1
    K = np.zeros((3 * nbl, 6 * nb))
    for i in range(nbl):
        p = bb[i]
        K[3 * i:3 * i + 3, 6 * p:6 * p + 3] = np.eye(3)
        dx, dy, dz = d[i]
        # w x d = -[d]_x w
        K[3 * i:3 * i + 3, 6 * p + 3:6 * p + 6] = -np.array([[0, -dz, dy], [dz, 0, -dx], [-dy, dx, 0]])
    return K


def K_apply(ref, offsets, quat, U):
    return K_apply_arms(arms(ref, offsets, quat), offsets, U)


def K_apply_arms(d, offsets, U):
    bb = body_of_blob(offsets)
    U = np.asarray(U).reshape(-1, 6)
    return (U[bb, :3] + np.cross(U[bb, 3:], d)).ravel()


def KT_apply(ref, offsets, quat, lam):
    """K^T lambda = [sum_i lambda_i ; sum_i (r_i - q) x lambda_i] per body."""
    return KT_apply_arms(arms(ref, offsets, quat), offsets, lam)


def KT_apply_arms(d, offsets, lam):
    bb = body_of_blob(offsets)
    lam = np.asarray(lam).reshape(-1, 3)
    nb = len(offsets) - 1
    out = np.zeros((nb, 6))
    np.add.at(out[:, :3], bb, lam)
    np.add.at(out[:, 3:], bb, np.cross(d, lam))
    return out.ravel()
