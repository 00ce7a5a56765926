"""Pins of the rigid-body maps, quaternion rotations and the Philox stream."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import rigid, philox, noise, Grid
import workloads


def _bodies(seed=0):
    rng = np.random.default_rng(seed)
    ref = np.concatenate([workloads.shell_12(1.0), workloads.shell_42(2.5)])
    off = np.array([0, 12, 54])
    q = rng.standard_normal((2, 3)) * 5
    quat = rng.standard_normal((2, 4)); quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    return ref, off, q, quat


def test_rotation_matrix_matches_library():
    ref, off, q, quat = _bodies()
    R = rigid.quat_to_rot(quat)
    Rs = Rotation.from_quat(quat[:, [1, 2, 3, 0]]).as_matrix()     # scipy wants (x, y, z, w)
    np.testing.assert_allclose(R, Rs, atol=1e-14)


def test_rotate_is_lab_frame_rotation():
    ref, off, q, quat = _bodies(1)
    phi = np.array([[0.3, -0.2, 0.5], [0.0, 0.0, 0.0]])
    new = rigid.rotate(quat, phi)
    expect = (Rotation.from_rotvec(phi) * Rotation.from_quat(quat[:, [1, 2, 3, 0]])).as_matrix()
    np.testing.assert_allclose(rigid.quat_to_rot(new), expect, atol=1e-14)


def test_K_and_KT_are_adjoint_and_physical():
    ref, off, q, quat = _bodies(2)
    rng = np.random.default_rng(3)
    U = rng.standard_normal(12)
    lam = rng.standard_normal(3 * 54)
    KU = rigid.K_apply(ref, off, quat, U)
    KTl = rigid.KT_apply(ref, off, quat, lam)
    assert abs(np.dot(KU, lam) - np.dot(U, KTl)) < 1e-12 * np.linalg.norm(KU) * np.linalg.norm(lam)
    K = rigid.K_matrix(ref, off, quat)
    np.testing.assert_allclose(K @ U, KU, atol=1e-13)
    np.testing.assert_allclose(K.T @ lam, KTl, atol=1e-12)
    # rigid motion: K U is the velocity u + w x (r - q) of each blob
    r = rigid.blob_positions(ref, off, q, quat)
    bb = rigid.body_of_blob(off)
    Ub = U.reshape(2, 6)
    vel = Ub[bb, :3] + np.cross(Ub[bb, 3:], r - q[bb])
    np.testing.assert_allclose(KU.reshape(-1, 3), vel, atol=1e-13)
    # K^T gives total force and torque about the tracking point
    l3 = lam.reshape(-1, 3)
    for p in range(2):
        s = slice(off[p], off[p + 1])
        np.testing.assert_allclose(KTl.reshape(2, 6)[p, :3], l3[s].sum(axis=0), atol=1e-13)
        np.testing.assert_allclose(KTl.reshape(2, 6)[p, 3:], np.cross(r[s] - q[p], l3[s]).sum(axis=0), atol=1e-12)


def test_body_length():
    ref, off, q, quat = _bodies()
    L = rigid.body_length(ref, off)
    np.testing.assert_allclose(L, [2.0, 5.0], atol=1e-12)     # antipodal blobs of the shells


def test_philox_words_match_numpy():
    """numpy's Philox4x64-10 increments its 256-bit counter before each
    block, so its k-th block uses counter c + k + 1."""
    for key, ctr in [((5, 7), (0, 0, 0, 0)), ((2 ** 64 - 1, 3), (2 ** 64 - 2, 5, 9, 1)),
                     ((0x1234, 0), (41, 17, (3 << 32) | 1, 0))]:
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(ctr, dtype=np.uint64))
        ref = bg.random_raw(12)
        c = np.array(ctr, dtype=object)
        mine = []
        for k in range(3):
            val = sum(int(c[i]) << (64 * i) for i in range(4)) + k + 1
            cc = [(val >> (64 * i)) & (2 ** 64 - 1) for i in range(4)]
            mine.append(philox.philox4x64_10(np.array([cc], dtype=np.uint64), np.array(key, dtype=np.uint64))[0])
        np.testing.assert_array_equal(np.concatenate(mine), ref)


def test_normals_moments_and_layout():
    z = philox.normals(seed=99, step=3, attempt=0, purpose=philox.PURPOSE_FLUID, count=400000)
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / n)
    assert abs(np.mean(z ** 4) - 3) < 5 * np.sqrt(96 / n)
    # lanes of a Box-Muller pair are uncorrelated
    zz = z[: n // 4 * 4].reshape(-1, 4)
    assert abs(np.mean(zz[:, 0] * zz[:, 1])) < 5 / np.sqrt(zz.shape[0])
    # stream separation by purpose / attempt / step
    a = philox.normals(99, 3, 0, philox.PURPOSE_BODY, 16)
    b = philox.normals(99, 3, 1, philox.PURPOSE_BODY, 16)
    c = philox.normals(99, 4, 0, philox.PURPOSE_BODY, 16)
    assert not np.allclose(a, b) and not np.allclose(a, c)
    # the first normals are a prefix of longer draws (counter-based)
    np.testing.assert_array_equal(philox.normals(99, 3, 0, 1, 10), z[:10])


def test_uniform_conversion_open_interval():
    w = np.array([0, 2 ** 64 - 1, 2 ** 63], dtype=np.uint64)
    u = philox.uniforms(w)
    assert u[0] == 2.0 ** -53 and u[1] == 1.0 - 2.0 ** -53 and u[2] == 0.5 + 2.0 ** -53


def test_stress_count_matches_blocks():
    g = Grid((4, 3, 5), periodic=(False, True, False))
    W = noise.stress(g, 1, 2)
    assert W.size == g.N_w == sum(int(np.prod(g.stress_ext(a, b))) for a, b in g.stress_blocks())
