"""Discrete fluctuation-dissipation balance of the whole GPU SEM step
(Algorithm 1): over many independent random streams from one configuration,
the covariance of the one-step displacements of two bodies (translations and
lab-frame rotation angles) is 2 kT dt N, N the body mobility the GPU's own
deterministic solves give (the short-time limit of the self- and
cross-mean-square displacements of Sec. V.A; Eqs. LangevinD1-D4 with the
stochastic stress of Eq. LangevinD1).  Checked entry by entry within five
standard deviations of the sample covariance (Wishart variance)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_1901_06427_gb300.binding as binding
    binding.lib()
    return binding


def _rotation_angles(q0, q1):
    """Lab-frame rotation vector phi with q1 = q(phi) (x) q0 (unit quaternions
    (w, x, y, z)), per body."""
    out = []
    for a, b in zip(q0.reshape(-1, 4), q1.reshape(-1, 4)):
        w0, v0 = a[0], a[1:]
        w1, v1 = b[0], b[1:]
        # r = q1 (x) conj(q0)
        wr = w1 * w0 + v1 @ v0
        vr = -w1 * v0 + w0 * v1 - np.cross(v1, v0)
        if wr < 0:
            wr, vr = -wr, -vr
        s = np.linalg.norm(vr)
        ang = 2.0 * np.arctan2(s, wr)
        out.append(vr * (ang / s) if s > 0 else np.zeros(3))
    return np.concatenate(out)


def test_step_covariance_is_2kT_dt_N(B):
    w = workloads.small_case(n=(14, 12, 12), n_bodies=2, blobs=12, radius=1.0, seed=31)
    w.potentials = {}
    dt, kT, samples = 1e-3, 1.0, 4000
    g = B.grid_for(w, rtol=1e-10)
    nb = w.n_bodies
    # deterministic body mobility from unit forces and torques
    N = np.zeros((6 * nb, 6 * nb))
    for k in range(6 * nb):
        F = np.zeros(6 * nb)
        F[k] = 1.0
        U, _ = g.mobility_solve(torch.tensor(F, device="cuda"))
        N[:, k] = U.cpu().numpy()
    q0 = torch.tensor(w.q.ravel(), device="cuda")
    t0 = torch.tensor(w.quat.ravel(), device="cuda")
    q = q0.clone()
    quat = t0.clone()
    p = B.sem_params({}, dt=dt, kT=kT)
    X = np.empty((samples, 6 * nb))
    for s in range(samples):
        q.copy_(q0)
        quat.copy_(t0)
        st, info = g.sem_step(p, 777, s, 0, q, quat)
        assert st == 0
        dq = (q.cpu().numpy() - w.q.ravel()).reshape(nb, 3)
        dth = _rotation_angles(w.quat.ravel(), quat.cpu().numpy()).reshape(nb, 3)
        X[s] = np.concatenate([np.concatenate([dq[b], dth[b]]) for b in range(nb)])
    C = (X - X.mean(axis=0)).T @ (X - X.mean(axis=0)) / (samples - 1) / dt
    target = 2.0 * kT * N
    sd = np.sqrt((np.outer(np.diag(target), np.diag(target)) + target ** 2) / samples)
    z = np.abs(C - target) / sd
    assert np.all(z < 5.0), f"max |C - 2kT N| / sigma = {z.max():.2f}"
    # the sample resolves the hydrodynamic coupling of the two bodies (about
    # 8 standard deviations here), not only the self terms
    assert np.abs(target[:6, 6:]).max() > 5 * sd[:6, 6:].max()
