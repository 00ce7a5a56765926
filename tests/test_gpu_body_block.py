"""The coupled body block of the preconditioner after a move (C ABI
rbfib_set_blob_positions, rbfib_body_block_info): its inverse RPY matrix,
updated by Newton-Schulz steps from the previous configuration's inverse,
matches a Gauss-Jordan inverse built from scratch for the moved bodies.  The
two grids' preconditioner outputs agree to the FP32 accuracy of the
inverse, for a small move (warm start taken) and a large one."""
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


def _rotate_about_z(quat, angle):
    """Left-multiply each (w, x, y, z) quaternion by a rotation about z."""
    c, s = np.cos(0.5 * angle), np.sin(0.5 * angle)
    w, x, y, z = quat[:, 0], quat[:, 1], quat[:, 2], quat[:, 3]
    return np.stack([c * w - s * z, c * x - s * y, c * y + s * x, c * z + s * w], axis=1)


def _grid(B, w, quat):
    g = B.Grid(w.n, h=w.h, eta=w.eta, periodic=w.periodic, wall_vel=w.wall_vel, precision=B.FP64, rtol=1e-8)
    g.set_bodies(w.blob_offsets, w.ref_blobs, w.q, quat)
    return g


@pytest.mark.parametrize("angle", [0.02, 1.2])
def test_moved_body_block_matches_fresh_build(B, angle):
    w = workloads.small_case(n=(16, 16, 16), n_bodies=3, blobs=12, seed=53)
    quat0 = np.asarray(w.quat, dtype=np.float64).reshape(-1, 4)
    quat1 = _rotate_about_z(quat0, angle)
    ga = _grid(B, w, quat0)          # Gauss-Jordan at the first configuration
    gb = _grid(B, w, quat1)          # Gauss-Jordan at the moved configuration
    dense, warm0 = ga.body_block_info()
    assert dense
    ga.set_blob_positions(gb.blob_positions())   # rebuilt from ga's inverse
    _, warm1 = ga.body_block_info()
    if angle < 0.1:
        assert warm1 == warm0 + 1
    n = ga.n_total
    gen = torch.Generator(device="cuda").manual_seed(7)
    r = torch.randn(n, dtype=torch.float64, device="cuda", generator=gen)
    za = ga.apply_preconditioner(r)
    zb = gb.apply_preconditioner(r)
    torch.cuda.synchronize()
    lay = ga.layout()
    body = slice(lay[4], lay[6])     # lambda and U rows: where the body block acts
    rel = (torch.linalg.norm(za[body] - zb[body]) / torch.linalg.norm(zb[body])).item()
    assert rel < 2e-3, rel
    rel_all = (torch.linalg.norm(za - zb) / torch.linalg.norm(zb)).item()
    assert rel_all < 2e-3, rel_all
    ga.close()
    gb.close()
