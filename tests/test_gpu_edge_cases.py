"""Degenerate and boundary inputs through the C ABI, against the oracle where
there is a result: a grid with no bodies (the saddle system reduces to the
Stokes system; an SEM step has nothing to move), the thinnest grid (two cells
along a wall axis, one unknown face row), blobs exactly on walls and in
corners, and rigid bodies the method cannot represent (a single blob, blobs
on one line), which set_bodies rejects."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import saddle, solve, ib  # noqa: E402
import workloads  # noqa: E402
from gpu_common import assert_close, F64_OP, F64_MATVEC, SOLVED, assert_close_blocks  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_1901_06427_gb300.binding as binding
    binding.lib()
    return binding


def dev(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x).ravel(), dtype=dtype, device="cuda")


def empty_workload(n, periodic=(False, False, False), wall_vel=None):
    w = workloads.Workload(name="empty", n=tuple(n), periodic=tuple(periodic), rtol=1e-12)
    if wall_vel is not None:
        w.wall_vel = np.asarray(wall_vel, dtype=np.float64)
    return w


NO_BODIES = saddle.Bodies(np.zeros((0, 3)), [0], np.zeros((0, 3)), np.zeros((0, 4)))


def test_no_bodies(B):
    wv = np.zeros((6, 3)); wv[5, 0] = 0.3
    w = empty_workload((11, 9, 8), periodic=(True, False, False), wall_vel=wv)
    og = oracle.Grid(w.n, periodic=w.periodic, wall_vel=w.wall_vel)
    g = B.grid_for(w, rtol=1e-12)
    lay = g.layout()
    assert lay[4] == lay[5] == lay[6] == og.N_f + og.N_c
    x = np.random.default_rng(1).standard_normal(g.n_total)
    assert_close_blocks(g.apply_saddle(dev(x)).cpu().numpy(), saddle.apply(og, NO_BODIES, w.eta, x), lay,
                        F64_MATVEC, "matvec without bodies")
    f = np.random.default_rng(2).standard_normal(og.N_f)
    v, pi, info = g.stokes_solve(dev(f))
    v0, p0 = solve.stokes(og, w.eta, f)
    assert_close(v.cpu().numpy(), v0, SOLVED, "Stokes velocity")
    # an SEM step with nothing to move
    q = torch.zeros(0, dtype=torch.float64, device="cuda")
    st, info = g.sem_step(B.sem_params({}, dt=0.05, kT=1.0), 3, 0, 0, q, q.clone())
    assert st == 0 and info["rejected"] == 0


def test_thinnest_grid(B):
    """Two cells along the wall axis x: one row of x-faces."""
    w = workloads.small_case(n=(2, 9, 10), periodic=(False, True, False), n_bodies=0)
    w.bodies = []
    og = oracle.Grid(w.n, periodic=w.periodic)
    g = B.grid_for(w, rtol=1e-12)
    x = np.random.default_rng(3).standard_normal(g.n_total)
    assert_close_blocks(g.apply_saddle(dev(x)).cpu().numpy(), saddle.apply(og, NO_BODIES, w.eta, x), g.layout(),
                        F64_MATVEC, "matvec on a 2-cell axis")
    f = np.random.default_rng(4).standard_normal(og.N_f)
    v, pi, info = g.stokes_solve(dev(f))
    v0, p0 = solve.stokes(og, w.eta, f)
    assert_close(v.cpu().numpy(), v0, SOLVED, "Stokes velocity on a 2-cell axis")


@pytest.mark.parametrize("kernel", [3, 6])
def test_blobs_on_walls_and_corners(B, kernel):
    """Blobs exactly on a wall, on an edge and in a corner of a closed box
    (the kernel's folding at its most degenerate)."""
    n = (10, 9, 8)
    L = np.array(n, dtype=float)
    ref = np.array([[0.0, 0.0, 0.0], [1.3, 0.0, 0.0], [0.0, 1.1, 0.0], [0.0, 0.0, 0.9]])
    w = workloads.Workload(name="corner", n=n, rtol=1e-12, kernel=kernel)
    q = [np.array([0.0, 4.5, 4.0]), np.array([L[0], L[1], 0.0]), np.array([0.0, 0.0, L[2]]), np.array([5.0, 0.0, 4.0])]
    w.bodies = [workloads.Body(ref * (1 if p % 2 == 0 else -1), q[p], np.array([1.0, 0, 0, 0])) for p in range(4)]
    og = oracle.Grid(n, kernel=kernel)
    ob = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
    g = B.grid_for(w)
    rng = np.random.default_rng(5)
    lam = rng.standard_normal(3 * w.n_blobs)
    v = rng.standard_normal(og.N_f)
    r = ob.positions()
    assert_close(g.spread(dev(lam)).cpu().numpy(), ib.spread(og, r, lam), F64_OP, "spread at walls")
    assert_close(g.interpolate(dev(v)).cpu().numpy(), ib.interpolate(og, r, v), F64_OP, "interpolate at walls")


@pytest.mark.parametrize("ref", [[[0.0, 0.0, 0.0]],
                                 [[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]],
                                 [[0.0, 0.0, 0.0], [0.5, 0.5, 0.5], [1.5, 1.5, 1.5]]])
def test_collinear_bodies_are_rejected(B, ref):
    w = empty_workload((10, 10, 10))
    g = B.grid_for(w)
    ref = np.array(ref)
    with pytest.raises(B.RbfibError) as e:
        g.set_bodies(np.array([0, ref.shape[0]]), ref, np.array([[5.0, 5.0, 5.0]]), np.array([[1.0, 0, 0, 0]]))
    assert e.value.code == B.EINVAL
    # a proper body is accepted afterwards
    g.set_bodies(np.array([0, 3]), np.array([[0.0, 0, 0], [1.0, 0, 0], [0, 1.0, 0]]), np.array([[5.0, 5.0, 5.0]]),
                 np.array([[1.0, 0, 0, 0]]))
