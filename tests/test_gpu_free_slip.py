"""Free-slip walls on the GPU (grid descriptor free_slip; the Introduction's
periodic / no-slip / free-slip combinations) against the oracle: spreading and
interpolation with the even mirror, the fluctuating forcing with zero
wall-edge weights, the saddle matvec in FP64 and FP32 per block (column and
pipelined stencils), the preconditioner's fluid block with exact inner solves
(the fast-diagonalisation bases DCT-II / DST-IV / DCT-IV), the Stokes and
mobility solves in FP64 and FP32-refined (also through the multigrid
V-cycles), one SEM step (Algorithm 1) and the adjoint of the mobility solve,
element by element."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import saddle, solve, ib, noise, sem, operators  # noqa: E402
import workloads  # noqa: E402
from gpu_common import (rel, assert_close, assert_close_blocks, F64_OP, F64_MATVEC, F32_MATVEC,  # noqa: E402
                        SOLVED, SEM_STEP)

pytestmark = pytest.mark.gpu

T, F = True, False
FS_CASES = {
    # x periodic, moving no-slip y walls and z bottom, free-slip top
    "top_free": dict(n=(16, 12, 11), periodic=(T, F, F), n_bodies=3, near_wall=True, wall_speed=0.4,
                     free_slip=(F, F, F, F, F, T)),
    # closed box, free-slip on -x, +y, -z
    "box_mixed": dict(n=(13, 11, 9), periodic=(F, F, F), n_bodies=3, near_wall=True,
                      free_slip=(T, F, F, T, T, F)),
    # x periodic, free-slip y walls, no-slip z walls
    "y_free": dict(n=(16, 10, 9), periodic=(T, F, F), n_bodies=2, near_wall=True, free_slip=(F, F, T, T, F, F)),
    # six-point kernel (12-blob shells of radius 3h: blobs about 3h apart), free-slip bottom
    "k6_bottom": dict(n=(20, 18, 10), periodic=(F, F, F), n_bodies=2, blobs=12, radius=3.0, kernel=6,
                      near_wall=True, free_slip=(F, F, F, F, T, F)),
}


@pytest.fixture(scope="module")
def B():
    import paper_1901_06427_gb300.binding as binding
    binding.lib()
    return binding


def fs_case(name, seed=5):
    w = workloads.small_case(seed=seed, **FS_CASES[name])
    og = oracle.Grid(w.n, periodic=w.periodic, wall_vel=w.wall_vel, kernel=w.kernel, free_slip=w.free_slip)
    ob = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
    return w, og, ob


def dev(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x).ravel(), dtype=dtype, device="cuda")


@pytest.mark.parametrize("name", list(FS_CASES))
def test_spread_interpolate_and_forcing_free_slip(B, name):
    w, og, ob = fs_case(name)
    g = B.grid_for(w)
    rng = np.random.default_rng(1)
    lam = rng.standard_normal(3 * w.n_blobs)
    v = rng.standard_normal(og.N_f)
    r = ob.positions()
    assert_close(g.spread(dev(lam)).cpu().numpy(), ib.spread(og, r, lam), F64_OP, "spread")
    assert_close(g.interpolate(dev(v)).cpu().numpy(), ib.interpolate(og, r, v), F64_OP, "interpolate")
    assert_close(g.interpolate(dev(v), with_walls=True).cpu().numpy(), ib.interpolate(og, r, v, with_walls=True),
                 F64_OP, "interpolate with moving-wall ghosts")
    f = g.stochastic_forcing(1.3, 0.02, 99, 5, 1).cpu().numpy()
    assert_close(f, noise.fluid_forcing(og, w.eta, 1.3, 0.02, 99, 5, 1), F64_OP, "fluid forcing")


@pytest.mark.parametrize("name", list(FS_CASES))
def test_apply_saddle_free_slip(B, name):
    w, og, ob = fs_case(name)
    g = B.grid_for(w)
    x = np.random.default_rng(3).standard_normal(g.n_total)
    assert_close_blocks(g.apply_saddle(dev(x)).cpu().numpy(), saddle.apply(og, ob, w.eta, x), g.layout(),
                        F64_MATVEC, "FP64 matvec")
    x32 = x.astype(np.float32).astype(np.float64)
    y32 = g.apply_saddle(dev(x32, torch.float32)).double().cpu().numpy()
    assert_close_blocks(y32, saddle.apply(og, ob, w.eta, x32), g.layout(), F32_MATVEC, "FP32 matvec")


@pytest.mark.parametrize("periodic,fs", [((F, F, F), (T, F, F, T, T, F)), ((T, F, F), (F, F, T, T, F, T))])
def test_matvec_large_grid_free_slip(B, periodic, fs):
    """Above two million unknowns the pipelined stencil runs; ragged tiles."""
    w = workloads.small_case(n=(100, 90, 76), periodic=periodic, n_bodies=3, blobs=12, seed=1, free_slip=fs)
    g = B.grid_for(w)
    assert g.n_total > 2 * 1024 * 1024
    og = oracle.Grid(w.n, periodic=w.periodic, wall_vel=w.wall_vel, free_slip=w.free_slip)
    ob = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
    x = np.random.default_rng(3).standard_normal(g.n_total)
    assert_close_blocks(g.apply_saddle(dev(x)).cpu().numpy(), saddle.apply(og, ob, w.eta, x), g.layout(),
                        F64_MATVEC, "FP64 matvec")
    x32 = x.astype(np.float32).astype(np.float64)
    y32 = g.apply_saddle(dev(x32, torch.float32)).double().cpu().numpy()
    assert_close_blocks(y32, saddle.apply(og, ob, w.eta, x32), g.layout(), F32_MATVEC, "FP32 matvec")


@pytest.mark.parametrize("name", list(FS_CASES))
def test_preconditioner_fluid_block_exact_free_slip(B, name):
    """On these grids both inner solves of the projection preconditioner are
    exact fast-diagonalisation solves, so its fluid block equals the
    projection method with exact inner solves (FP32)."""
    from scipy.sparse.linalg import cg
    w, og, ob = fs_case(name)
    g = B.grid_for(w)
    lay = g.layout()
    nf, nc = lay[3], lay[4] - lay[3]
    r = np.random.default_rng(11).standard_normal(g.n_total)
    z = g.apply_preconditioner(dev(r)).cpu().numpy()
    vt = solve.viscous_solve(og, w.eta, r[None, :nf])[0]
    D, G = operators.divergence(og), operators.gradient(og)
    q = r[nf:nf + nc] + D @ vt
    phi, info = cg(-(D @ G), q - q.mean(), rtol=1e-13, maxiter=20000)
    assert info == 0
    assert rel(z[:nf], vt + G @ phi) < 1e-4
    assert rel(z[nf:nf + nc], -w.eta * q) < 1e-4


@pytest.mark.parametrize("name", ["top_free", "y_free"])
def test_stokes_solve_free_slip(B, name):
    w, og, ob = fs_case(name)
    g = B.grid_for(w, rtol=1e-12)
    f = np.random.default_rng(5).standard_normal(og.N_f)
    v, pi, info = g.stokes_solve(dev(f))
    v0, p0 = solve.stokes(og, w.eta, f)
    assert info["rel_residual"] <= 1e-12
    assert_close(v.cpu().numpy(), v0, SOLVED, "Stokes velocity")
    assert_close(pi.cpu().numpy(), p0, SOLVED, "Stokes pressure")


@pytest.mark.parametrize("name,precision", [("top_free", "fp64"), ("box_mixed", "fp64"), ("y_free", "refined"),
                                            ("k6_bottom", "fp64")])
def test_mobility_solve_free_slip(B, name, precision):
    w, og, ob = fs_case(name)
    prec = B.FP64 if precision == "fp64" else B.FP32_REFINED
    g = B.grid_for(w, precision=prec, rtol=1e-12 if precision == "fp64" else 1e-11)
    U, info, x = g.mobility_solve(dev(w.force_torque), slip=dev(w.slip), return_x=True)
    f = saddle.rhs(og, ob, w.eta, F=w.force_torque, slip=w.slip)
    x0 = solve.constrained(og, ob, w.eta, f)
    gate = SOLVED if precision == "fp64" else (1e-7, 1e-8)
    assert_close(U.cpu().numpy(), x0[-6 * w.n_bodies:], gate, f"U ({precision})")
    assert_close_blocks(x.cpu().numpy(), x0, g.layout(), gate if precision == "fp64" else (1e-6, 1e-7),
                        f"solution ({precision})")


def test_mobility_solve_free_slip_multigrid(B):
    """A grid with more than 48 points along x: the preconditioner runs red-
    black V-cycles with the free-slip ghosts in the smoothers and transfers
    down to an exact coarse solve."""
    w = workloads.small_case(n=(64, 16, 12), periodic=(F, T, F), n_bodies=2, blobs=12, seed=3, near_wall=True,
                             free_slip=(T, F, F, F, F, T))
    og = oracle.Grid(w.n, periodic=w.periodic, wall_vel=w.wall_vel, free_slip=w.free_slip)
    ob = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
    for prec, gate in ((B.FP64, SOLVED), (B.FP32_REFINED, (1e-7, 1e-8))):
        g = B.grid_for(w, precision=prec, rtol=1e-12 if prec == B.FP64 else 1e-11)
        U, info = g.mobility_solve(dev(w.force_torque))
        x0 = solve.constrained(og, ob, w.eta, saddle.rhs(og, ob, w.eta, F=w.force_torque))
        assert_close(U.cpu().numpy(), x0[-6 * w.n_bodies:], gate, f"U (multigrid, precision {prec})")


@pytest.mark.parametrize("name", ["top_free", "box_mixed"])
def test_sem_step_free_slip(B, name):
    w, og, ob = fs_case(name)
    g = B.grid_for(w, rtol=1e-12)
    q, quat = dev(w.q), dev(w.quat)
    st, info = g.sem_step(B.sem_params(w.potentials, dt=0.05, kT=1.0), 11, 2, 1, q, quat)
    ref = sem.sem_step(og, ob, w.eta, 1.0, 0.05, w.potentials, seed=11, step=2, attempt=1)
    assert st == 0 and not ref["reject"]
    assert_close(q.cpu().numpy().reshape(-1, 3) - w.q, ref["q"] - w.q, SEM_STEP, "SEM displacement")
    assert_close(quat.cpu().numpy() - w.quat.ravel(), ref["quat"].ravel() - w.quat.ravel(), SEM_STEP,
                 "SEM orientation increment")


def test_adjoint_free_slip(B):
    """Gradient of sum |U|^2 with respect to blob positions and slip next to
    free-slip walls (the even mirror in the kernel derivative) against the
    oracle's adjoint."""
    from oracle import adjoint
    w = workloads.small_case(n=(12, 10, 9), n_bodies=2, blobs=12, radius=1.0, seed=9, near_wall=True,
                             free_slip=(T, F, F, T, T, F))
    og = oracle.Grid(w.n, free_slip=w.free_slip)
    ob = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
    x0, U0 = adjoint.forward(og, ob, w.eta, w.slip.ravel(), w.force_torque)
    dr0, ds0 = adjoint.gradient(og, ob, w.eta, x0, 2.0 * U0)
    g = B.grid_for(w, rtol=1e-12)
    U, info, x = g.mobility_solve(dev(w.force_torque), slip=dev(w.slip), return_x=True)
    assert_close(U.cpu().numpy(), U0, SOLVED, "U")
    dr, ds, ainfo = g.mobility_solve_adjoint(2.0 * U, x)
    assert_close(dr.cpu().numpy(), dr0.ravel(), (1e-7, 1e-8), "dL/dr")
    assert_close(ds.cpu().numpy(), ds0, (1e-7, 1e-8), "dL/dslip")


def test_free_slip_descriptor_errors(B):
    """A velocity component with no no-slip wall, a moving free-slip wall and
    a flag other than 0 / 1 are rejected."""
    import ctypes
    bad = []
    d = B._desc((8, 8, 8), periodic=(F, T, T), free_slip=(T, T, F, F, F, F))
    bad.append(d)
    wv = np.zeros((6, 3)); wv[5, 0] = 0.3
    bad.append(B._desc((8, 8, 8), periodic=(T, T, F), wall_vel=wv, free_slip=(F, F, F, F, F, T)))
    d = B._desc((8, 8, 8))
    d.free_slip[2] = 2
    bad.append(d)
    for d in bad:
        h = ctypes.c_void_p()
        assert B.lib().rbfib_create_grid(ctypes.byref(d), None, ctypes.byref(h)) == B.EINVAL
