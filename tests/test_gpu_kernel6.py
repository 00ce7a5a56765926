"""The paper's six-point kernel (Sec. III.B; grid descriptor kernel = 6) on the
GPU against the oracle: spreading and interpolation (with moving-wall
ghosts), the saddle matvec in FP64 and FP32 per block, the mobility solve in
FP64 and FP32-refined, and one SEM step (Algorithm 1), on small seeded
cases with bodies close to walls, x-periodic moving walls and a ragged
42-blob case, gated element by element."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import saddle, solve, ib, sem  # noqa: E402
import workloads  # noqa: E402
from gpu_common import (CASES, assert_close, assert_close_blocks, F64_OP, F64_MATVEC, F32_MATVEC,  # noqa: E402
                        SOLVED, SEM_STEP)

pytestmark = pytest.mark.gpu

NAMES = ["walls", "xper_moving", "ragged42"]


@pytest.fixture(scope="module")
def B():
    import paper_1901_06427_gb300.binding as binding
    binding.lib()
    return binding


def case6(name, seed=5):
    kw = dict(CASES[name])
    w = workloads.small_case(seed=seed, kernel=6, **kw)
    og = oracle.Grid(w.n, periodic=w.periodic, wall_vel=w.wall_vel, kernel=6)
    ob = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
    return w, og, ob


def dev(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x).ravel(), dtype=dtype, device="cuda")


@pytest.mark.parametrize("name", NAMES)
def test_spread_and_interpolate_six_point(B, name):
    w, og, ob = case6(name)
    g = B.grid_for(w)
    assert g.desc.kernel == 6
    rng = np.random.default_rng(21)
    lam = rng.standard_normal(3 * w.n_blobs)
    v = rng.standard_normal(og.N_f)
    r = ob.positions()
    assert_close(g.spread(dev(lam)).cpu().numpy(), ib.spread(og, r, lam), F64_OP, "spread (6-point)")
    assert_close(g.interpolate(dev(v)).cpu().numpy(), ib.interpolate(og, r, v), F64_OP, "interpolate (6-point)")
    assert_close(g.interpolate(dev(v), with_walls=True).cpu().numpy(), ib.interpolate(og, r, v, with_walls=True),
                 F64_OP, "interpolate with moving-wall ghosts (6-point)")


@pytest.mark.parametrize("name", NAMES)
def test_apply_saddle_six_point(B, name):
    w, og, ob = case6(name)
    g = B.grid_for(w)
    x = np.random.default_rng(22).standard_normal(g.n_total)
    assert_close_blocks(g.apply_saddle(dev(x)).cpu().numpy(), saddle.apply(og, ob, w.eta, x), g.layout(),
                        F64_MATVEC, "FP64 matvec (6-point)")
    x32 = x.astype(np.float32).astype(np.float64)
    y32 = g.apply_saddle(dev(x32, torch.float32)).double().cpu().numpy()
    assert_close_blocks(y32, saddle.apply(og, ob, w.eta, x32), g.layout(), F32_MATVEC, "FP32 matvec (6-point)")


@pytest.mark.parametrize("name,precision", [("walls", "fp64"), ("xper_moving", "fp64"), ("ragged42", "refined")])
def test_mobility_solve_six_point(B, name, precision):
    w, og, ob = case6(name)
    prec = B.FP64 if precision == "fp64" else B.FP32_REFINED
    g = B.grid_for(w, precision=prec, rtol=1e-12 if precision == "fp64" else 1e-11)
    U, info, x = g.mobility_solve(dev(w.force_torque), slip=dev(w.slip), return_x=True)
    x0 = solve.constrained(og, ob, w.eta, saddle.rhs(og, ob, w.eta, F=w.force_torque, slip=w.slip))
    gate = SOLVED if precision == "fp64" else (1e-7, 1e-8)
    assert_close(U.cpu().numpy(), x0[-6 * w.n_bodies:], gate, f"U (6-point, {precision})")


def test_sem_step_six_point(B):
    w, og, ob = case6("walls")
    g = B.grid_for(w, rtol=1e-12)
    q, quat = dev(w.q), dev(w.quat)
    st, info = g.sem_step(B.sem_params(w.potentials, dt=0.05, kT=1.0), 11, 2, 1, q, quat)
    ref = sem.sem_step(og, ob, w.eta, 1.0, 0.05, w.potentials, seed=11, step=2, attempt=1)
    assert st == 0 and not ref["reject"]
    assert_close(q.cpu().numpy().reshape(-1, 3) - w.q, ref["q"] - w.q, SEM_STEP, "SEM displacement (6-point)")
    assert_close(quat.cpu().numpy() - w.quat.ravel(), ref["quat"].ravel() - w.quat.ravel(), SEM_STEP,
                 "SEM orientation increment (6-point)")


def test_adjoint_six_point(B):
    """Gradient of sum |U|^2 with respect to blob positions and slip with the
    six-point kernel (its derivative in J and S) against the oracle's."""
    from oracle import adjoint
    w = workloads.small_case(n=(12, 10, 9), n_bodies=2, blobs=12, radius=1.0, seed=9, near_wall=True, kernel=6)
    og = oracle.Grid(w.n, kernel=6)
    ob = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
    x0, U0 = adjoint.forward(og, ob, w.eta, w.slip.ravel(), w.force_torque)
    dr0, ds0 = adjoint.gradient(og, ob, w.eta, x0, 2.0 * U0)
    g = B.grid_for(w, rtol=1e-12)
    U, info, x = g.mobility_solve(dev(w.force_torque), slip=dev(w.slip), return_x=True)
    assert_close(U.cpu().numpy(), U0, SOLVED, "U (6-point)")
    dr, ds, ainfo = g.mobility_solve_adjoint(2.0 * U, x)
    assert_close(dr.cpu().numpy(), dr0.ravel(), (1e-7, 1e-8), "dL/dr (6-point)")
    assert_close(ds.cpu().numpy(), ds0, (1e-7, 1e-8), "dL/dslip (6-point)")
