"""GPU parity of every hot-path step against the FP64 oracle, through the
C ABI (paper_1901_06427_gb300.binding), on small seeded cases that span
several thread blocks with ragged tails and every boundary combination.

Gates, all element by element (gpu_common.assert_close: |a_i - b_i| <= rtol
|b_i| + floor ||b||_inf, per block of the saddle layout): binning and Philox
words bit-exact; Philox normals to a few ulps (they differ only through
log/sincos rounding); FP64 single operators rtol 1e-12, the FP64 saddle matvec
1e-11; the FP32 matvec 1e-5 on the same FP32-rounded input; solved
quantities 1e-8."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import saddle, solve, ib, binning, philox, noise, forces, sem  # noqa: E402
from gpu_common import (case, rel, CASES, assert_close, assert_close_blocks, F64_OP, F64_MATVEC,  # noqa: E402
                        F32_MATVEC, SOLVED, SEM_STEP)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_1901_06427_gb300.binding as binding
    binding.lib()
    return binding


def dev(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x).ravel(), dtype=dtype, device="cuda")


@pytest.mark.parametrize("name", list(CASES))
def test_binning_bit_exact(B, name):
    w, og, ob = case(name)
    g = B.grid_for(w)
    perm, off = g.binning()
    p0, o0 = binning.counting_sort(og, ob.positions())
    assert np.array_equal(perm.cpu().numpy(), p0)
    assert np.array_equal(off.cpu().numpy(), o0)


def test_binning_exact_cell_boundaries(B):
    """Blobs exactly on cell faces and outside the box on a wall axis."""
    w, og, ob = case("xper_moving")
    w.bodies[0].q = np.array([4.0, 3.0, 2.0])
    w.bodies[0].quat = np.array([1.0, 0.0, 0.0, 0.0])
    g = B.grid_for(w)
    ob = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
    perm, off = g.binning()
    p0, o0 = binning.counting_sort(og, ob.positions())
    assert np.array_equal(perm.cpu().numpy(), p0) and np.array_equal(off.cpu().numpy(), o0)


@pytest.mark.parametrize("n_blocks,first", [(1, 0), (3, 5), (1001, 0), (65536 + 7, 123456789)])
def test_philox_words_bit_exact(B, n_blocks, first):
    """Raw Philox4x64-10 words of the GPU equal the oracle's bit for bit
    (the oracle's words are themselves pinned to numpy's Philox)."""
    w, og, ob = case("walls")
    g = B.grid_for(w)
    for seed, step, attempt, purpose in ((0xDEADBEEF12345, 77, 3, 1), (2 ** 64 - 1, 2 ** 63 + 5, 2 ** 32 - 1, 2)):
        got = g.philox_words(seed, step, attempt, purpose, n_blocks, first).cpu().numpy().view(np.uint64)
        want = philox.words(seed, step, attempt, purpose, n_blocks, first_block=first)
        assert np.array_equal(got, want)


@pytest.mark.parametrize("count", [1, 3, 4, 1001, 65536 + 7])
def test_philox_normals(B, count):
    w, og, ob = case("walls")
    g = B.grid_for(w)
    for purpose in (1, 2):
        z = g.philox_normals(0xDEADBEEF12345, 77, 3, purpose, count).cpu().numpy()
        z0 = philox.normals(0xDEADBEEF12345, 77, 3, purpose, count)
        assert np.all(np.abs(z - z0) <= 4e-15 * np.maximum(1.0, np.abs(z0)))


@pytest.mark.parametrize("name", list(CASES))
def test_stochastic_forcing(B, name):
    w, og, ob = case(name)
    g = B.grid_for(w)
    f = g.stochastic_forcing(1.3, 0.02, 99, 5, 1).cpu().numpy()
    f0 = noise.fluid_forcing(og, w.eta, 1.3, 0.02, 99, 5, 1)
    assert_close(f, f0, F64_OP, "fluid forcing")


@pytest.mark.parametrize("name", list(CASES))
def test_spread_and_interpolate(B, name):
    w, og, ob = case(name)
    g = B.grid_for(w)
    rng = np.random.default_rng(1)
    lam = rng.standard_normal(3 * w.n_blobs)
    v = rng.standard_normal(og.N_f)
    r = ob.positions()
    assert_close(g.blob_positions().cpu().numpy(), r, (1e-15, 1e-15), "blob positions")
    assert_close(g.spread(dev(lam)).cpu().numpy(), ib.spread(og, r, lam), F64_OP, "spread")
    assert_close(g.interpolate(dev(v)).cpu().numpy(), ib.interpolate(og, r, v), F64_OP, "interpolate")
    assert_close(g.interpolate(dev(v), with_walls=True).cpu().numpy(), ib.interpolate(og, r, v, with_walls=True),
                 F64_OP, "interpolate with moving-wall ghosts")


@pytest.mark.parametrize("name", list(CASES))
def test_apply_saddle_fp64(B, name):
    w, og, ob = case(name)
    g = B.grid_for(w)
    x = np.random.default_rng(3).standard_normal(g.n_total)
    y = g.apply_saddle(dev(x)).cpu().numpy()
    y0 = saddle.apply(og, ob, w.eta, x)
    lay = g.layout()
    assert lay == saddle.layout(og, ob)
    assert_close_blocks(y, y0, lay, F64_MATVEC, "FP64 matvec")


@pytest.mark.parametrize("name", list(CASES))
def test_apply_saddle_fp32(B, name):
    w, og, ob = case(name)
    g = B.grid_for(w)
    x = np.random.default_rng(4).standard_normal(g.n_total).astype(np.float32).astype(np.float64)
    y = g.apply_saddle(dev(x, torch.float32)).double().cpu().numpy()
    assert_close_blocks(y, saddle.apply(og, ob, w.eta, x), g.layout(), F32_MATVEC, "FP32 matvec")


@pytest.mark.parametrize("name", ["walls", "xper_moving"])
def test_body_forces(B, name):
    w, og, ob = case(name)
    pot = dict(w.potentials)
    pot["yukawa"] = {"u0": 20.0, "d_h": 2.0, "lambda_d": 0.3}
    pot["blob_wall_soft"] = {"phi0": 4.0, "b": 0.1, "d": 1.0}
    pot["substrate"] = {"u0": 4.0, "s_lattice": 6.0}
    g = B.grid_for(w)
    F = g.body_forces(B.sem_params(pot)).cpu().numpy()
    F0 = forces.body_forces(og, ob, pot).ravel()
    assert_close(F, F0, F64_OP, "body forces")


@pytest.mark.parametrize("name", ["walls", "xper_moving", "yzper"])
def test_stokes_solve(B, name):
    w, og, ob = case(name)
    g = B.grid_for(w, rtol=1e-12)
    f = np.random.default_rng(5).standard_normal(og.N_f)
    v, pi, info = g.stokes_solve(dev(f))
    v0, p0 = solve.stokes(og, w.eta, f)
    assert info["rel_residual"] <= 1e-12
    assert_close(v.cpu().numpy(), v0, SOLVED, "Stokes velocity")
    assert_close(pi.cpu().numpy(), p0, SOLVED, "Stokes pressure")


@pytest.mark.parametrize("name", list(CASES))
def test_mobility_solve(B, name):
    w, og, ob = case(name)
    g = B.grid_for(w, rtol=1e-12)
    U, info, x = g.mobility_solve(dev(w.force_torque), slip=dev(w.slip), return_x=True)
    f = saddle.rhs(og, ob, w.eta, F=w.force_torque, slip=w.slip)
    x0 = solve.constrained(og, ob, w.eta, f)
    assert info["rel_residual"] <= 1e-12
    assert_close(U.cpu().numpy(), x0[-6 * w.n_bodies:], SOLVED, "U")
    xg = x.cpu().numpy()
    assert np.linalg.norm(saddle.apply(og, ob, w.eta, xg) - f) <= 1e-11 * np.linalg.norm(f)
    assert_close_blocks(xg, x0, g.layout(), SOLVED, "solution")


def test_mobility_solve_with_fluid_forcing(B):
    w, og, ob = case("xper_moving")
    g = B.grid_for(w, rtol=1e-12)
    fl = np.random.default_rng(6).standard_normal(og.N_f)
    U, info = g.mobility_solve(dev(w.force_torque), fluid_rhs=dev(fl))
    f = saddle.rhs(og, ob, w.eta, F=w.force_torque, f_fluid=fl)
    x0 = solve.constrained(og, ob, w.eta, f)
    assert_close(U.cpu().numpy(), x0[-6 * w.n_bodies:], SOLVED, "U")


@pytest.mark.parametrize("name", ["walls", "xper_moving", "ragged42"])
def test_sem_step(B, name):
    w, og, ob = case(name)
    g = B.grid_for(w, rtol=1e-12)
    q, quat = dev(w.q), dev(w.quat)
    st, info = g.sem_step(B.sem_params(w.potentials, dt=0.05, kT=1.0), 11, 2, 1, q, quat)
    ref = sem.sem_step(og, ob, w.eta, 1.0, 0.05, w.potentials, seed=11, step=2, attempt=1)
    assert st == 0 and not ref["reject"]
    dq = q.cpu().numpy().reshape(-1, 3) - w.q
    assert_close(dq, ref["q"] - w.q, SEM_STEP, "SEM displacement")
    assert_close(quat.cpu().numpy() - w.quat.ravel(), ref["quat"].ravel() - w.quat.ravel(), SEM_STEP,
                 "SEM orientation increment")


def test_sem_step_rejects_unphysical_configuration(B):
    """A huge force pushes a body through the bottom wall: the step is
    rejected, q and quat are unchanged (Sec. V)."""
    w, og, ob = case("walls")
    g = B.grid_for(w, rtol=1e-10)
    fext = np.zeros((w.n_bodies, 6)); fext[:, 2] = -1e5
    q, quat = dev(w.q), dev(w.quat)
    p = B.sem_params(w.potentials, dt=0.05, kT=1.0, force_ext=dev(fext))
    st, info = g.sem_step(p, 1, 0, 0, q, quat)
    assert st == B.EREJECT and info["rejected"] == 1
    assert np.array_equal(q.cpu().numpy(), w.q.ravel())
    assert np.array_equal(quat.cpu().numpy(), w.quat.ravel())


def test_errors_are_status_codes(B):
    import ctypes
    d = B.GridDesc()
    d.n[0] = d.n[1] = d.n[2] = 8
    d.periodic[0] = d.periodic[1] = d.periodic[2] = 1     # fully periodic: rejected
    d.h, d.eta, d.kernel, d.restart, d.max_iter, d.rtol = 1.0, 1.0, 3, 10, 10, 1e-8
    h = ctypes.c_void_p()
    assert B.lib().rbfib_create_grid(ctypes.byref(d), None, ctypes.byref(h)) == B.EINVAL
    w, og, ob = case("walls")
    g = B.grid_for(w, rtol=1e-14, max_iter=3)
    with pytest.raises(B.RbfibError) as e:
        g.mobility_solve(dev(w.force_torque))
    assert e.value.code == B.ENOCONV


# ----------------------------------------------- FP32 inside FP64 refinement
@pytest.mark.parametrize("name", ["walls", "xper_moving", "ragged42"])
def test_refined_mobility_solve(B, name):
    """FP32 stencils, spreading, multigrid and Krylov basis inside an FP64
    iterative-refinement loop reach the FP64 tolerance; the error against the
    FP64 oracle is reported per output block."""
    w, og, ob = case(name)
    g = B.grid_for(w, precision=B.FP32_REFINED, rtol=1e-10)
    U, info, x = g.mobility_solve(dev(w.force_torque), slip=dev(w.slip), return_x=True)
    f = saddle.rhs(og, ob, w.eta, F=w.force_torque, slip=w.slip)
    x0 = solve.constrained(og, ob, w.eta, f)
    assert info["rel_residual"] <= 1e-10 and info["refinements"] >= 1
    xg = x.cpu().numpy()
    lay = g.layout()
    errs = {blk: rel(xg[lay[i]:lay[i + 1]], x0[lay[i]:lay[i + 1]])
            for i, blk in enumerate(["vx", "vy", "vz", "pi", "lambda", "U"])}
    print("refined errors vs oracle:", {k: f"{v:.2e}" for k, v in errs.items()})
    assert errs["U"] < 1e-8
    assert max(errs.values()) < 1e-7


def test_refined_sem_step(B):
    w, og, ob = case("walls")
    g = B.grid_for(w, precision=B.FP32_REFINED, rtol=1e-11)
    q, quat = dev(w.q), dev(w.quat)
    st, info = g.sem_step(B.sem_params(w.potentials, dt=0.05, kT=1.0), 11, 2, 1, q, quat)
    ref = sem.sem_step(og, ob, w.eta, 1.0, 0.05, w.potentials, seed=11, step=2, attempt=1)
    assert st == 0
    for k in ("solve_rfd", "solve_stokes", "solve_main"):
        assert info[k]["rel_residual"] <= 1e-11
    dq = q.cpu().numpy().reshape(-1, 3) - w.q
    assert rel(dq, ref["q"] - w.q) < 1e-7


@pytest.mark.parametrize("name", list(CASES))
def test_preconditioner_fluid_block_exact(B, name):
    """On grids with at most 32 points per axis the V-cycles reduce to the exact
    coarse-level solve (fast diagonalisation), so the fluid block of the
    preconditioner is the projection method with exact inner solves:
    v~ = (-eta LL)^-1 r_v, q = r_pi + D v~, phi = (-DG)^+ q, v = v~ + G phi,
    pi = -eta q.  The preconditioner computes in FP32."""
    from scipy.sparse.linalg import cg
    from oracle import operators
    w, og, ob = case(name)
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
    v = vt + G @ phi
    assert rel(z[:nf], v) < 1e-4
    assert rel(z[nf:nf + nc], -w.eta * q) < 1e-4
