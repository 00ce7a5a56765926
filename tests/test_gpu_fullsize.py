"""GPU checks at the benchmark workloads' full sizes, in the configuration
bench.py times: the saddle matvec element by element against the oracle,
solved body velocities against stored oracle values (tests/golden/, written
by make_golden.py from oracle/ only) and properties that hold at any size."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import saddle  # noqa: E402
import workloads  # noqa: E402
from gpu_common import rel, assert_close, assert_close_blocks, F64_MATVEC, F32_MATVEC, SOLVED, SEM_STEP  # noqa: E402

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def B():
    import paper_1901_06427_gb300.binding as binding
    binding.lib()
    return binding


def dev(x):
    return torch.tensor(np.asarray(x).ravel(), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("make", [workloads.single_sphere_box, lambda: workloads.two_sphere_cavity(steps=1)])
def test_fullsize_matvec(B, make):
    w = make()
    g = B.grid_for(w)
    og = oracle.Grid(w.n, periodic=w.periodic, wall_vel=w.wall_vel)
    ob = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
    x = np.random.default_rng(0).standard_normal(g.n_total)
    y = g.apply_saddle(dev(x)).cpu().numpy()
    y0 = saddle.apply(og, ob, w.eta, x)
    assert_close_blocks(y, y0, g.layout(), F64_MATVEC, "FP64 matvec")
    x32 = x.astype(np.float32).astype(np.float64)
    y32 = g.apply_saddle(torch.tensor(x32, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    assert_close_blocks(y32, saddle.apply(og, ob, w.eta, x32), g.layout(), F32_MATVEC, "FP32 matvec")


def test_single_sphere_mobility_against_oracle(B):
    w = workloads.single_sphere_box()
    gold = json.load(open(os.path.join(GOLD, "single_sphere_32.json")))
    g = B.grid_for(w, rtol=1e-12)
    U, info = g.mobility_solve(dev(w.force_torque))
    U = U.cpu().numpy()
    assert info["rel_residual"] <= 1e-12
    assert_close(U, gold["U"], SOLVED, "U")
    # symmetry of the centred shell in the cube: no coupling between axes
    assert np.all(np.abs(U[[1, 2, 3, 4]]) < 1e-8 * np.abs(U).max())
    # at the benchmark tolerance (1e-10) the answer stays within the tolerance band
    g2 = B.grid_for(w)
    U2, info2 = g2.mobility_solve(dev(w.force_torque))
    assert info2["rel_residual"] <= 1e-10
    assert rel(U2.cpu().numpy(), gold["U"]) < 1e-7


def test_two_sphere_sem_step_against_oracle(B):
    w = workloads.two_sphere_cavity(steps=1)
    gold = json.load(open(os.path.join(GOLD, "two_sphere_step0.json")))
    g = B.grid_for(w, rtol=1e-12)
    q, quat = dev(w.q), dev(w.quat)
    p = B.sem_params(w.potentials, dt=w.dt, kT=w.kT)
    st, info = g.sem_step(p, w.seed, 0, 0, q, quat)
    assert st == 0
    dq = q.cpu().numpy() - np.array(gold["q0"])
    assert_close(dq, np.array(gold["q"]) - np.array(gold["q0"]), SEM_STEP, "SEM displacement")
    dquat = quat.cpu().numpy() - np.array(gold["quat0"])
    assert_close(dquat, np.array(gold["quat"]) - np.array(gold["quat0"]), SEM_STEP, "SEM orientation increment")
    # benchmark configuration (rel. residual 1e-8): every solve meets it and the
    # step stays within the tolerance band of the oracle's
    g8 = B.grid_for(w, rtol=1e-8)
    q8, quat8 = dev(w.q), dev(w.quat)
    st, info8 = g8.sem_step(p, w.seed, 0, 0, q8, quat8)
    for k in ("solve_rfd", "solve_stokes", "solve_main"):
        assert info8[k]["rel_residual"] <= 1e-8
    dq8 = q8.cpu().numpy() - np.array(gold["q0"])
    assert rel(dq8, np.array(gold["q"]) - np.array(gold["q0"])) < 1e-5


@pytest.mark.parametrize("periodic,wall_speed", [((False, False, False), 0.0), ((True, False, False), 0.3),
                                                 ((False, True, True), 0.0)])
def test_matvec_large_grid(B, periodic, wall_speed):
    """Grids above two million unknowns take the pipelined Stokes kernel; the
    sizes leave ragged tiles in x, y and z."""
    w = workloads.small_case(n=(100, 90, 76), periodic=periodic, n_bodies=3, blobs=12, seed=1,
                             wall_speed=wall_speed)
    g = B.grid_for(w)
    assert g.n_total > 2 * 1024 * 1024
    og = oracle.Grid(w.n, periodic=w.periodic, wall_vel=w.wall_vel)
    ob = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
    x = np.random.default_rng(3).standard_normal(g.n_total)
    y0 = saddle.apply(og, ob, w.eta, x)
    y = g.apply_saddle(dev(x)).cpu().numpy()
    assert_close_blocks(y, y0, g.layout(), F64_MATVEC, "FP64 matvec")
    x32 = x.astype(np.float32).astype(np.float64)
    y32 = g.apply_saddle(torch.tensor(x32, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    assert_close_blocks(y32, saddle.apply(og, ob, w.eta, x32), g.layout(), F32_MATVEC, "FP32 matvec")
