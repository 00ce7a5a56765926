"""Batched ensembles (independent systems of uneven sizes advanced together)
and the block-size autotuner, through the C ABI."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import saddle, sem  # noqa: E402
import workloads  # noqa: E402
from gpu_common import rel  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_1901_06427_gb300.binding as binding
    binding.lib()
    return binding


def _systems():
    out = []
    for k, (n, nb) in enumerate([((12, 12, 12), 2), ((16, 16, 16), 3), ((12, 10, 8), 1), ((20, 20, 20), 4),
                                 ((16, 12, 12), 2)]):
        w = workloads.small_case(n=n, n_bodies=nb, blobs=12, seed=20 + k)
        out.append(w)
    return out


@pytest.mark.parametrize("precision", ["fp64", "refined"])
def test_batch_step_matches_single_grids_and_oracle(B, precision):
    ws = _systems()
    prec = B.FP64 if precision == "fp64" else B.FP32_REFINED
    for w in ws:
        w.rtol = 1e-11
    batch = B.Batch(ws, precision=prec, workers=3)
    q = [torch.tensor(w.q.ravel(), device="cuda") for w in ws]
    quat = [torch.tensor(w.quat.ravel(), device="cuda") for w in ws]
    params = [B.sem_params(w.potentials, dt=0.05, kT=1.0) for w in ws]
    seeds = [1000 + i for i in range(len(ws))]
    status, infos = batch.sem_step(params, seeds, 3, q, quat)
    assert all(s == 0 for s in status)
    assert all(m.step_mode() == 1 for m in batch.systems)   # each system ran its device-driven step graph
    for i, w in enumerate(ws):
        # the same system through a single grid
        g = B.grid_for(w, precision=prec, rtol=1e-11)
        q1, quat1 = torch.tensor(w.q.ravel(), device="cuda"), torch.tensor(w.quat.ravel(), device="cuda")
        st, _ = g.sem_step(params[i], seeds[i], 3, 0, q1, quat1)
        assert st == 0
        dq_b = q[i].cpu().numpy() - w.q.ravel()
        assert rel(dq_b, q1.cpu().numpy() - w.q.ravel()) < 1e-9
        for k in ("solve_rfd", "solve_stokes", "solve_main"):
            assert infos[i][k]["rel_residual"] <= 1e-11
    # two systems against the oracle
    for i in (0, 3):
        w = ws[i]
        og = oracle.Grid(w.n, periodic=w.periodic, wall_vel=w.wall_vel)
        ob = saddle.Bodies(w.ref_blobs, w.blob_offsets, w.q, w.quat)
        ref = sem.sem_step(og, ob, w.eta, 1.0, 0.05, w.potentials, seed=seeds[i], step=3)
        assert rel(q[i].cpu().numpy().reshape(-1, 3) - w.q, ref["q"] - w.q) < 1e-8
    batch.close()


def test_autotuner_picks_a_candidate(B):
    w = workloads.small_case(n=(24, 20, 16), n_bodies=1)
    g = B.grid_for(w)
    t = g.tuned_blocks()
    # uniform spacing: the Stokes kernels have fixed tile shapes (0 = not tuned);
    # the smoothing sweeps take one of the candidate block sizes
    assert t[0] == 0 and t[1] == 0
    assert all(v in (64, 128, 256, 512) for v in t[2:])


@pytest.mark.parametrize("precision", ["fp64", "refined"])
def test_one_graph_batch_matches_worker_streams(B, precision):
    # the same ensemble advanced by the worker streams and by one graph launch
    # per batch step (every system a branch of the graph), three steps each
    ws = _systems()
    prec = B.FP64 if precision == "fp64" else B.FP32_REFINED
    for w in ws:
        w.rtol = 1e-11
    runs = []
    for one_graph in (False, True):
        batch = B.Batch(ws, precision=prec, workers=3, one_graph=one_graph)
        q = [torch.tensor(w.q.ravel(), device="cuda") for w in ws]
        quat = [torch.tensor(w.quat.ravel(), device="cuda") for w in ws]
        params = [B.sem_params(w.potentials, dt=0.05, kT=1.0) for w in ws]
        seeds = [2000 + i for i in range(len(ws))]
        hist = []
        for k in range(3):
            status, infos = batch.sem_step(params, seeds, k, q, quat)
            assert all(s == 0 for s in status)
            for info in infos:
                for key in ("solve_rfd", "solve_stokes", "solve_main"):
                    assert info[key]["rel_residual"] <= 1e-11 and info[key]["iterations"] > 0
            hist.append([(x.cpu().numpy().copy(), y.cpu().numpy().copy()) for x, y in zip(q, quat)])
        # captured once, then relaunched (the configuration buffers stay the same)
        runs.append((hist, batch.graph_steps()))
        batch.close()
    (h0, n0), (h1, n1) = runs
    assert n0 == 0 and n1 == 3
    for k in range(3):
        for i, w in enumerate(ws):
            # the changes since the start agree (FP32 atomics in the refined
            # mode's spreading sum in another order on each path)
            assert rel(h1[k][i][0] - w.q.ravel(), h0[k][i][0] - w.q.ravel()) < 1e-9
            assert rel(h1[k][i][1] - w.quat.ravel(), h0[k][i][1] - w.quat.ravel()) < 1e-9


def test_one_graph_flag_is_checked(B):
    w = workloads.small_case(n=(12, 12, 12), n_bodies=1, blobs=12, seed=5)
    batch = B.Batch([w], workers=1)
    assert B.lib().rbfib_batch_set_one_graph(batch._h, 2) == B.EINVAL
    assert B.lib().rbfib_batch_set_one_graph(batch._h, 1) == B.OK
    assert B.lib().rbfib_batch_set_one_graph(None, 1) == B.EINVAL
    assert B.lib().rbfib_batch_graph_steps(None) == -1
    assert batch.graph_steps() == 0
    batch.close()
