"""Short-time Stokes-Einstein relation of the confined two-sphere dynamics
(Sec. V.A, Eq. SErel) on the GPU: equilibrium trajectories of the tight
cavity (12-blob spheres, six-point kernel, dtau = 0.0044) started from
Gibbs-Boltzmann samples of the oracle's sampler (tests/golden/, written by
make_golden.py from oracle/ only) have one-step mean-square displacements
MSD(dt) / dt = 2 kT <N^tt>_GB, the Gibbs-Boltzmann average of the
translational body mobility taken over the same samples with the GPU's own
deterministic solves.  Checked entry by entry (self and cross blocks) within
five standard errors of the replica means plus the O(dt) bias allowance."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads  # noqa: E402

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def B():
    import paper_1901_06427_gb300.binding as binding
    binding.lib()
    return binding


def mean_translational_mobility(B, w, starts):
    """<N^tt> over the starts: columns from unit forces on each centre."""
    g = B.grid_for(w, rtol=1e-10)
    nb = w.n_bodies
    acc = np.zeros((3 * nb, 3 * nb))
    for q, quat in zip(starts["q"], starts["quat"]):
        g.set_bodies(w.blob_offsets, w.ref_blobs, np.array(q).reshape(nb, 3), np.array(quat).reshape(nb, 4))
        for p in range(nb):
            for c in range(3):
                F = np.zeros(6 * nb)
                F[6 * p + c] = 1.0
                U, _ = g.mobility_solve(torch.tensor(F, device="cuda"))
                U = U.cpu().numpy().reshape(nb, 6)
                acc[:, 3 * p + c] += U[:, :3].ravel()
    g.close()
    return acc / len(starts["q"])


def replica_trajectories(B, w, starts, n_rep, steps):
    """Centres (steps + 1, n_rep, 3 N_b) of n_rep batched trajectories."""
    nb = w.n_bodies
    ws = []
    for r in range(n_rep):
        wr = workloads.two_sphere_msd(w.n_blobs // nb)
        for p, body in enumerate(wr.bodies):
            body.q = np.array(starts["q"][r]).reshape(nb, 3)[p]
            body.quat = np.array(starts["quat"][r]).reshape(nb, 4)[p]
        ws.append(wr)
    batch = B.Batch(ws, precision=B.FP64, workers=16)
    q = [torch.tensor(x.q.ravel(), device="cuda") for x in ws]
    quat = [torch.tensor(x.quat.ravel(), device="cuda") for x in ws]
    params = [B.sem_params(x.potentials, dt=x.dt, kT=x.kT) for x in ws]
    seeds = [x.seed + 101 * r for r, x in enumerate(ws)]
    hist = [torch.stack(q).cpu().numpy()]
    for k in range(steps):
        status, _ = batch.sem_step(params, seeds, k, q, quat)
        for r, st in enumerate(status):
            attempt = 0
            while st == B.EREJECT and attempt < 20:      # Sec. V: retry with new noise
                attempt += 1
                st, _ = batch.systems[r].sem_step(params[r], seeds[r], k, attempt, q[r], quat[r])
            assert st == B.OK
        hist.append(torch.stack(q).cpu().numpy())
    batch.close()
    return np.array(hist)


def test_short_time_msd_is_stokes_einstein(B):
    gold = json.load(open(os.path.join(GOLD, "gb_two_sphere_msd_12.json")))
    w = workloads.two_sphere_msd(12)
    n_rep, steps = 32, 150
    Nt = mean_translational_mobility(B, w, gold["starts"])
    X = replica_trajectories(B, w, gold["starts"], n_rep, steps)
    D = X[1:] - X[:-1]                                          # one-step displacements
    per_rep = np.einsum("trj,trk->rjk", D, D) / D.shape[0]      # MSD(dt) per replica
    msd = per_rep.mean(axis=0)
    se = per_rep.std(axis=0, ddof=1) / np.sqrt(n_rep)
    want = 2.0 * w.kT * w.dt * Nt
    scale = np.sqrt(np.outer(np.diag(want), np.diag(want)))
    # entries with a sizeable coupling: self blocks and the along-x cross term
    for j, k in [(0, 0), (1, 1), (2, 2), (3, 3), (4, 4), (5, 5), (0, 3), (3, 0)]:
        lim = 5.0 * se[j, k] + 0.05 * scale[j, k]
        assert abs(msd[j, k] - want[j, k]) <= lim, (j, k, msd[j, k], want[j, k], lim)
    # the remaining cross terms vanish on average within their errors
    assert np.all(np.abs(msd - want) <= 5.0 * se + 0.05 * scale)
