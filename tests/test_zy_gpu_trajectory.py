"""Ten-step trajectory parity (Algorithm 1): ten SEM steps on the GPU and ten
oracle steps from the same initial state with the same Philox seed stay on
one trajectory.  Each side advances from its own state, so the check covers
what a step carries over to the next (configuration refresh, the body
block's update from the previous inverse, the cached restart graphs).
Bodies start near the walls of a 13 x 11 x 9 box."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import saddle, sem, solve  # noqa: E402
from gpu_common import case, rel  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import paper_1901_06427_gb300.binding as binding
    binding.lib()
    return binding


def test_ten_step_trajectory_matches_oracle(B):
    w, og, _ = case("walls")
    g = B.grid_for(w, rtol=1e-12)
    p = B.sem_params(w.potentials, dt=0.05, kT=1.0)
    q = torch.tensor(np.asarray(w.q, dtype=np.float64).ravel(), device="cuda")
    quat = torch.tensor(np.asarray(w.quat, dtype=np.float64).ravel(), device="cuda")
    op = solve.StokesOperator(og, w.eta)
    q0 = np.asarray(w.q, dtype=np.float64).reshape(-1, 3)
    qo, quato = q0.copy(), np.asarray(w.quat, dtype=np.float64).reshape(-1, 4).copy()
    for k in range(10):
        q_prev = q.cpu().numpy().reshape(-1, 3)
        st, _ = g.sem_step(p, 11, k, 0, q, quat)
        bo = saddle.Bodies(w.ref_blobs, w.blob_offsets, qo, quato)
        ref = sem.sem_step(og, bo, w.eta, 1.0, 0.05, w.potentials, seed=11, step=k, op=op)
        assert st == 0 and not ref["reject"], k
        # this step's displacement, each side from its own state
        assert rel(q.cpu().numpy().reshape(-1, 3) - q_prev, ref["q"] - qo) < 1e-6, k
        qo, quato = ref["q"], ref["quat"]
    torch.cuda.synchronize()
    # where the trajectories end up
    assert rel(q.cpu().numpy().reshape(-1, 3) - q0, qo - q0) < 1e-6
    assert rel(quat.cpu().numpy().reshape(-1, 4), quato) < 1e-6
    g.close()
