"""The kernel timer (C ABI rbfib_kernel_timer / _read / _overhead): the
algorithmic bytes and operations it adds up follow the per-launch counts the
header states, only the selected class is timed, and the event-bracket
overhead is measured on an empty kernel."""
import pytest

torch = pytest.importorskip("torch")

import workloads  # noqa: E402

pytestmark = pytest.mark.gpu

MATVEC, DOT = 1, 3


@pytest.fixture(scope="module")
def B():
    import paper_1901_06427_gb300.binding as binding
    binding.lib()
    return binding


@pytest.fixture(scope="module")
def grid(B):
    w = workloads.small_case(n=(16, 16, 12), n_bodies=2, blobs=12, seed=41)
    g = B.grid_for(w, precision=B.FP64, rtol=1e-8)
    yield g
    g.close()


def _solve(g):
    FT = torch.zeros(6 * g.n_bodies, dtype=torch.float64, device="cuda")
    FT[0] = 1.0
    FT[11] = 0.5
    return g.mobility_solve(FT)


def test_matvec_counts_follow_stated_formula(grid):
    lay = grid.layout()
    n, n_f, n_c = lay[6], lay[3], lay[4] - lay[3]
    nbl, nb = grid.n_blobs, grid.n_bodies
    grid.kernel_timer(MATVEC)
    _, info = _solve(grid)
    ms, launches, nbytes, nflops = grid.kernel_timer_read()
    grid.kernel_timer(0)
    # one saddle matvec per FGMRES iteration, plus the restart residuals
    assert launches >= info["iterations"] >= 1
    assert ms > 0.0
    per_bytes = 2.0 * n * 8 + 24.0 * nbl + 56.0 * nb
    per_ops = 10.0 * n_f + 6.0 * n_c + 400.0 * nbl
    assert nbytes == pytest.approx(launches * per_bytes, rel=1e-12)
    assert nflops == pytest.approx(launches * per_ops, rel=1e-12)


def test_unselected_classes_add_nothing(grid):
    grid.kernel_timer(0)
    _solve(grid)
    ms, launches, nbytes, nflops = grid.kernel_timer_read()
    assert (ms, launches, nbytes, nflops) == (0.0, 0, 0.0, 0.0)
    grid.kernel_timer(DOT)
    _solve(grid)
    ms, launches, _, nflops = grid.kernel_timer_read()
    grid.kernel_timer(0)
    assert launches > 0 and ms > 0.0 and nflops > 0.0


def test_event_overhead_is_measured(grid):
    us = grid.kernel_timer_overhead(50)
    # an empty kernel between two events: a few microseconds on GB300
    assert 0.0 < us < 200.0
