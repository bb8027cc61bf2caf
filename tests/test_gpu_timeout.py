"""Bounded device waits: the persistent solver's grid barrier spins at most
the handle's wait budget (SM clock cycles).  With a budget of one cycle the
barrier's partners cannot arrive in time: every CTA returns, the step reports
NH_ERR_TIMEOUT and is not taken, and the same handle then steps normally (the
context stays usable).  No fault, trap or endless wait is involved: the wait
that runs out is the library's own bounded spin.

Both cases use a global criterion on more than one 8192-row preconditioner
block, so the solve runs the grid-wide loop (the member-local loop has no grid
barrier)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N = pytest.importorskip("paper_2505_17025_gb300.nhswe")
W = pytest.importorskip("paper_2505_17025_gb300.workloads")


def test_timeout_1d_step_not_taken_and_handle_usable():
    wl = W.slide_1d(n_members=1, nx=20000, length=16.0, xc0=2.0, T=0.2, seed0=3)

    def grid():
        G = N.grid_from_workload(wl)
        G.set_criterion(N.NH_CRIT_GLOBAL, 1e-3, 1, False)
        G.set_solver(N.NH_SOLVER_AUTO, 1e-12, 20000, N.NH_GUESS_PREV)
        return G

    ref = grid()
    ref.step(wl.dt)
    G = grid()
    before = G.get_state()
    G.set_wait_budget(1)
    st, info = G.step(wl.dt, check=False)
    assert st == N.NH_ERR_TIMEOUT, st
    after = G.get_state()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    G.set_wait_budget(0)
    st, info = G.step(wl.dt)
    assert st == N.NH_OK and info["iters"] > 0
    for a, b in zip(ref.get_state(), G.get_state()):
        assert np.array_equal(a, b)
    with pytest.raises(N.NHError):
        G.set_wait_budget(-1)


def test_timeout_2d_step_not_taken_and_handle_usable():
    nx, ny, dx = 120, 100, 0.05
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    X, Y = np.meshgrid(x, y)
    d0 = 0.5 + 0.1 * X
    eta = 0.03 * np.exp(-((X - 3.0) ** 2 + (Y - 2.5) ** 2) / 0.2)
    z = np.zeros((ny, nx))

    def grid():
        G = N.Grid2D(nx, ny, dx, dx, d0)
        G.set_criterion(N.NH_CRIT_GLOBAL, 1e-3, 1)
        G.set_solver(1e-12, 20000, N.NH_GUESS_PREV)
        G.set_state(d0 + eta, z, z, z)
        return G

    dt = 0.005
    ref = grid()
    ref.step(dt)
    G = grid()
    before = G.get_state()
    G.set_wait_budget(1)
    st, info = G.step(dt, check=False)
    assert st == N.NH_ERR_TIMEOUT, st
    for a, b in zip(before[:4], G.get_state()[:4]):
        assert np.array_equal(a, b)
    G.set_wait_budget(0)
    st, info = G.step(dt)
    assert st == N.NH_OK and info["iters"] > 0
    for a, b in zip(ref.get_state(), G.get_state()):
        assert np.array_equal(a, b)
