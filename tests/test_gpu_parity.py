"""GPU (C ABI, FP64 path) vs the FP64 oracle, element by element.

Tolerance (FP64 path): max |d eta| <= 1e-9 a (a = the workload's wave or
slide amplitude) and max |d hu|, |d hw| <= 1e-9 a sqrt(g h_max), after every
run below; masks equal cell for cell.  Both sides round
differently (FMA contraction, reduction order, scaled unknown), so equality is
to the tolerance, not to the bit.
"""
import copy
import math

import numpy as np
import pytest

import oracle as O
from paper_2505_17025_gb300 import nhswe as N
from paper_2505_17025_gb300 import workloads as W

from _helpers import compare, make_gpu, run_oracle

pytestmark = pytest.mark.gpu


def _small_slide(n_members=3, nx=2000, length=4.0, T=0.5, seed0=11):
    # the sliding-mound workload on a short slope; nx = 2000 spans 8 tiles of
    # 256 cells plus a ragged tail of 208
    return W.slide_1d(n_members=n_members, nx=nx, length=length, xc0=1.0, T=T, seed0=seed0)


def test_solitary_global_and_adaptive_parity():
    wl = W.solitary_1d()
    n = 200
    for crit in (O.CRIT_GLOBAL, O.CRIT_ETA_D):
        ref = run_oracle(wl, n, crit=crit)
        # unpreconditioned CG: the same iteration as the oracle's
        G = make_gpu(wl, crit, precond=N.NH_PRECOND_NONE)
        st, info = G.run(wl.dt, n)
        compare(wl, G, ref, what=f"solitary crit={crit}")
        m, iters, rel = G.get_mask()
        assert np.array_equal(m[0], ref[0][2])
        ref_it = ref[0][1][-1]["iters"]
        assert abs(int(iters[0]) - ref_it) <= max(2, 0.02 * ref_it)
        G.close()


@pytest.mark.parametrize("crit", [O.CRIT_ETA_D, O.CRIT_ETA_X, O.CRIT_U, O.CRIT_U_X, O.CRIT_W,
                                  O.CRIT_W_X])
@pytest.mark.parametrize("enlarge", [0, 1, 3])
def test_criteria_masks_and_state(crit, enlarge):
    wl = _small_slide(n_members=2)
    n = 25
    first = 1 if crit in (O.CRIT_W, O.CRIT_W_X) else 0
    ref = run_oracle(wl, n, crit=crit, enlarge=enlarge, first=first, knh=1e-4)
    G = make_gpu(wl, crit, enlarge=enlarge, first=first, knh=1e-4)
    G.run(wl.dt, n)
    compare(wl, G, ref, what=f"crit={crit} e={enlarge}")
    m, _, _ = G.get_mask()
    for b in range(2):
        assert np.array_equal(m[b], ref[b][2]), (b, np.flatnonzero(m[b] != ref[b][2]))
    G.close()


def test_batch_of_slides_matches_each_member():
    wl = _small_slide(n_members=5)
    n = 40
    ref = run_oracle(wl, n, crit=O.CRIT_ETA_D)
    G = make_gpu(wl, O.CRIT_ETA_D)
    st, info = G.run(wl.dt, n)
    compare(wl, G, ref, what="batch")
    assert info["last"]["n_active"] == sum(int(r[2].sum()) for r in ref)
    G.close()


@pytest.mark.parametrize("solver", [O.SOLVER_CG, O.SOLVER_BICGSTAB])
def test_forced_solver_kinds(solver):
    wl = _small_slide(n_members=2)
    n = 15
    ref = run_oracle(wl, n, crit=O.CRIT_GLOBAL, solver=solver)
    G = make_gpu(wl, O.CRIT_GLOBAL, solver=solver, precond=N.NH_PRECOND_NONE)
    G.run(wl.dt, n)
    compare(wl, G, ref, what=f"solver={solver}")
    _, iters, rel = G.get_mask()
    for b in range(2):
        ref_it = ref[b][1][-1]["iters"]
        assert rel[b] <= 1e-12
        if solver == O.SOLVER_CG:
            # same algorithm; rounding differs, so a long ill-conditioned solve
            # may stop a few iterations apart (both at the same residual)
            assert abs(int(iters[b]) - ref_it) <= max(2, 0.02 * ref_it)
    G.close()


@pytest.mark.parametrize("crit", [O.CRIT_GLOBAL, O.CRIT_ETA_D])
@pytest.mark.parametrize("solver", [O.SOLVER_CG, O.SOLVER_BICGSTAB])
def test_line_preconditioned_krylov(crit, solver):
    """PCG / right-preconditioned BiCGStab with the block-tridiagonal FP32
    preconditioner converge to the same solution as the oracle's plain
    Krylov solve, in far fewer iterations."""
    wl = _small_slide(n_members=3)
    n = 30
    ref = run_oracle(wl, n, crit=crit, solver=solver)
    G = make_gpu(wl, crit, solver=solver, precond=N.NH_PRECOND_LINE)
    st, info = G.run(wl.dt, n)
    compare(wl, G, ref, what=f"pcg crit={crit}")
    _, iters, rel = G.get_mask()
    for b in range(3):
        assert rel[b] <= 1e-12
        assert iters[b] <= max(30, ref[b][1][-1]["iters"] // 20), (iters[b], ref[b][1][-1]["iters"])
    G.close()


def test_auto_with_negative_gamma():
    """A sharp, tall mound makes the reaction term negative on its convex
    flank.  The operator stays symmetric positive definite there, so AUTO's
    CG converges; the oracle (gamma > 0 rule) uses BiCGStab; both must reach
    the same solution."""
    nx, dx = 600, 0.01
    d0 = np.full(nx, 1.0)
    m = W.Member1D(nx=nx, dx=dx, xl=0.0, d0=d0, h=d0.copy(), hu=np.zeros(nx), hw=np.zeros(nx),
                   slide=1, A=0.3, L=0.15, xc0=3.0, s0=1.0, t0=0.5)
    wl = W.Workload1D("sharp", [m], 0.002, 10, 0.02, amplitude=0.3)
    ref = run_oracle(wl, 3, crit=O.CRIT_GLOBAL)
    assert ref[0][1][-1]["solver_used"] == O.SOLVER_BICGSTAB
    for precond in (N.NH_PRECOND_LINE, N.NH_PRECOND_NONE):
        G = make_gpu(wl, O.CRIT_GLOBAL, precond=precond)
        st, info = G.run(wl.dt, 3)
        assert info["last"]["min_gamma"] < 0
        assert info["last"]["solver"] in (N.NH_SOLVER_CG, N.NH_SOLVER_BICGSTAB)
        compare(wl, G, ref, what="auto-negative-gamma")
        G.close()


def test_periodic_boundaries():
    wl = W.solitary_1d(nx=1000, length=100.0, a=0.1, T=3.0)
    wl.bc = N.NH_BC_PERIODIC
    n = 60
    ref = run_oracle(wl, n, crit=O.CRIT_ETA_D, bc=O.BC_PERIODIC, enlarge=2)
    G = make_gpu(wl, O.CRIT_ETA_D, bc=O.BC_PERIODIC, enlarge=2)
    G.run(wl.dt, n)
    compare(wl, G, ref, what="periodic")
    G.close()


@pytest.mark.parametrize("limiter", [O.LIM_NONE, O.LIM_MINMOD, O.LIM_MC])
def test_limiters(limiter):
    wl = _small_slide(n_members=1)
    n = 20
    ref = run_oracle(wl, n, crit=O.CRIT_ETA_D, limiter=limiter)
    G = make_gpu(wl, O.CRIT_ETA_D, limiter=limiter)
    G.run(wl.dt, n)
    compare(wl, G, ref, what=f"limiter={limiter}")
    G.close()


def test_empty_mask_is_predictor_and_mass_conserved():
    wl = _small_slide(n_members=2)
    n = 30
    ref = run_oracle(wl, n, crit=O.CRIT_HYDROSTATIC)
    G = make_gpu(wl, O.CRIT_HYDROSTATIC)
    st, i0 = G.step(wl.dt)
    m0 = i0["mass"]
    st, info = G.run(wl.dt, n - 1)
    assert info["last"]["n_active"] == 0 and info["last"]["solver"] == -1
    compare(wl, G, ref, what="hydrostatic")
    assert abs(info["last"]["mass"] - m0) <= 1e-13 * m0
    G.close()


@pytest.mark.parametrize("nx", [8, 9, 33, 255, 256, 257, 1000])
def test_ragged_and_tiny_grids(nx):
    """Grids from the minimum size through tile edges and ragged tails."""
    length = nx * 0.01
    wl = W.slide_1d(n_members=2, nx=nx, length=length, xc0=length * 0.4, L=length * 0.2,
                    A=0.01, T=0.05, seed0=3)
    n = 6
    ref = run_oracle(wl, n, crit=O.CRIT_GLOBAL)
    G = make_gpu(wl, O.CRIT_GLOBAL)
    G.run(wl.dt, n)
    compare(wl, G, ref, tol_eta=1e-8, what=f"nx={nx}")
    G.close()


def test_single_active_cell():
    """One marked cell, no enlargement: a 1x1 elliptic problem."""
    nx, dx = 64, 0.05
    d0 = np.full(nx, 1.0)
    h = d0.copy()
    h[30] += 0.01
    m = W.Member1D(nx=nx, dx=dx, xl=0.0, d0=d0, h=h, hu=np.zeros(nx), hw=np.zeros(nx))
    wl = W.Workload1D("one", [m], 1e-4, 1, 1e-4, amplitude=0.01)
    ref = run_oracle(wl, 1, crit=O.CRIT_ETA_D, enlarge=0, knh=5e-3)
    assert ref[0][2].sum() == 1
    G = make_gpu(wl, O.CRIT_ETA_D, enlarge=0, knh=5e-3)
    st, info = G.step(wl.dt)
    assert info["n_active"] == 1
    compare(wl, G, ref, what="single")
    G.close()


def test_not_converged_rolls_back():
    wl = _small_slide(n_members=2)
    G = make_gpu(wl, O.CRIT_GLOBAL, max_iter=2, rtol=1e-14)
    h0, hu0, hw0, _ = G.get_state()
    st, info = G.step(wl.dt, check=False)
    assert st == N.NH_ERR_NOT_CONVERGED
    h1, hu1, hw1, _ = G.get_state()
    assert np.array_equal(h0, h1) and np.array_equal(hu0, hu1) and np.array_equal(hw0, hw1)
    G.set_solver(N.NH_SOLVER_AUTO, 1e-12, 20000)
    st, info = G.step(wl.dt)
    assert st == N.NH_OK and info["step"] == 1
    G.close()


def test_full_size_slide_sampled_members():
    """The benchmark's launch configuration: 64 members x 50 000 cells in one
    batch, run until the non-hydrostatic region exists; members 0 and 63 are
    recomputed by the oracle and compared."""
    wl = W.slide_1d()
    n = 360
    G = make_gpu(wl, O.CRIT_ETA_D)
    st, info = G.run(wl.dt, n)
    assert info["last"]["n_active"] > 0
    sub = copy.copy(wl)
    sub.members = [wl.members[0], wl.members[63]]
    ref = run_oracle(sub, n, crit=O.CRIT_ETA_D)
    h, hu, hw, p = G.get_state()
    m, _, _ = G.get_mask()
    qscale = wl.amplitude * math.sqrt(9.81)
    for r, b in enumerate((0, 63)):
        s = ref[r][0]
        assert np.max(np.abs(h[b] - s.h)) <= 1e-9 * wl.amplitude
        assert np.max(np.abs(hu[b] - s.hu)) <= 1e-9 * qscale
        assert np.max(np.abs(hw[b] - s.hw)) <= 1e-9 * qscale
        assert np.array_equal(m[b], ref[r][2])
    G.close()
