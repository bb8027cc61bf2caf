"""Uneven ensembles (one handle, members with different cell counts) and
CUDA-graph replay of nh_run.

* every member of an uneven ensemble matches the FP64 oracle run on that
  member alone (|d eta| <= 1e-9 a, |d hu|, |d hw| <= 1e-9 a sqrt(g h_max));
* a graph-replayed nh_run gives the same state as the step-by-step path
  (same kernels and arithmetic: equal to 1e-13 relative);
* a step that fails inside a replay leaves the last accepted state intact.
"""
import copy

import numpy as np
import pytest

import oracle as O
from paper_2505_17025_gb300 import nhswe as N
from paper_2505_17025_gb300 import workloads as W

from _helpers import compare, make_gpu, run_oracle

pytestmark = pytest.mark.gpu


def _small_ensemble(n=4):
    wl = W.ensemble_1d(n_members=n, nx_min=512, nx_max=4096, T=0.2)
    return wl


def test_uneven_ensemble_matches_oracle_per_member():
    wl = _small_ensemble(4)
    assert len({m.nx for m in wl.members}) > 1
    nsteps = 60
    ref = run_oracle(wl, nsteps, crit=O.CRIT_ETA_D, knh=1e-4)
    G = make_gpu(wl, O.CRIT_ETA_D, knh=1e-4)
    G.set_run_mode(False)
    st, info = G.run(wl.dt, nsteps)
    h, hu, hw, p = G.get_state()
    m, _, _ = G.get_mask()
    a = wl.amplitude
    for b, (s, infos, mk) in enumerate(ref):
        q = a * np.sqrt(9.81 * np.max(wl.members[b].d0))
        assert np.max(np.abs(h[b] - s.h)) <= 1e-9 * a
        assert np.max(np.abs(hu[b] - s.hu)) <= 1e-9 * q
        assert np.max(np.abs(hw[b] - s.hw)) <= 1e-9 * q
        assert np.array_equal(m[b], mk)
    assert info["last"]["n_active"] == sum(int(r[2].sum()) for r in ref)
    G.close()


@pytest.mark.parametrize("uneven", [False, True])
def test_graph_run_equals_step_by_step(uneven):
    wl = _small_ensemble(3) if uneven else W.slide_1d(n_members=3, nx=2000, length=4.0, xc0=1.0,
                                                      T=0.5, seed0=11)
    n = 120
    A = make_gpu(wl, O.CRIT_ETA_D, knh=1e-4)
    B = make_gpu(wl, O.CRIT_ETA_D, knh=1e-4)
    B.set_run_mode(False)
    sa, ia = A.run(wl.dt, n // 2)
    sa2, ia2 = A.run(wl.dt, n - n // 2)
    for _ in range(n):
        B.step(wl.dt)
    ha, hua, hwa, pa = A.get_state()
    hb, hub, hwb, pb = B.get_state()
    for x, y in ((ha, hb), (hua, hub), (hwa, hwb), (pa, pb)):
        for b in range(len(wl.members)):
            xa, yb = np.asarray(x[b]), np.asarray(y[b])
            assert np.max(np.abs(xa - yb)) <= 1e-13 * max(np.max(np.abs(yb)), 1e-30)
    assert ia2["steps"] == n - n // 2 and ia2["last"]["step"] == n
    assert ia2["iters_total"] > 0
    A.close()
    B.close()


def test_graph_run_stops_at_failed_step_with_state_intact():
    wl = W.slide_1d(n_members=2, nx=2000, length=4.0, xc0=1.0, T=0.5, seed0=11)
    G = make_gpu(wl, O.CRIT_GLOBAL)
    G.run(wl.dt, 5)                       # graph-replayed, converges
    h5, hu5, hw5, _ = G.get_state()
    G.set_solver(N.NH_SOLVER_AUTO, 1e-15, 1, N.NH_GUESS_PREV)   # cannot converge in 1 iteration
    st, info = G.run(wl.dt, 4, check=False)
    assert st == N.NH_ERR_NOT_CONVERGED
    assert info["steps"] == 0
    h, hu, hw, _ = G.get_state()
    assert np.array_equal(h, h5) and np.array_equal(hu, hu5) and np.array_equal(hw, hw5)
    G.set_solver(N.NH_SOLVER_AUTO, 1e-12, 20000, N.NH_GUESS_PREV)
    st, info = G.run(wl.dt, 3)
    assert st == N.NH_OK and info["last"]["step"] == 8
    G.close()


def test_predictor_tiles_identical_and_autotuned():
    """Every predictor tile (128, 256, 512 cells per CTA) computes the same
    cells with the same arithmetic, so forced tiles give identical states;
    an untouched handle picks one of them on its first step."""
    wl = W.slide_1d(n_members=2, nx=3000, length=6.0, xc0=1.0, T=0.5, seed0=5)
    out = []
    for tile in (128, 256, 512):
        G = make_gpu(wl, O.CRIT_ETA_D, knh=1e-4)
        assert G.set_tile(tile) == tile
        G.run(wl.dt, 40)
        out.append(G.get_state())
        G.close()
    for st in out[1:]:
        for x, y in zip(st, out[0]):
            assert np.array_equal(np.asarray(x), np.asarray(y))
    G = make_gpu(wl, O.CRIT_ETA_D)
    assert G.set_tile(0) == 0
    G.step(wl.dt)
    assert G.set_tile(0) in (128, 256, 512)
    G.close()
