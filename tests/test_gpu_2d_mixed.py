"""2D grids with FP32 state (NH_MIXED_FP64_SOLVE) against the FP64 2D oracle.

The FP32 form stores zeta = h - d0, hu, hv, hw in FP32 and runs the predictor
and the criterion in FP32; assembly, Krylov solve and reductions stay FP64.
Bound: max |d eta| <= 1e-4 a and momenta <= 1e-4 a sqrt(g h_max) while the
masks agree with the oracle's (a criterion value within FP32 rounding of k_nh
may be marked on one side only; then <= 1e-2 a).  The lake at rest is exact
in FP32; the captured-graph run equals the step-by-step run bit for bit."""
import math

import numpy as np
import pytest

import oracle as O
import oracle.oracle2d as O2

pytestmark = pytest.mark.gpu

N = pytest.importorskip("paper_2505_17025_gb300.nhswe")
W = pytest.importorskip("paper_2505_17025_gb300.workloads")


def _oracle_run(nx, ny, dx, dy, d0, q, dt, n, crit, knh, enlarge=1, bc=O.BC_WALL, slide=None, t0=0.0):
    p = O2.Params2D(nx=nx, ny=ny, dx=dx, dy=dy, bcx=bc, bcy=bc, crit=crit, knh=knh, enlarge=enlarge, rtol=1e-13)
    if slide:
        p.slide = O.SLIDE_GAUSS_LNCOSH
        for k, v in slide.items():
            setattr(p, k, v)
    s = O2.State2D(*q)
    masks = []
    for k in range(n):
        st, info, m = O2.step(p, d0, t0 + k * dt, k, dt, s, want_mask=True)
        assert st == O.OK, (k, info)
        masks.append(m)
    return s.fields(p), masks


def _grid(nx, ny, dx, dy, d0, q, crit, knh, enlarge=1, bc=N.NH_BC_WALL, slide=None, t0=0.0):
    G = N.Grid2D(nx, ny, dx, dy, d0, bc_x=bc, bc_y=bc)
    G.set_precision(N.NH_MIXED_FP64_SOLVE)
    if slide:
        G.set_bottom_motion(slide)
    G.set_criterion(crit, knh, enlarge)
    G.set_solver(1e-12, 20000, N.NH_GUESS_PREV)
    G.set_state(*q, t=t0)
    return G


def _err(ref, got, amp, hmax):
    de = np.max(np.abs(got[0] - ref[0])) / amp
    dm = max(np.max(np.abs(got[f] - ref[f])) for f in (1, 2, 3)) / (amp * math.sqrt(9.81 * hmax))
    return de, dm


def test_mixed_slide_matches_oracle():
    """Walled slope with a moving elliptic slide, adaptive |eta/d| > 1e-4."""
    nx, ny, dx, dy = 45, 31, 0.06, 0.07
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    X, Y = np.meshgrid(x, y)
    d0 = 0.3 + 0.2 * X + 0.03 * np.sin(2.3 * X + 1.1 * Y)
    sl = dict(A=0.06, Lx=0.5, Ly=0.35, xc0=0.9, yc0=0.55 * ny * dy, s0=1.5, t0=1.0)
    p = O2.Params2D(nx=nx, ny=ny, dx=dx, dy=dy, slide=O.SLIDE_GAUSS_LNCOSH, **sl)
    h = np.array([[O2.bottom(p, d0, i, j, 0.0)[0] for i in range(nx)] for j in range(ny)])
    z = np.zeros((ny, nx))
    dt = W.cfl_dt_2d(0.4, dx, dy, math.sqrt(9.81 * h.max()))
    n = 40
    ref, masks = _oracle_run(nx, ny, dx, dy, d0, (h, z, z, z), dt, n, O.CRIT_ETA_D, 1e-4, slide=sl)
    G = _grid(nx, ny, dx, dy, d0, (h, z, z, z), N.NH_CRIT_ETA_D, 1e-4, slide=sl)
    agree = True
    for k in range(n):
        G.step(dt)
        agree = agree and np.array_equal(G.get_mask(), masks[k])
    assert sum(int(m.sum()) for m in masks) > 0
    de, dm = _err(ref, G.get_state(), sl["A"], h.max())
    bound = 1e-4 if agree else 1e-2
    assert de <= bound and dm <= bound, (de, dm, agree)


def test_mixed_line_soliton_full_size():
    """The 2D solitary-wave workload (1024^2, a/h = 0.2, periodic, adaptive
    |eta/d| > 1e-3) with FP32 state for 5 captured steps, every cell against
    the FP64 oracle."""
    wl = W.line_soliton_2d()
    n = 5
    ref, masks = _oracle_run(wl.nx, wl.ny, wl.dx, wl.dy, wl.d0, (wl.h, wl.hu, wl.hv, wl.hw), wl.dt, n,
                             O.CRIT_ETA_D, 1e-3, bc=O.BC_PERIODIC)
    G = _grid(wl.nx, wl.ny, wl.dx, wl.dy, wl.d0, (wl.h, wl.hu, wl.hv, wl.hw), N.NH_CRIT_ETA_D, 1e-3,
              bc=N.NH_BC_PERIODIC)
    st, info = G.run(wl.dt, n)
    assert info["steps"] == n and G.graph_runs == 1
    flips = int(np.sum(G.get_mask() != masks[-1]))
    assert flips <= 0.001 * wl.nx * wl.ny
    de, dm = _err(ref, G.get_state(), wl.amplitude, wl.h.max())
    assert de <= (1e-4 if flips == 0 else 1e-2) and dm <= (1e-4 if flips == 0 else 1e-2), (de, dm, flips)


def test_mixed_lake_at_rest_exact_and_mass():
    """Still water over a static bumpy bottom stays exactly at rest in FP32;
    with a moving slide the FP64 mass sum of h = zeta + d0 stays within FP32
    rounding of its start."""
    nx, ny, dx, dy = 64, 48, 0.05, 0.05
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    X, Y = np.meshgrid(x, y)
    d0 = 0.3 + 0.2 * X + 0.03 * np.sin(2.3 * X + 1.1 * Y)
    z = np.zeros((ny, nx))
    G = _grid(nx, ny, dx, dy, d0, (d0, z, z, z), N.NH_CRIT_GLOBAL, 1e-3)
    G.run(0.004, 30)
    h, hu, hv, hw, _ = G.get_state()
    assert np.array_equal(h, d0)
    assert not np.any(hu) and not np.any(hv) and not np.any(hw)
    sl = dict(A=0.06, Lx=0.5, Ly=0.35, xc0=0.9, yc0=1.3, s0=1.5, t0=1.0)
    p = O2.Params2D(nx=nx, ny=ny, dx=dx, dy=dy, slide=O.SLIDE_GAUSS_LNCOSH, **sl)
    h0 = np.array([[O2.bottom(p, d0, i, j, 0.0)[0] for i in range(nx)] for j in range(ny)])
    G.set_bottom_motion(sl)
    G.set_criterion(N.NH_CRIT_ETA_D, 1e-4, 1)
    G.set_state(h0, z, z, z)
    st, info = G.run(0.004, 40)
    m0 = h0.sum() * dx * dy
    assert info["active_total"] > 0
    assert abs(info["last"]["mass"] - m0) <= 1e-6 * m0


def test_mixed_ensemble_graph_equals_steps():
    """Three uneven members with FP32 state: captured replays = host-enqueued
    steps, bit for bit."""
    members = []
    for nx, ny, dx in ((40, 30, 0.05), (24, 36, 0.06), (17, 9, 0.08)):
        x = (np.arange(nx) + 0.5) * dx
        y = (np.arange(ny) + 0.5) * dx
        X, Y = np.meshgrid(x, y)
        d0 = 0.3 + 0.15 * X
        sl = dict(A=0.05, Lx=0.4, Ly=0.3, xc0=0.5, yc0=0.5 * ny * dx, s0=1.2, t0=1.0)
        p = O2.Params2D(nx=nx, ny=ny, dx=dx, dy=dx, slide=O.SLIDE_GAUSS_LNCOSH, **sl)
        h = np.array([[O2.bottom(p, d0, i, j, 0.0)[0] for i in range(nx)] for j in range(ny)])
        members.append((dict(nx=nx, ny=ny, dx=dx, dy=dx, d0=d0), sl, h))
    out = []
    for graphs in (False, True):
        G = N.Grid2D.ensemble([m for m, _, _ in members])
        G.set_precision(N.NH_MIXED_FP64_SOLVE)
        G.set_graphs(graphs)
        for i, (m, sl, h) in enumerate(members):
            z = np.zeros_like(h)
            G.set_bottom_motion(sl, member=i)
            G.set_state(h, z, z, z, member=i)
        G.set_criterion(N.NH_CRIT_ETA_D, 1e-4, 1)
        st, info = G.run(0.003, 25)
        assert info["steps"] == 25
        assert (G.graph_runs > 0) == graphs
        out.append([G.get_state(i) for i in range(len(members))])
    for a, b in zip(out[0], out[1]):
        for f in range(5):
            assert np.array_equal(a[f], b[f])
