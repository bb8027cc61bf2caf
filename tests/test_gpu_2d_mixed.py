"""2D grids with FP32 state (NH_MIXED_FP64_SOLVE) against the FP64 2D oracle.

The FP32 form stores zeta = h - d0, hu, hv, hw in FP32 and runs the predictor
and the criterion in FP32; assembly, Krylov solve and reductions stay FP64.
Bound: max |d eta| <= 1e-4 a and momenta <= 1e-4 a sqrt(g h_max) on every
step where the masks agree with the oracle's.  The FP32 state carries eta with
an absolute rounding of about 1e-7 m, so a cell whose criterion value lies
that close to k_nh may be marked on one side only; such a decision is
checked to be a near-tie of the oracle's own criterion value, and the runs
are not compared after it (the two methods then solve on different
sub-domains).  The lake at rest is exact in FP32; the captured-graph run
equals the step-by-step run bit for bit."""
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


def _params(nx, ny, dx, dy, crit, knh, enlarge=1, bc=O.BC_WALL, slide=None):
    p = O2.Params2D(nx=nx, ny=ny, dx=dx, dy=dy, bcx=bc, bcy=bc, crit=crit, knh=knh, enlarge=enlarge, rtol=1e-13)
    if slide:
        p.slide = O.SLIDE_GAUSS_LNCOSH
        for k, v in slide.items():
            setattr(p, k, v)
    return p


def _near_ties(p, d0, t, dt, s, cells, rel=1e-3):
    """True when, for every differing mask cell, some cell of its Moore
    enlargement has an oracle criterion value within rel of k_nh on the
    oracle's predicted state of the step from time t (state s before it)."""
    ht, hut, hvt, hwt = O2.predict(p, d0, t, dt, *(a.reshape(p.ny, p.nx) for a in (s.h, s.hu, s.hv, s.hw)))
    c = O2.criterion(p, d0, t + dt, ht, hut, hvt, hwt)
    e = p.enlarge
    for j, i in zip(*np.nonzero(cells)):
        win = c[max(0, j - e):j + e + 1, max(0, i - e):i + e + 1]
        if not np.any(np.abs(win - p.knh) <= rel * p.knh):
            return False
    return True


def _stepwise(p, d0, G, dt, n, amp, hmax, t0=0.0):
    """Oracle and GPU step by step: the errors while the masks agree, and the
    first step whose masks differ (checked to be a near-tie), or None."""
    s = O2.State2D(*[np.asarray(a) for a in G.get_state()[:4]])
    worst = 0.0
    for k in range(n):
        before = O2.State2D(s.h, s.hu, s.hv, s.hw, s.q)
        st, info, m = O2.step(p, d0, t0 + k * dt, k, dt, s, want_mask=True)
        assert st == O.OK, (k, info)
        G.step(dt)
        gm = G.get_mask()
        if not np.array_equal(gm, m):
            assert _near_ties(p, d0, t0 + k * dt, dt, before, gm != m), k
            return worst, k + 1
        de, dm = _err(s.fields(p), G.get_state(), amp, hmax)
        worst = max(worst, de, dm)
        assert de <= 1e-4 and dm <= 1e-4, (k, de, dm)
    return worst, None


def test_mixed_slide_matches_oracle():
    """Walled slope with a moving elliptic slide, adaptive |eta/d| > 1e-4."""
    nx, ny, dx, dy = 45, 31, 0.06, 0.07
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    X, Y = np.meshgrid(x, y)
    d0 = 0.3 + 0.2 * X + 0.03 * np.sin(2.3 * X + 1.1 * Y)
    sl = dict(A=0.06, Lx=0.5, Ly=0.35, xc0=0.9, yc0=0.55 * ny * dy, s0=1.5, t0=1.0)
    p = _params(nx, ny, dx, dy, O.CRIT_ETA_D, 1e-4, slide=sl)
    h = np.array([[O2.bottom(p, d0, i, j, 0.0)[0] for i in range(nx)] for j in range(ny)])
    z = np.zeros((ny, nx))
    dt = W.cfl_dt_2d(0.4, dx, dy, math.sqrt(9.81 * h.max()))
    G = _grid(nx, ny, dx, dy, d0, (h, z, z, z), N.NH_CRIT_ETA_D, 1e-4, slide=sl)
    worst, flip = _stepwise(p, d0, G, dt, 40, sl["A"], h.max())
    print(f"2D FP32 state, walled slide: worst error {worst:.2e} a while masks agree; first flip {flip}")


@pytest.mark.parametrize("nx,ny,bc", [(3, 3, O.BC_WALL), (5, 17, O.BC_WALL), (33, 9, O.BC_PERIODIC),
                                      (40, 21, O.BC_WALL), (37, 36, O.BC_PERIODIC)])
def test_fused_predictor_small_and_ragged_grids(nx, ny, bc):
    """The one-launch FP32 predictor on grids smaller than, equal to and
    ragged against its 32 x 16 tile, walled and periodic, global mask: every
    step within 1e-4 a of the oracle."""
    dx = 0.05
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    X, Y = np.meshgrid(x, y)
    Lx, Ly = nx * dx, ny * dx
    d0 = 0.4 + 0.05 * np.cos(2 * np.pi * X / Lx) * np.cos(2 * np.pi * Y / Ly)
    eta = 0.02 * np.exp(-((X - 0.4 * Lx) ** 2 + (Y - 0.6 * Ly) ** 2) / (0.05 * (Lx * Lx + Ly * Ly)))
    h = d0 + eta
    hu = 0.01 * h * np.sin(2 * np.pi * Y / Ly)
    hv = 0.005 * h * np.cos(2 * np.pi * X / Lx)
    hw = 0.001 * eta
    dt = W.cfl_dt_2d(0.4, dx, dx, math.sqrt(9.81 * h.max()) + 0.05)
    p = _params(nx, ny, dx, dx, O.CRIT_GLOBAL, 1e-3, bc=bc)
    G = _grid(nx, ny, dx, dx, d0, (h, hu, hv, hw), N.NH_CRIT_GLOBAL, 1e-3, bc=bc)
    worst, flip = _stepwise(p, d0, G, dt, 12, 0.02, h.max())
    assert flip is None
    print(f"fused FP32 predictor {nx}x{ny} bc={bc}: worst {worst:.2e} a")


def test_mixed_line_soliton_full_size():
    """The 2D solitary-wave workload (1024^2, a/h = 0.2, periodic, adaptive
    |eta/d| > 1e-3) with FP32 state for 5 captured steps, every cell against
    the FP64 oracle; differing mask cells must be near-ties."""
    wl = W.line_soliton_2d()
    n = 5
    p = _params(wl.nx, wl.ny, wl.dx, wl.dy, O.CRIT_ETA_D, 1e-3, bc=O.BC_PERIODIC)
    s = O2.State2D(wl.h, wl.hu, wl.hv, wl.hw)
    masks = []
    before = None
    for k in range(n):
        before = O2.State2D(s.h, s.hu, s.hv, s.hw, s.q)
        st, info, m = O2.step(p, wl.d0, k * wl.dt, k, wl.dt, s, want_mask=True)
        assert st == O.OK
        masks.append(m)
    G = _grid(wl.nx, wl.ny, wl.dx, wl.dy, wl.d0, (wl.h, wl.hu, wl.hv, wl.hw), N.NH_CRIT_ETA_D, 1e-3,
              bc=N.NH_BC_PERIODIC)
    st, info = G.run(wl.dt, n)
    assert info["steps"] == n and G.graph_runs == 1
    diff = G.get_mask() != masks[-1]
    if np.any(diff):
        assert _near_ties(p, wl.d0, (n - 1) * wl.dt, wl.dt, before, diff)
    else:
        de, dm = _err(s.fields(p), G.get_state(), wl.amplitude, wl.h.max())
        assert de <= 1e-4 and dm <= 1e-4, (de, dm)
    print(f"FP32 line soliton: {int(diff.sum())} mask cells differ after {n} steps")


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


def test_fused_predictor_tiles_give_identical_results():
    """Every tile candidate of the one-launch FP32 predictor (32 x 16, 64 x 8,
    32 x 8, 64 x 16) gives the same state bit for bit on an uneven ensemble
    (walls and periodic sides, sizes ragged against every tile); the autotuned
    choice is one of them."""
    members = []
    for m, (nx, ny, per) in enumerate(((70, 37, False), (33, 50, True), (129, 9, False))):
        dx = 0.05
        x = (np.arange(nx) + 0.5) * dx
        y = (np.arange(ny) + 0.5) * dx
        X, Y = np.meshgrid(x, y)
        d0 = 0.4 + 0.1 * X / (nx * dx)
        eta = 0.02 * np.exp(-((X - 0.3 * nx * dx) ** 2 + (Y - 0.5 * ny * dx) ** 2) / 0.1)
        members.append(dict(nx=nx, ny=ny, dx=dx, dy=dx, d0=d0, bc_x=int(per), bc_y=int(per),
                            q=(d0 + eta, 0.01 * (d0 + eta), np.zeros_like(d0), 0.001 * eta)))
    out = []
    for tile in (0, 1, 2, 3, None):
        G = N.Grid2D.ensemble([{k: v for k, v in mm.items() if k != "q"} for mm in members])
        G.set_precision(N.NH_MIXED_FP64_SOLVE)
        G.set_criterion(N.NH_CRIT_ETA_D, 1e-3, 1)
        G.set_solver(1e-12, 20000, N.NH_GUESS_PREV)
        for i, mm in enumerate(members):
            G.set_state(*mm["q"], member=i)
        if tile is not None:
            assert G.set_tile(tile) == tile
        G.run(0.004, 6)
        out.append([G.get_state(i)[:4] for i in range(len(members))])
        chosen = G.set_tile(-1)
        assert chosen in (0, 1, 2, 3)
        G.close()
    for s in out[1:]:
        for i in range(len(members)):
            for q in range(4):
                assert np.array_equal(s[i][q], out[0][i][q]), (i, q)
