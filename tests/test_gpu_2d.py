"""The 2D grid on the GPU against the 2D FP64 oracle (oracle/nh_oracle2d.c).

Tolerance as for the 1D FP64 path: max |d eta| <= 1e-9 a and
max |d hu|, |d hv|, |d hw| <= 1e-9 a sqrt(g h_max) (a = the wave or slide
amplitude); masks bit for bit.  Cases span walls and periodic sides, ragged
sizes, every criterion family, limiters, the moving 2D slide (cross terms of
the 9-point operator) and the two 2D workloads at their full sizes (a few
steps), plus the y-uniform reduction against the 1D GPU path."""
import math

import numpy as np
import pytest

import oracle as O
import oracle.oracle2d as O2

pytestmark = pytest.mark.gpu

N = pytest.importorskip("paper_2505_17025_gb300.nhswe")
W = pytest.importorskip("paper_2505_17025_gb300.workloads")

_CRIT = {O.CRIT_GLOBAL: N.NH_CRIT_GLOBAL, O.CRIT_HYDROSTATIC: N.NH_CRIT_HYDROSTATIC,
         O.CRIT_ETA_D: N.NH_CRIT_ETA_D, O.CRIT_ETA_X: N.NH_CRIT_ETA_X, O.CRIT_U: N.NH_CRIT_U,
         O.CRIT_U_X: N.NH_CRIT_U_X, O.CRIT_W: N.NH_CRIT_W, O.CRIT_W_X: N.NH_CRIT_W_X}


def _case(nx, ny, dx, dy, slide=True, bump=True):
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    X, Y = np.meshgrid(x, y)
    d0 = 0.3 + 0.2 * X
    if bump:
        d0 = d0 + 0.03 * np.sin(2.3 * X + 1.1 * Y)
    sl = dict(A=0.06, Lx=0.5, Ly=0.35, xc0=0.9, yc0=0.55 * ny * dy, s0=1.5, t0=1.0) if slide else None
    return X, Y, d0, sl


def _run_both(nx, ny, dx, dy, d0, h, hu, hv, hw, dt, n, crit, knh, enlarge=1, bcx=0, bcy=0, lim=O.LIM_CENTRAL,
              slide=None, first=0):
    p = O2.Params2D(nx=nx, ny=ny, dx=dx, dy=dy, bcx=bcx, bcy=bcy, limiter=lim, crit=crit, knh=knh,
                    enlarge=enlarge, first_step_global=first, rtol=1e-13)
    if slide:
        p.slide = O.SLIDE_GAUSS_LNCOSH
        for k, v in slide.items():
            setattr(p, k, v)
    s = O2.State2D(h, hu, hv, hw)
    masks_o = []
    for k in range(n):
        st, info, m = O2.step(p, d0, k * dt, k, dt, s, want_mask=True)
        assert st == O.OK, (k, info)
        masks_o.append(m)
    G = N.Grid2D(nx, ny, dx, dy, d0, bc_x=bcx, bc_y=bcy, limiter=lim)
    if slide:
        G.set_bottom_motion(slide)
    G.set_criterion(_CRIT[crit], knh, enlarge, bool(first))
    G.set_solver(1e-12, 20000, N.NH_GUESS_PREV)
    G.set_state(h, hu, hv, hw)
    masks_g = []
    for k in range(n):
        st, info = G.step(dt)
        masks_g.append(G.get_mask())
    return s.fields(p), G.get_state(), masks_o, masks_g


def _compare(ref, got, amp, hmax, what):
    h_o, hu_o, hv_o, hw_o, _ = ref
    h_g, hu_g, hv_g, hw_g, _ = got
    deta = np.max(np.abs(h_g - h_o))
    assert deta <= 1e-9 * amp, (what, deta / amp)
    mom = 1e-9 * amp * math.sqrt(9.81 * hmax)
    for name, a, b in (("hu", hu_g, hu_o), ("hv", hv_g, hv_o), ("hw", hw_g, hw_o)):
        assert np.max(np.abs(a - b)) <= mom, (what, name, np.max(np.abs(a - b)))
    return deta / amp


@pytest.mark.parametrize("crit,knh,enlarge,first", [(O.CRIT_ETA_D, 1e-4, 1, 0), (O.CRIT_GLOBAL, 1e-3, 1, 0),
                                                    (O.CRIT_ETA_X, 2e-4, 2, 0), (O.CRIT_U_X, 1e-3, 1, 0),
                                                    (O.CRIT_W, 1e-6, 0, 1)])
def test_slide_matches_oracle(crit, knh, enlarge, first):
    """Walls, ragged size, moving 2D slide on a bumpy slope: state and masks.
    The |w| criterion starts with the first step global (Sec. 5.1.2): from
    rest hw only grows through the correction."""
    nx, ny, dx, dy = 45, 31, 0.06, 0.07
    X, Y, d0, sl = _case(nx, ny, dx, dy)
    p = O2.Params2D(nx=nx, ny=ny, dx=dx, dy=dy, slide=O.SLIDE_GAUSS_LNCOSH, **sl)
    h = np.array([[O2.bottom(p, d0, i, j, 0.0)[0] for i in range(nx)] for j in range(ny)])
    z = np.zeros((ny, nx))
    dt = W.cfl_dt_2d(0.4, dx, dy, math.sqrt(9.81 * h.max()))
    ref, got, mo, mg = _run_both(nx, ny, dx, dy, d0, h, z, z, z, dt, 25, crit, knh, enlarge, slide=sl,
                                 first=first)
    for k, (a, b) in enumerate(zip(mo, mg)):
        assert np.array_equal(a, b), (k, int(np.sum(a != b)))
    assert sum(int(m.sum()) for m in mo) > 0
    _compare(ref, got, sl["A"], h.max(), f"crit {crit}")


@pytest.mark.parametrize("lim", [O.LIM_MINMOD, O.LIM_MC])
def test_periodic_hump_matches_oracle(lim):
    """Periodic in x and y, static bumpy bottom, a Gaussian hump with a flow."""
    nx, ny, dx, dy = 40, 36, 0.05, 0.05
    X, Y, d0, _ = _case(nx, ny, dx, dy, slide=False)
    d0 = 0.5 + 0.05 * np.sin(2 * np.pi * X / (nx * dx)) * np.cos(2 * np.pi * Y / (ny * dy))
    eta = 0.03 * np.exp(-((X - 1.0) ** 2 + (Y - 0.9) ** 2) / 0.05)
    h = d0 + eta
    hu = 0.02 * h * np.sin(2 * np.pi * Y / (ny * dy))
    hv = -0.015 * h
    hw = 0.002 * eta
    dt = W.cfl_dt_2d(0.4, dx, dy, math.sqrt(9.81 * h.max()) + 0.05)
    ref, got, mo, mg = _run_both(nx, ny, dx, dy, d0, h, hu, hv, hw, dt, 20, O.CRIT_ETA_D, 1e-3, 1,
                                 bcx=O.BC_PERIODIC, bcy=O.BC_PERIODIC, lim=lim)
    for a, b in zip(mo, mg):
        assert np.array_equal(a, b)
    _compare(ref, got, 0.03, h.max(), f"periodic lim {lim}")


def test_first_step_global_and_tiny_grid():
    nx, ny, dx, dy = 9, 7, 0.1, 0.12
    X, Y, d0, sl = _case(nx, ny, dx, dy)
    p = O2.Params2D(nx=nx, ny=ny, dx=dx, dy=dy, slide=O.SLIDE_GAUSS_LNCOSH, **sl)
    h = np.array([[O2.bottom(p, d0, i, j, 0.0)[0] for i in range(nx)] for j in range(ny)])
    z = np.zeros((ny, nx))
    dt = W.cfl_dt_2d(0.4, dx, dy, math.sqrt(9.81 * h.max()))
    ref, got, mo, mg = _run_both(nx, ny, dx, dy, d0, h, z, z, z, dt, 6, O.CRIT_W_X, 1e-2, 1, slide=sl, first=1)
    assert mo[0].sum() == nx * ny
    for a, b in zip(mo, mg):
        assert np.array_equal(a, b)
    _compare(ref, got, sl["A"], h.max(), "tiny")


def test_y_uniform_equals_1d_gpu():
    """A line soliton replicated in y (periodic) on the 2D grid gives the 1D
    GPU path's result in every row."""
    wl = W.solitary_1d(nx=600, length=60.0, a=0.1, T=3.0)
    m = wl.members[0]
    ny = 6
    G1 = N.grid_from_workload(wl)
    G1.set_criterion(N.NH_CRIT_ETA_D, 1e-3, 1, False)
    G1.set_solver(N.NH_SOLVER_AUTO, 1e-12, 20000, N.NH_GUESS_PREV)
    G1.run(wl.dt, 50)
    h1, hu1, hw1, _ = G1.get_state()
    rep = lambda a: np.tile(np.asarray(a, dtype=np.float64), (ny, 1))
    G2 = N.Grid2D(m.nx, ny, m.dx, 0.3, rep(m.d0), bc_y=N.NH_BC_PERIODIC)
    G2.set_criterion(N.NH_CRIT_ETA_D, 1e-3, 1)
    G2.set_solver(1e-12, 20000, N.NH_GUESS_PREV)
    G2.set_state(rep(m.h), rep(m.hu), np.zeros((ny, m.nx)), rep(m.hw))
    G2.run(wl.dt, 50)
    h2, hu2, hv2, hw2, _ = G2.get_state()
    for row in range(ny):
        assert np.max(np.abs(h2[row] - h1[0])) <= 1e-10 * wl.amplitude
        assert np.max(np.abs(hu2[row] - hu1[0])) <= 1e-10 * wl.amplitude * math.sqrt(9.81)
    assert np.max(np.abs(hv2)) <= 1e-12


def test_line_soliton_full_size():
    """The 2D solitary-wave workload (1024 x 1024, dx = 0.05 m, a/h = 0.2,
    periodic, adaptive |eta/d| > 1e-3) for 3 steps, every cell against the
    oracle."""
    wl = W.line_soliton_2d()
    ref, got, mo, mg = _run_both(wl.nx, wl.ny, wl.dx, wl.dy, wl.d0, wl.h, wl.hu, wl.hv, wl.hw, wl.dt, 3,
                                 O.CRIT_ETA_D, 1e-3, 1, bcx=O.BC_PERIODIC, bcy=O.BC_PERIODIC)
    for a, b in zip(mo, mg):
        assert np.array_equal(a, b)
    _compare(ref, got, wl.amplitude, wl.h.max(), "line soliton 1024^2")


def test_landslide_full_size():
    """The 2D landslide workload (2048 x 2048, dx = 0.02 m, elliptic slide on a
    0.2 slope, walls, adaptive |eta/d| > 1e-4) for 3 steps from t = 0.3 s,
    every cell against the oracle."""
    wl = W.landslide_2d()
    sl = wl.slide
    t0 = 0.3
    # start from the still water over the slide's position at t0
    s = sl["s0"] * math.log(math.cosh(t0 / sl["t0"]))
    x = (np.arange(wl.nx) + 0.5) * wl.dx
    X, Y = np.meshgrid(x, x)
    h = wl.d0 - sl["A"] * np.exp(-((X - sl["xc0"] - s) / sl["Lx"]) ** 2 - ((Y - sl["yc0"]) / sl["Ly"]) ** 2)
    z = np.zeros_like(h)
    p = O2.Params2D(nx=wl.nx, ny=wl.ny, dx=wl.dx, dy=wl.dy, crit=O.CRIT_ETA_D, knh=1e-4, enlarge=1, rtol=1e-13,
                    slide=O.SLIDE_GAUSS_LNCOSH, **sl)
    st_o = O2.State2D(h, z, z, z)
    masks_o = []
    for k in range(3):
        st, info, m = O2.step(p, wl.d0, t0 + k * wl.dt, k, wl.dt, st_o, want_mask=True)
        assert st == O.OK
        masks_o.append(m)
    assert masks_o[-1].sum() > 0
    G = N.Grid2D(wl.nx, wl.ny, wl.dx, wl.dy, wl.d0)
    G.set_bottom_motion(sl)
    G.set_criterion(N.NH_CRIT_ETA_D, 1e-4, 1)
    G.set_solver(1e-12, 20000, N.NH_GUESS_PREV)
    G.set_state(h, z, z, z, t=t0)
    for k in range(3):
        G.step(wl.dt)
        assert np.array_equal(G.get_mask(), masks_o[k]), k
    _compare(st_o.fields(p), G.get_state(), sl["A"], wl.d0.max(), "landslide 2048^2")


def test_mass_and_lake_at_rest_2d_gpu():
    """Walls: total mass constant while the slide moves; still water over a
    static bumpy bottom stays at rest."""
    nx, ny, dx, dy = 64, 48, 0.05, 0.05
    X, Y, d0, sl = _case(nx, ny, dx, dy)
    G = N.Grid2D(nx, ny, dx, dy, d0)
    G.set_criterion(N.NH_CRIT_GLOBAL, 1e-3, 1)
    z = np.zeros((ny, nx))
    G.set_state(d0, z, z, z)
    G.run(0.004, 30)
    h, hu, hv, hw, _ = G.get_state()
    assert np.max(np.abs(h - d0)) < 1e-13
    assert max(np.max(np.abs(hu)), np.max(np.abs(hv)), np.max(np.abs(hw))) < 1e-13
    p = O2.Params2D(nx=nx, ny=ny, dx=dx, dy=dy, slide=O.SLIDE_GAUSS_LNCOSH, **sl)
    h0 = np.array([[O2.bottom(p, d0, i, j, 0.0)[0] for i in range(nx)] for j in range(ny)])
    G.set_bottom_motion(sl)
    G.set_criterion(N.NH_CRIT_ETA_D, 1e-4, 1)
    G.set_state(h0, z, z, z)
    st, info = G.run(0.004, 40)
    assert info["active_total"] > 0
    assert abs(info["last"]["mass"] - h0.sum() * dx * dy) <= 1e-12 * h0.sum() * dx * dy
