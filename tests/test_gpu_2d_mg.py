"""The multigrid-preconditioned CG of 2D grids (nh_mg2d.cuh) against the 2D
FP64 oracle and against the line-preconditioned solve.

The preconditioner changes the iteration, not the solution: both solves stop
at ||r|| <= 1e-12 ||R||, so the states agree with the oracle to the FP64
parity bound (|d eta| <= 1e-9 a, momenta 1e-9 a sqrt(g h_max)) and with each
other.  Cases: a large global problem (one member split over several CTAs,
with the group barrier), periodic sides whose whole extent is active (coarse
levels that wrap, odd widths), a walled slide with a moving mask, an uneven
ensemble (members of one CTA each), and the full-size landslide, where the
multigrid solve must need far fewer iterations than the line solve.
"""
import math

import numpy as np
import pytest

import oracle as O
import oracle.oracle2d as O2

pytestmark = pytest.mark.gpu

N = pytest.importorskip("paper_2505_17025_gb300.nhswe")
W = pytest.importorskip("paper_2505_17025_gb300.workloads")


def _oracle_run(nx, ny, dx, d0, h, hu, hv, hw, dt, n, crit, knh, bcx=0, bcy=0, slide=None):
    p = O2.Params2D(nx=nx, ny=ny, dx=dx, dy=dx, bcx=bcx, bcy=bcy, crit=crit, knh=knh, enlarge=1, rtol=1e-13)
    if slide:
        p.slide = O.SLIDE_GAUSS_LNCOSH
        for k, v in slide.items():
            setattr(p, k, v)
    s = O2.State2D(h, hu, hv, hw)
    masks = []
    for k in range(n):
        st, info, m = O2.step(p, d0, k * dt, k, dt, s, want_mask=True)
        assert st == O.OK, (k, info)
        masks.append(m)
    return s.fields(p), masks


def _gpu_run(nx, ny, dx, d0, h, hu, hv, hw, dt, n, crit, knh, precond, bcx=0, bcy=0, slide=None):
    G = N.Grid2D(nx, ny, dx, dx, d0, bc_x=bcx, bc_y=bcy)
    if slide:
        G.set_bottom_motion(slide)
    G.set_criterion(crit, knh, 1)
    G.set_solver(1e-12, 20000, N.NH_GUESS_PREV)
    G.set_preconditioner(precond)
    G.set_state(h, hu, hv, hw)
    masks, iters = [], []
    for k in range(n):
        st, info = G.step(dt)
        masks.append(G.get_mask())
        iters.append(info["iters"])
    out = G.get_state()
    G.close()
    return out, masks, iters


def _check(ref, got, amp, hmax, what):
    deta = float(np.max(np.abs(got[0] - ref[0])))
    assert deta <= 1e-9 * amp, (what, deta / amp)
    mom = 1e-9 * amp * math.sqrt(9.81 * hmax)
    for q in (1, 2, 3):
        assert np.max(np.abs(got[q] - ref[q])) <= mom, (what, q)
    return deta / amp


def _hump(nx, ny, dx, periodic):
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    X, Y = np.meshgrid(x, y)
    Lx, Ly = nx * dx, ny * dx
    if periodic:
        d0 = 0.6 + 0.08 * np.sin(2 * np.pi * X / Lx) * np.cos(2 * np.pi * Y / Ly)
    else:
        d0 = 0.4 + 0.15 * X / Lx + 0.03 * np.sin(3.1 * X + 1.7 * Y)
    eta = 0.03 * np.exp(-((X - 0.45 * Lx) ** 2 + (Y - 0.55 * Ly) ** 2) / (0.02 * Lx * Ly))
    h = d0 + eta
    hu = 0.01 * h * np.sin(2 * np.pi * Y / Ly)
    hv = -0.008 * h
    hw = 0.001 * eta
    return d0, h, hu, hv, hw


@pytest.mark.parametrize("nx,ny,periodic", [(150, 120, False), (97, 83, True)])
def test_global_multi_cta_member_matches_oracle_and_line(nx, ny, periodic):
    """One member with every cell active: 18 000 (walls) and 8 051 (periodic,
    odd sizes: the coarse levels wrap) rows, so the member's solve runs on
    several CTAs joined by the group barrier."""
    dx = 0.05
    d0, h, hu, hv, hw = _hump(nx, ny, dx, periodic)
    bc = O.BC_PERIODIC if periodic else O.BC_WALL
    dt = W.cfl_dt_2d(0.4, dx, dx, math.sqrt(9.81 * h.max()) + 0.05)
    n = 6
    ref, mo = _oracle_run(nx, ny, dx, d0, h, hu, hv, hw, dt, n, O.CRIT_GLOBAL, 1e-3, bc, bc)
    mg, _, it_mg = _gpu_run(nx, ny, dx, d0, h, hu, hv, hw, dt, n, N.NH_CRIT_GLOBAL, 1e-3, N.NH_PRECOND_MG, bc, bc)
    line, _, it_line = _gpu_run(nx, ny, dx, d0, h, hu, hv, hw, dt, n, N.NH_CRIT_GLOBAL, 1e-3, N.NH_PRECOND_LINE,
                                bc, bc)
    e_mg = _check(ref, mg, 0.03, h.max(), "mg")
    e_line = _check(ref, line, 0.03, h.max(), "line")
    print(f"{nx}x{ny} periodic={periodic}: iterations per step MG {it_mg}, line {it_line}; "
          f"|d eta|/a MG {e_mg:.1e}, line {e_line:.1e}")
    assert max(it_mg) < max(it_line)


def test_walled_slide_moving_mask_matches_oracle():
    nx, ny, dx = 64, 48, 0.05
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    X, Y = np.meshgrid(x, y)
    d0 = 0.2 + 0.25 * X
    sl = dict(A=0.06, Lx=0.5, Ly=0.3, xc0=0.8, yc0=0.5 * ny * dx, s0=1.5, t0=1.0)
    p = O2.Params2D(nx=nx, ny=ny, dx=dx, dy=dx, slide=O.SLIDE_GAUSS_LNCOSH, **sl)
    h = np.array([[O2.bottom(p, d0, i, j, 0.0)[0] for i in range(nx)] for j in range(ny)])
    z = np.zeros((ny, nx))
    dt = W.cfl_dt_2d(0.4, dx, dx, math.sqrt(9.81 * h.max()))
    n = 30
    ref, mo = _oracle_run(nx, ny, dx, d0, h, z, z, z, dt, n, O.CRIT_ETA_D, 1e-4, slide=sl)
    got, mg, it = _gpu_run(nx, ny, dx, d0, h, z, z, z, dt, n, N.NH_CRIT_ETA_D, 1e-4, N.NH_PRECOND_MG, slide=sl)
    for k, (a, b) in enumerate(zip(mo, mg)):
        assert np.array_equal(a, b), k
    assert sum(int(m.sum()) for m in mo) > 0
    _check(ref, got, sl["A"], h.max(), "slide")


def test_uneven_ensemble_mg_equals_members_alone():
    """Three uneven members in one handle (one CTA each) give what each gives
    alone, and the captured-graph run equals the step-by-step run bit for bit."""
    sizes = [(40, 31), (23, 57), (71, 18)]
    members = []
    for m, (nx, ny) in enumerate(sizes):
        d0, h, hu, hv, hw = _hump(nx, ny, 0.05, periodic=(m == 1))
        members.append((nx, ny, d0, h, hu, hv, hw))
    dt = 0.004
    n = 12

    def ensemble(graphs):
        G = N.Grid2D.ensemble([dict(nx=m[0], ny=m[1], dx=0.05, dy=0.05, d0=m[2],
                                    bc_x=O.BC_PERIODIC if i == 1 else O.BC_WALL,
                                    bc_y=O.BC_PERIODIC if i == 1 else O.BC_WALL)
                               for i, m in enumerate(members)])
        G.set_criterion(N.NH_CRIT_ETA_D, 1e-3, 1)
        G.set_solver(1e-12, 20000, N.NH_GUESS_PREV)
        for i, m in enumerate(members):
            G.set_state(*m[3:], member=i)
        G.set_graphs(graphs)
        G.run(dt, n)
        out = [G.get_state(i) for i in range(len(members))]
        G.close()
        return out

    a = ensemble(False)
    b = ensemble(True)
    for i, m in enumerate(members):
        for q in range(4):
            assert np.array_equal(a[i][q], b[i][q]), (i, q)
        bc = O.BC_PERIODIC if i == 1 else O.BC_WALL
        ref, _ = _oracle_run(m[0], m[1], 0.05, m[2], *m[3:], dt, n, O.CRIT_ETA_D, 1e-3, bc, bc)
        _check(ref, a[i], 0.03, m[3].max(), f"member {i}")


def test_landslide_full_size_fewer_iterations():
    """The 2048^2 landslide from t = 0.3 s: the multigrid solve and the line
    solve give the same state, the multigrid one in far fewer iterations."""
    wl = W.landslide_2d()
    t0 = 0.3
    sl = wl.slide
    s = sl["s0"] * math.log(math.cosh(t0 / sl["t0"]))
    x = (np.arange(wl.nx) + 0.5) * wl.dx
    y = (np.arange(wl.ny) + 0.5) * wl.dy
    X, Y = np.meshgrid(x, y)
    h = wl.d0 - sl["A"] * np.exp(-((X - sl["xc0"] - s) / sl["Lx"]) ** 2 - ((Y - sl["yc0"]) / sl["Ly"]) ** 2)
    out = {}
    for pc in (N.NH_PRECOND_MG, N.NH_PRECOND_LINE):
        G = N.Grid2D(wl.nx, wl.ny, wl.dx, wl.dy, wl.d0)
        G.set_bottom_motion(sl)
        G.set_criterion(N.NH_CRIT_ETA_D, 1e-4, 1)
        G.set_solver(1e-12, 20000, N.NH_GUESS_PREV)
        G.set_preconditioner(pc)
        G.set_state(h, wl.hu, wl.hv, wl.hw, t=t0)
        its = []
        for k in range(8):
            st, info = G.step(wl.dt)
            its.append(info["iters"])
        out[pc] = (G.get_state(), its)
        G.close()
    (smg, imgs), (sline, ilines) = out[N.NH_PRECOND_MG], out[N.NH_PRECOND_LINE]
    print(f"landslide 2048^2: iterations per step MG {imgs}, line {ilines}")
    a = sl["A"]
    assert np.max(np.abs(smg[0] - sline[0])) <= 1e-9 * a
    assert sum(imgs) * 3 <= sum(ilines)
