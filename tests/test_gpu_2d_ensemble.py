"""Ensembles of 2D grids on the GPU (nh2d_create_ensemble) against the 2D
FP64 oracle run on each member alone.

Members differ in size, spacing, sides, limiter, static depth and slide and
share one dt, criterion and solver setting.  Tolerances as for one grid:
max |d eta| <= 1e-9 a, momenta <= 1e-9 a sqrt(g h_max) per member (a = the
member's amplitude); masks bit for bit.  The captured-graph run (nh2d_run)
must give the step-by-step result bit for bit.  At full size (32 landslide
runs of 256^2 to 1024^2 cells) the smallest and the largest member are
compared with the oracle and every member's mass is checked."""
import math

import numpy as np
import pytest

import oracle as O
import oracle.oracle2d as O2

pytestmark = pytest.mark.gpu

N = pytest.importorskip("paper_2505_17025_gb300.nhswe")
W = pytest.importorskip("paper_2505_17025_gb300.workloads")

_LIM = {O.LIM_CENTRAL: N.NH_LIM_CENTRAL, O.LIM_MINMOD: N.NH_LIM_MINMOD, O.LIM_MC: N.NH_LIM_MC}


def _members():
    """Four uneven members: walled slides on bumpy slopes (two sizes), a
    periodic hump with a flow, a tiny walled grid."""
    out = []
    for (nx, ny, dx, dy, A, xc0, lim) in ((45, 31, 0.06, 0.07, 0.06, 0.9, O.LIM_CENTRAL),
                                          (30, 22, 0.08, 0.05, 0.04, 0.7, O.LIM_MINMOD),
                                          (9, 7, 0.1, 0.12, 0.05, 0.3, O.LIM_CENTRAL)):
        x = (np.arange(nx) + 0.5) * dx
        y = (np.arange(ny) + 0.5) * dy
        X, Y = np.meshgrid(x, y)
        d0 = 0.3 + 0.2 * X + 0.03 * np.sin(2.3 * X + 1.1 * Y)
        sl = dict(A=A, Lx=0.5, Ly=0.35, xc0=xc0, yc0=0.55 * ny * dy, s0=1.5, t0=1.0)
        p = O2.Params2D(nx=nx, ny=ny, dx=dx, dy=dy, slide=O.SLIDE_GAUSS_LNCOSH, **sl)
        h = np.array([[O2.bottom(p, d0, i, j, 0.0)[0] for i in range(nx)] for j in range(ny)])
        z = np.zeros((ny, nx))
        out.append(dict(nx=nx, ny=ny, dx=dx, dy=dy, bc=O.BC_WALL, lim=lim, d0=d0, slide=sl,
                        q=(h, z, z, z), amp=A))
    nx, ny, dx, dy = 40, 36, 0.05, 0.05
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    X, Y = np.meshgrid(x, y)
    d0 = 0.5 + 0.05 * np.sin(2 * np.pi * X / (nx * dx)) * np.cos(2 * np.pi * Y / (ny * dy))
    eta = 0.03 * np.exp(-((X - 1.0) ** 2 + (Y - 0.9) ** 2) / 0.05)
    h = d0 + eta
    out.insert(1, dict(nx=nx, ny=ny, dx=dx, dy=dy, bc=O.BC_PERIODIC, lim=O.LIM_MC, d0=d0, slide=None,
                       q=(h, 0.02 * h * np.sin(2 * np.pi * Y / (ny * dy)), -0.015 * h, 0.002 * eta), amp=0.03))
    return out


def _dt(ms):
    return min(W.cfl_dt_2d(0.4, m["dx"], m["dy"], math.sqrt(9.81 * m["q"][0].max()) + 0.05) for m in ms)


def _oracle(m, dt, n, crit, knh, enlarge, t0=0.0):
    p = O2.Params2D(nx=m["nx"], ny=m["ny"], dx=m["dx"], dy=m["dy"], bcx=m["bc"], bcy=m["bc"], limiter=m["lim"],
                    crit=crit, knh=knh, enlarge=enlarge, rtol=1e-13)
    if m["slide"]:
        p.slide = O.SLIDE_GAUSS_LNCOSH
        for k, v in m["slide"].items():
            setattr(p, k, v)
    s = O2.State2D(*m["q"])
    masks = []
    for k in range(n):
        st, info, mk = O2.step(p, m["d0"], t0 + k * dt, k, dt, s, want_mask=True)
        assert st == O.OK, (k, info)
        masks.append(mk)
    return s.fields(p), masks


def _ensemble(ms, crit, knh, enlarge, t0=0.0):
    bc = {O.BC_WALL: N.NH_BC_WALL, O.BC_PERIODIC: N.NH_BC_PERIODIC}
    G = N.Grid2D.ensemble([dict(nx=m["nx"], ny=m["ny"], dx=m["dx"], dy=m["dy"], d0=m["d0"], bc_x=bc[m["bc"]],
                                bc_y=bc[m["bc"]], limiter=_LIM[m["lim"]]) for m in ms])
    for i, m in enumerate(ms):
        G.set_bottom_motion(m["slide"], member=i)
        G.set_state(*m["q"], t=t0, member=i)
    G.set_criterion(crit, knh, enlarge)
    G.set_solver(1e-12, 20000, N.NH_GUESS_PREV)
    return G


def _compare(ref, got, amp, hmax, what):
    deta = np.max(np.abs(got[0] - ref[0]))
    assert deta <= 1e-9 * amp, (what, deta / amp)
    mom = 1e-9 * amp * math.sqrt(9.81 * hmax)
    for f, name in ((1, "hu"), (2, "hv"), (3, "hw")):
        assert np.max(np.abs(got[f] - ref[f])) <= mom, (what, name, np.max(np.abs(got[f] - ref[f])))


def test_ensemble_matches_oracle_and_graph_equals_steps():
    ms = _members()
    dt = _dt(ms)
    n = 20
    refs = [_oracle(m, dt, n, O.CRIT_ETA_D, 1e-4, 1) for m in ms]
    assert sum(int(mk.sum()) for _, masks in refs for mk in masks) > 0
    # step by step, masks every step
    G = _ensemble(ms, N.NH_CRIT_ETA_D, 1e-4, 1)
    assert G.members == len(ms)
    for k in range(n):
        G.step(dt)
        for i in range(len(ms)):
            assert np.array_equal(G.get_mask(i), refs[i][1][k]), (k, i)
    stepped = [G.get_state(i) for i in range(len(ms))]
    for i, m in enumerate(ms):
        _compare(refs[i][0], stepped[i], m["amp"], m["q"][0].max() + 0.1, f"member {i}")
    # captured-graph replays: the same numbers, bit for bit
    Gg = _ensemble(ms, N.NH_CRIT_ETA_D, 1e-4, 1)
    st, info = Gg.run(dt, n)
    assert info["steps"] == n and Gg.graph_runs == 1
    for i in range(len(ms)):
        got = Gg.get_state(i)
        for f in range(5):
            assert np.array_equal(got[f], stepped[i][f]), (i, f)
        assert np.array_equal(Gg.get_mask(i), refs[i][1][-1])
    # per-member figures: walls and periodic sides conserve each member's mass
    for i, m in enumerate(ms):
        mi = Gg.member_info(i)
        m0 = m["q"][0].sum() * m["dx"] * m["dy"]
        assert abs(mi["mass"] - m0) <= 1e-12 * m0, i
    assert abs(info["last"]["mass"] - sum(Gg.member_info(i)["mass"] for i in range(len(ms)))) <= 1e-12 * \
        info["last"]["mass"]


def test_ensemble_global_first_step_and_split_runs():
    """First step global by request (run on its own, then graph replays);
    a run split in two equals one run; a change of dt leaves the graphs."""
    ms = _members()
    dt = _dt(ms)
    A = _ensemble(ms, N.NH_CRIT_W_X, 1e-2, 1)
    A.set_criterion(N.NH_CRIT_W_X, 1e-2, 1, True)
    A.run(dt, 12)
    B = _ensemble(ms, N.NH_CRIT_W_X, 1e-2, 1)
    B.set_criterion(N.NH_CRIT_W_X, 1e-2, 1, True)
    B.run(dt, 5)
    B.run(dt, 7)
    for i in range(len(ms)):
        a, b = A.get_state(i), B.get_state(i)
        for f in range(5):
            assert np.array_equal(a[f], b[f]), (i, f)
    # against the oracle (first step global)
    for i, m in enumerate(ms):
        p = O2.Params2D(nx=m["nx"], ny=m["ny"], dx=m["dx"], dy=m["dy"], bcx=m["bc"], bcy=m["bc"],
                        limiter=m["lim"], crit=O.CRIT_W_X, knh=1e-2, enlarge=1, first_step_global=1, rtol=1e-13)
        if m["slide"]:
            p.slide = O.SLIDE_GAUSS_LNCOSH
            for k, v in m["slide"].items():
                setattr(p, k, v)
        s = O2.State2D(*m["q"])
        for k in range(12):
            st, info, mk = O2.step(p, m["d0"], k * dt, k, dt, s, want_mask=True)
            assert st == O.OK
            if k == 0:
                assert mk.sum() == m["nx"] * m["ny"]
        _compare(s.fields(p), A.get_state(i), m["amp"], m["q"][0].max() + 0.1, f"first-global member {i}")
    # a new dt leaves the captured graphs for the step-by-step path
    runs = B.graph_runs
    st, info = B.run(dt * 0.5, 3)
    assert info["steps"] == 3 and B.graph_runs == runs


def test_ensemble_bad_arguments():
    ms = _members()
    G = _ensemble(ms[:2], N.NH_CRIT_ETA_D, 1e-3, 1)
    with pytest.raises(N.NHError):
        G.set_state(*ms[0]["q"], member=2)
    with pytest.raises(N.NHError):
        G.get_mask(member=-1)
    # a member never given a state: no step
    H = N.Grid2D.ensemble([dict(nx=m["nx"], ny=m["ny"], dx=m["dx"], dy=m["dy"], d0=m["d0"]) for m in ms[:2]])
    H.set_state(*ms[0]["q"], member=0)
    st, _ = H.step(0.001, check=False)
    assert st == N.NH_ERR_STATE


def _landslide_at(w, t0):
    sl = w.slide
    s = sl["s0"] * math.log(math.cosh(t0 / sl["t0"]))
    x = (np.arange(w.nx) + 0.5) * w.dx
    y = (np.arange(w.ny) + 0.5) * w.dy
    X, Y = np.meshgrid(x, y)
    return w.d0 - sl["A"] * np.exp(-((X - sl["xc0"] - s) / sl["Lx"]) ** 2 - ((Y - sl["yc0"]) / sl["Ly"]) ** 2)


def test_landslide_ensemble_full_size():
    """32 uneven landslide runs (nx, ny drawn from 256 .. 1024, dx = 0.02 m,
    drawn slope, A, L, s0) for 3 captured steps from t = 0.3 s: every
    member's mass; the smallest and the largest member against the oracle,
    every cell and mask."""
    ws, dt = W.landslide_ensemble_2d()
    t0 = 0.3
    hs = [_landslide_at(w, t0) for w in ws]
    G = N.Grid2D.ensemble([dict(nx=w.nx, ny=w.ny, dx=w.dx, dy=w.dy, d0=w.d0) for w in ws])
    for i, w in enumerate(ws):
        G.set_bottom_motion(w.slide, member=i)
        z = np.zeros_like(hs[i])
        G.set_state(hs[i], z, z, z, t=t0, member=i)
    G.set_criterion(N.NH_CRIT_ETA_D, 1e-4, 1)
    G.set_solver(1e-12, 20000, N.NH_GUESS_PREV)
    st, info = G.run(dt, 3)
    assert info["steps"] == 3 and G.graph_runs == 1
    assert info["last"]["n_active"] > 0
    for i, w in enumerate(ws):
        m0 = hs[i].sum() * w.dx * w.dy
        assert abs(G.member_info(i)["mass"] - m0) <= 1e-12 * m0, i
    sizes = [w.nx * w.ny for w in ws]
    for i in (int(np.argmin(sizes)), int(np.argmax(sizes))):
        w = ws[i]
        p = O2.Params2D(nx=w.nx, ny=w.ny, dx=w.dx, dy=w.dy, crit=O.CRIT_ETA_D, knh=1e-4, enlarge=1, rtol=1e-13,
                        slide=O.SLIDE_GAUSS_LNCOSH, **w.slide)
        z = np.zeros_like(hs[i])
        s = O2.State2D(hs[i], z, z, z)
        for k in range(3):
            r, oi, mk = O2.step(p, w.d0, t0 + k * dt, k, dt, s, want_mask=True)
            assert r == O.OK
        assert np.array_equal(G.get_mask(i), mk), i
        _compare(s.fields(p), G.get_state(i), w.amplitude, w.d0.max(), f"landslide member {i} ({w.nx}x{w.ny})")
