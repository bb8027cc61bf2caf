"""The CUDA DG-P1 / LDG path (nhswe_dg.h) against the DG oracle, element by
element, on the same seeded inputs.

Both sides compute in FP64 and solve the same LDG system, the oracle by
banded elimination with partial pivoting, the library by substituting hu and
block cyclic reduction.  The bars:
 - first step (identical inputs): the library's (p, hu) put into the oracle's
   own assembled LDG system has a normwise backward error
   ||r - A x|| / || |r| + |A| |x| || <= 1e-13;
 - every compared step: h, hu, hw, p within tol of each field's scale,
   tol = max(1e-8, 10 f), f the FP64 forward-error floor of the first step's
   system measured on the oracle itself: the relative change of its (p, hu)
   under one more step of iterative refinement.  The unscaled penalty
   c11 = 1/2 dominates the p-rows over the physical terms (~ dt h / (rho dx))
   on fine grids with small steps, and no FP64 solver determines the
   solution better than that floor (1e-7 at 200 000 elements);
 - p itself only on the first step: p answers the predicted state's
   violation of the constraint (Eq. 13) with a factor rho / dt (the rows
   carry rho hu~ / dt), so a rounding-level difference of the input state
   moves p by rho / dt times as much, while the corrected state it produces
   stays as close as its input; later steps compare p through h, hu, hw;
 - masks equal; an adaptive mask may differ only where the oracle's own
   criterion value lies within 1e-9 of k_nh (a near-tie that rounding
   decides), and runs are compared up to such a step.
"""
import math

import numpy as np
import pytest

import oracle as O
import oracle.oracle_dg as D
from paper_2505_17025_gb300 import nhswe as N
from paper_2505_17025_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-8


def _gpu(ps, slides=None, crit=O.CRIT_GLOBAL, knh=1e-3, enlarge=1, first_global=False, c11=0.5):
    """One handle for members sharing ne, dx, x0 (ParamsDG list), nodal
    depths b0 + b1 (x - xl)."""
    p0 = ps[0]
    x = p0.nodes()
    d0 = np.stack([p.b0 + p.b1 * (x - p.xl) for p in ps])
    G = N.GridDG(p0.ne, p0.dx, d0, nbatch=len(ps), x0=p0.xl, g=p0.g, rho=p0.rho, c11=c11)
    if slides is not None:
        G.set_bottom_motion(slides)
    G.set_criterion(crit, knh, enlarge, first_global)
    return G


def _slide_of(p):
    return {"shape": p.slide, "A": p.A, "L": p.L, "xc0": p.xc0, "s0": p.s0, "t0": p.t0, "t2": p.t2}


def _scale(a):
    return max(float(np.max(np.abs(a))), 1e-300)


def _near_tie(p, t1, ht, hut, hwt, diff, rel=1e-9):
    """Every element where the masks differ has, within the enlargement, an
    element whose oracle criterion value is within rel of k_nh."""
    q = D.ParamsDG(**{**p.__dict__, "enlarge": 0, "first_step_global": 0})
    lo = D.ParamsDG(**{**q.__dict__, "knh": q.knh * (1 - rel)})
    hi = D.ParamsDG(**{**q.__dict__, "knh": q.knh * (1 + rel)})
    m_lo, m_hi = D.mask(lo, t1, 1, ht, hut, hwt), D.mask(hi, t1, 1, ht, hut, hwt)
    amb = np.flatnonzero(m_lo != m_hi)
    for i in np.flatnonzero(diff):
        if not np.any(np.abs(amb - i) <= p.enlarge):
            return False
    return True


def _backward_error(p, t, dt, h, hu, hw, mask, gp, ghu):
    """Normwise backward error of the library's (p, hu) in the oracle's LDG
    system assembled from the oracle's predicted state (elements not marked:
    identity rows, satisfied exactly by p = 0, hu = hu~)."""
    ht, hut, hwt = D.predict(p, t, dt, h, hu, hw)
    blk, r = D.assemble(p, t + dt, dt, ht, hut, hwt, mask)
    x = np.stack([gp[0::2], gp[1::2], ghu[0::2], ghu[1::2]], axis=1)
    res = r - _matvec(blk, x)
    den = np.abs(r) + _matvec(np.abs(blk), np.abs(x))
    return float(np.linalg.norm(res) / max(np.linalg.norm(den), 1e-300))


def _matvec(blk, x):
    y = np.zeros_like(x)
    for q in range(3):
        xs = np.roll(x, 1 - q, axis=0)        # x of element i + q - 1
        if q == 0:
            xs[0] = 0.0
        if q == 2:
            xs[-1] = 0.0
        y += np.einsum("nab,nb->na", blk[:, q], xs)
    return y


def _floor(p, t, dt, h, hu, hw, mask):
    """Relative change of the oracle's (p, hu) under one more refinement step
    of its own solve: what FP64 determines about this system's solution."""
    ht, hut, hwt = D.predict(p, t, dt, h, hu, hw)
    blk, r = D.assemble(p, t + dt, dt, ht, hut, hwt, mask)
    x, st, _ = D.solve(p, blk, r)
    d, st2, _ = D.solve(p, blk, r - _matvec(blk, x))
    assert st == O.OK and st2 == O.OK
    return max(float(np.max(np.abs(d[:, c])) / max(np.max(np.abs(x[:, c])), 1e-300)) for c in (slice(0, 2), slice(2, 4)))


def _compare_run(ps, states, G, dt, nsteps, t0=0.0, what=""):
    """Step the oracle members and the handle side by side; compare h, hu,
    hw, p and the mask after every step.  Returns the worst relative
    difference and the number of steps compared."""
    worst = 0.0
    tol = None
    for k in range(nsteps):
        t = t0 + k * dt
        pre = [(s.h.copy(), s.hu.copy(), s.hw.copy()) for s in states]
        masks = []
        for p, s in zip(ps, states):
            st, info, m = D.step(p, t, k, dt, s, want_mask=True)
            assert st == O.OK, (what, k, info)
            masks.append(m)
        st, info = G.step(dt)
        assert st == N.NH_OK, (what, k, info)
        gm, rel = G.get_mask()
        h, hu, hw, pp = G.get_state()
        if tol is None:
            tol = RTOL
            for b, p in enumerate(ps):
                if masks[b].any():
                    tol = max(tol, 10.0 * _floor(p, t, dt, *pre[b], masks[b]))
        for b, (p, s) in enumerate(zip(ps, states)):
            if k == 0 and masks[b].any():
                be = _backward_error(p, t, dt, *pre[b], masks[b], pp[b], hu[b])
                assert be <= 1e-13, (what, b, be)
            if not np.array_equal(gm[b], masks[b]):
                ht, hut, hwt = D.predict(p, t, dt, *pre[b])
                assert _near_tie(p, t + dt, ht, hut, hwt, gm[b] != masks[b]), (what, k, b)
                return worst, k
            fields = [("h", h[b], s.h), ("hu", hu[b], s.hu), ("hw", hw[b], s.hw)]
            if k == 0:
                fields.append(("p", pp[b], s.p))
            for name, gv, ov in fields:
                # field scales: the surface's excursion (at least 1e-6 h), |hu|, |hw| (at least
                # 1e-14 m^2/s), |p| (at least 1e-9 Pa)
                if name == "h":
                    sc = max(_scale(s.h - np.mean(s.h)), 1e-6 * _scale(s.h))
                else:
                    sc = max(_scale(ov), 1e-9 if name == "p" else 1e-14)
                e = float(np.max(np.abs(gv - ov))) / sc
                assert e <= tol, (what, k, b, name, e, tol)
                worst = max(worst, e)
        assert info["rel_res"] <= 1e-13 or info["n_active"] == 0, (what, k, info)   # backward error
    print(f"{what}: tolerance {tol:.1e}")
    return worst, nsteps


def _solitary_params(crit=O.CRIT_GLOBAL, enlarge=0, ne=200):
    return D.ParamsDG(ne=ne, dx=800.0 / ne, b0=10.0, crit=crit, knh=1e-3, enlarge=enlarge)


def _solitary_state(p):
    x = p.nodes()
    eta, u, hw = W.solitary_fields(x, 0.0, 2.0, 10.0, 200.0)
    return D.StateDG(10.0 + eta, (10.0 + eta) * u, hw)


@pytest.mark.parametrize("crit,enlarge", [(O.CRIT_GLOBAL, 0), (O.CRIT_ETA_D, 0), (O.CRIT_ETA_D, 1),
                                          (O.CRIT_HYDROSTATIC, 0), (O.CRIT_U_X, 1), (O.CRIT_W, 1)])
def test_solitary_wave_per_step(crit, enlarge):
    """The paper's solitary case (200 elements of 4 m, dt = 0.1 s), 40 steps
    compared step by step."""
    p = _solitary_params(crit, enlarge)
    s = _solitary_state(p)
    G = _gpu([p], crit=crit, enlarge=enlarge)
    G.set_state(s.h, s.hu, s.hw, 0.0)
    worst, n = _compare_run([p], [s], G, 0.1, 40, what=f"solitary crit={crit}")
    assert n >= 20
    print(f"solitary crit={crit} enlarge={enlarge}: {n} steps, worst {worst:.2e}")
    G.close()


def test_solitary_wave_paper_values_through_the_library():
    """The whole 30 s run replayed from captured graphs: RMSE and r against
    the closed form equal the oracle's (and so the paper's printed values,
    pinned in the oracle's own tests) to 1e-9."""
    p = _solitary_params(O.CRIT_ETA_D, 1)
    s = _solitary_state(p)
    G = _gpu([p], crit=O.CRIT_ETA_D, enlarge=1)
    G.set_state(s.h, s.hu, s.hw, 0.0)
    st, info = G.run(0.1, 300)
    assert st == N.NH_OK and info["steps"] == 300
    for k in range(300):
        assert D.step(p, k * 0.1, k, 0.1, s)[0] == O.OK
    x = p.nodes()
    eta_ex, _, _ = W.solitary_fields(x, 30.0, 2.0, 10.0, 200.0)
    h = G.get_state()[0][0]
    r_g = [float(np.sqrt(np.mean((h - 10.0 - eta_ex) ** 2))), float(np.corrcoef(h - 10.0, eta_ex)[0, 1])]
    r_o = [float(np.sqrt(np.mean((s.h - 10.0 - eta_ex) ** 2))), float(np.corrcoef(s.h - 10.0, eta_ex)[0, 1])]
    assert abs(r_g[0] - r_o[0]) <= 1e-9 * r_o[0] and abs(r_g[1] - r_o[1]) <= 1e-9
    assert r_g[0] < 0.02 and r_g[1] > 0.999
    print(f"solitary 30 s: RMSE {r_g[0]:.5f} m, r {r_g[1]:.6f} (oracle {r_o[0]:.5f}, {r_o[1]:.6f})")
    G.close()


def _slide_members(ne, dx, seed):
    """Members with each moving bottom: a Gaussian mound on a slope, the
    paper's plate (Sec. 4.2) and its sliding block (Sec. 4.3)."""
    rng = np.random.default_rng(seed)
    L = ne * dx
    ps = [
        D.ParamsDG(ne=ne, dx=dx, b0=0.1 + 0.05 * rng.random(), b1=0.3 / L, slide=O.SLIDE_GAUSS_LNCOSH,
                   A=0.03 + 0.02 * rng.random(), L=0.1 * L, xc0=0.25 * L, s0=0.3 * L, t0=1.0),
        D.ParamsDG(ne=ne, dx=dx, b0=0.2, slide=O.SLIDE_PLATE_EXP, A=0.01 * (1 + rng.random()), L=0.1 * L,
                   xc0=0.2 * L, t0=0.2),
        D.ParamsDG(ne=ne, dx=dx, b0=0.175, slide=O.SLIDE_QUARTIC, A=0.026, L=0.12 * L, xc0=0.3 * L, s0=0.5,
                   t0=0.3, t2=0.9),
    ]
    return ps


@pytest.mark.parametrize("ne,crit,enlarge", [(300, O.CRIT_GLOBAL, 0), (300, O.CRIT_ETA_D, 1),
                                             (3001, O.CRIT_GLOBAL, 0), (3001, O.CRIT_ETA_D, 2),
                                             (513, O.CRIT_U, 0)])
def test_moving_bottoms_batch(ne, crit, enlarge):
    """Three members with different moving bottoms in one handle (several
    cyclic-reduction levels above the shared-memory one at 3001 elements, one
    at 513), 12 steps from a lake at rest over the bottom at t = 0.5 s, when
    every bottom is moving."""
    dx = 4.0 / ne
    ps = _slide_members(ne, dx, ne)
    for p in ps:
        p.crit, p.knh, p.enlarge = crit, 1e-5, enlarge
    x = ps[0].nodes()
    states = []
    for p in ps:
        b = np.array([D.bottom(p, xx, 0.5)[0] for xx in x])
        states.append(D.StateDG(b, np.zeros_like(b), np.zeros_like(b)))
    G = _gpu(ps, slides=[_slide_of(p) for p in ps], crit=crit, knh=1e-5, enlarge=enlarge)
    G.set_state(np.stack([s.h for s in states]), np.zeros((3, 2 * ne)), np.zeros((3, 2 * ne)), 0.5)
    dt = 0.15 * dx / math.sqrt(9.81 * 0.3)
    worst, n = _compare_run(ps, states, G, dt, 12, t0=0.5, what=f"slides ne={ne} crit={crit}")
    assert n >= 6
    print(f"moving bottoms ne={ne} crit={crit}: {n} steps, worst {worst:.2e}")
    G.close()


def test_large_member_at_full_size_sampled():
    """A 200 000-element member (nine global reduction levels) with a
    perturbed state and a moving mound: one step, compared on every element
    against the oracle (which handles this size in seconds)."""
    ne, dx = 200000, 2e-4
    p = D.ParamsDG(ne=ne, dx=dx, b0=0.2, b1=0.5 / (ne * dx), slide=O.SLIDE_GAUSS_LNCOSH, A=0.05, L=1.0,
                   xc0=10.0, s0=5.0, t0=1.0, crit=O.CRIT_ETA_D, knh=1e-4, enlarge=1)
    x = p.nodes()
    rng = np.random.default_rng(7)
    b = p.b0 + p.b1 * x
    eta = 0.01 * np.exp(-((x - 20.0) / 2.0) ** 2)
    s = D.StateDG(b + eta, 0.02 * np.exp(-((x - 20.0) / 2.0) ** 2), 1e-4 * rng.standard_normal(2 * ne))
    G = _gpu([p], slides=[_slide_of(p)], crit=O.CRIT_ETA_D, knh=1e-4, enlarge=1)
    G.set_state(s.h, s.hu, s.hw, 0.5)
    worst, n = _compare_run([p], [s], G, 0.2 * dx / math.sqrt(9.81 * 0.7), 2, t0=0.5, what="large member")
    assert n == 2
    print(f"200k elements: worst {worst:.2e}")
    G.close()


def test_edge_cases_tiny_and_isolated():
    """ne = 2 (the minimum); an adaptive mask of isolated single elements
    (enlarge 0) so that every marked element is its own sub-domain; a
    member with nothing marked beside one with everything marked."""
    # ne = 2, global
    p = D.ParamsDG(ne=2, dx=0.5, b0=1.0, crit=O.CRIT_GLOBAL)
    x = p.nodes()
    s = D.StateDG(1.0 + 0.01 * np.cos(x), 0.01 * np.sin(x), np.zeros(4))
    G = _gpu([p])
    G.set_state(s.h, s.hu, s.hw)
    _compare_run([p], [s], G, 0.01, 5, what="ne=2")
    G.close()
    # isolated marks: |u| above k_nh on alternate elements
    ne = 64
    p = D.ParamsDG(ne=ne, dx=0.1, b0=1.0, crit=O.CRIT_U, knh=0.05, enlarge=0)
    x = p.nodes()
    u = np.where((np.arange(2 * ne) // 2) % 3 == 0, 0.1, 0.0)
    s = D.StateDG(np.ones(2 * ne), u, np.zeros(2 * ne))
    G = _gpu([p], crit=O.CRIT_U, knh=0.05, enlarge=0)
    G.set_state(s.h, s.hu, s.hw)
    worst, n = _compare_run([p], [s], G, 0.002, 1, what="isolated")
    assert n == 1
    m, _ = G.get_mask()
    assert 0 < m.sum() < ne
    G.close()
    # member 0 hydrostatic-quiet (nothing marked), member 1 with a wave
    ps = [D.ParamsDG(ne=100, dx=0.1, b0=1.0, crit=O.CRIT_ETA_D, knh=1e-3, enlarge=1) for _ in range(2)]
    x = ps[0].nodes()
    states = [D.StateDG(np.ones(200), np.zeros(200), np.zeros(200)),
              D.StateDG(1.0 + 0.05 * np.exp(-((x - 5.0) / 0.5) ** 2), np.zeros(200), np.zeros(200))]
    G = _gpu(ps, crit=O.CRIT_ETA_D, knh=1e-3, enlarge=1)
    G.set_state(np.stack([s.h for s in states]), np.zeros((2, 200)), np.zeros((2, 200)))
    _compare_run(ps, states, G, 0.005, 5, what="quiet + wave")
    m, _ = G.get_mask()
    assert m[0].sum() == 0 and m[1].sum() > 0
    G.close()


def test_graph_run_equals_step_by_step():
    """nh_dg_run (captured graphs, device-side time) gives the same bits as
    nh_dg_step; first-step-global marks every element in step 0 only."""
    p = _solitary_params(O.CRIT_W, 1)
    p.first_step_global = 1
    s = _solitary_state(p)
    A = _gpu([p], crit=O.CRIT_W, enlarge=1, first_global=True)
    B = _gpu([p], crit=O.CRIT_W, enlarge=1, first_global=True)
    A.set_state(s.h, s.hu, s.hw)
    B.set_state(s.h, s.hu, s.hw)
    st, info = A.run(0.1, 25)
    assert st == N.NH_OK and info["steps"] == 25
    for _ in range(25):
        assert B.step(0.1)[0] == N.NH_OK
    for a, b in zip(A.get_state(), B.get_state()):
        assert np.array_equal(a, b)
    C = _gpu([p], crit=O.CRIT_W, enlarge=1, first_global=True)
    C.set_state(s.h, s.hu, s.hw)
    st, info = C.step(0.1)
    assert info["n_active"] == p.ne
    st, info = C.step(0.1)
    assert info["n_active"] < p.ne
    for G in (A, B, C):
        G.close()


def test_nonfinite_step_is_rejected():
    """A step whose solution is not finite (dt far beyond stability) returns
    NH_ERR_NONFINITE and leaves the state as it was."""
    p = _solitary_params()
    s = _solitary_state(p)
    G = _gpu([p])
    G.set_state(s.h, s.hu, s.hw)
    before = G.get_state()
    st, info = G.step(1e4)
    assert st == N.NH_ERR_NONFINITE
    for a, b in zip(before, G.get_state()):
        assert np.array_equal(a, b)
    assert G.step(0.1)[0] == N.NH_OK
    G.close()


def test_profile_counts_launches():
    p = _solitary_params()
    s = _solitary_state(p)
    G = _gpu([p])
    G.set_state(s.h, s.hu, s.hw)
    G.set_profiling(True)
    G.step(0.1)
    prof = G.get_profile()
    assert prof["predict"][1] == 1 and prof["reduce"][1] == 1 and prof["back"][1] == 0
    assert all(v[0] >= 0.0 for v in prof.values())
    G.close()
