"""Mixed precision (FP32 state, predictor, Krylov vectors and preconditioner;
FP64 coefficients, inner products, norms, refinement residual and pressure)
against the FP64 oracle.

Tolerance: max |d eta| <= 1e-4 a and max |d hu|, |d hw| <= 1e-4 a sqrt(g h_max)
(a = wave or slide amplitude), for every run whose non-hydrostatic cells are
the same on both sides: global and hydrostatic runs, and adaptive runs up to
the first step where a criterion value lies within FP32 rounding of k_nh and
the two sides mark a different cell.  Such a decision must be a near-tie of
the oracle's own criterion value; after it the two runs solve on different
sub-domains and are not compared.
"""
import numpy as np
import pytest

import oracle as O
from paper_2505_17025_gb300 import nhswe as N
from paper_2505_17025_gb300 import workloads as W

from _helpers import compare, make_gpu, oracle_params, run_oracle

pytestmark = pytest.mark.gpu

MIXED_RTOL = 1e-10   # attainable FP64 true-residual level for kappa ~ 1e6


def _slide():
    return W.slide_1d(n_members=3, nx=2000, length=4.0, xc0=1.0, T=0.5, seed0=11)


@pytest.mark.parametrize("crit", [O.CRIT_GLOBAL, O.CRIT_HYDROSTATIC])
def test_mixed_fixed_mask_slide(crit):
    wl = _slide()
    n = 300
    ref = run_oracle(wl, n, crit=crit)
    G = make_gpu(wl, crit, precision=N.NH_MIXED, rtol=MIXED_RTOL)
    st, info = G.run(wl.dt, n)
    if crit == O.CRIT_GLOBAL:
        assert info["last"]["ir_passes"] >= 1
        assert info["last"]["rel_res"] <= MIXED_RTOL
    worst = compare(wl, G, ref, tol_eta=1e-4, what=f"mixed crit={crit}")
    print(f"mixed crit={crit}: max |d eta| / a = {worst:.2e}")
    G.close()


def test_mixed_global_solitary():
    wl = W.solitary_1d()
    n = 400
    ref = run_oracle(wl, n, crit=O.CRIT_GLOBAL)
    G = make_gpu(wl, O.CRIT_GLOBAL, precision=N.NH_MIXED, rtol=MIXED_RTOL)
    G.run(wl.dt, n)
    worst = compare(wl, G, ref, tol_eta=1e-4, what="mixed solitary")
    print(f"mixed global solitary: max |d eta| / a = {worst:.2e}")
    G.close()


def _near_tie(p, d0, t, dt, s, cells, rel=1e-3):
    """Every differing mask cell has, within its enlargement, an oracle
    criterion value within rel of k_nh (state s before the step)."""
    ht, hut, hwt = O.predict(p, d0, t, dt, s.h, s.hu, s.hw)
    c = O.criterion(p, d0, t + dt, ht, hut, hwt)
    e = p.enlarge
    return all(np.any(np.abs(c[max(0, i - e):i + e + 1] - p.knh) <= rel * p.knh) for i in cells)


@pytest.mark.parametrize("wl_name", ["slide", "solitary"])
def test_mixed_adaptive_until_decision_flip(wl_name):
    """Step by step: while both sides mark the same cells the mixed state is
    within 1e-4 a; the first differing decision of a member is a near-tie,
    and that member is not compared afterwards."""
    wl = _slide() if wl_name == "slide" else W.solitary_1d()
    n = 300
    members = range(len(wl.members))
    params = [oracle_params(m, crit=O.CRIT_ETA_D) for m in wl.members]
    states = [O.State(m.h, m.hu, m.hw) for m in wl.members]
    G = make_gpu(wl, O.CRIT_ETA_D, precision=N.NH_MIXED, rtol=MIXED_RTOL)
    a = wl.amplitude
    agree = [True] * len(wl.members)
    first_flip = [None] * len(wl.members)
    worst_agree = 0.0
    for k in range(n):
        masks = []
        befores = []
        for b in members:
            befores.append(states[b].copy())
            st, info, mk = O.step(params[b], wl.members[b].d0, k * wl.dt, k, wl.dt, states[b],
                                  want_mask=True)
            masks.append(mk)
        G.step(wl.dt)
        gm, _, _ = G.get_mask()
        h, hu, hw, _ = G.get_state()
        for b in members:
            if not agree[b]:
                continue
            if not np.array_equal(gm[b], masks[b]):
                agree[b] = False
                first_flip[b] = k + 1
                diff = np.flatnonzero(gm[b] != masks[b])
                assert _near_tie(params[b], wl.members[b].d0, k * wl.dt, wl.dt, befores[b], diff), (b, k, diff)
                continue
            e = float(np.max(np.abs(h[b] - states[b].h))) / a
            worst_agree = max(worst_agree, e)
            assert e <= 1e-4, (b, k, e)
    print(f"mixed adaptive {wl_name}: worst |d eta|/a with equal masks {worst_agree:.2e}; "
          f"first decision flip at steps {first_flip}")
    G.close()


def test_mixed_matches_fp64_path_globally():
    """Mixed and FP64 library paths on the same global run stay within the
    mixed tolerance of each other; the mixed path's mass (FP64 sum of the
    FP32 state) is conserved to 1e-9."""
    wl = W.slide_1d(n_members=2, nx=3000, length=6.0, xc0=1.0, T=0.5, seed0=2)
    n = 200
    G64 = make_gpu(wl, O.CRIT_GLOBAL)
    G32 = make_gpu(wl, O.CRIT_GLOBAL, precision=N.NH_MIXED, rtol=MIXED_RTOL)
    G64.run(wl.dt, n)
    st0, i0 = G32.step(wl.dt)
    _, i32 = G32.run(wl.dt, n - 1)
    h64, _, _, _ = G64.get_state()
    h32, _, _, _ = G32.get_state()
    assert np.max(np.abs(h64 - h32)) <= 1e-4 * wl.amplitude
    assert abs(i32["last"]["mass"] - i0["mass"]) <= 1e-9 * i0["mass"]
    G64.close()
    G32.close()


# ------------------------------------------- FP32 state with an FP64 solve

@pytest.mark.parametrize("crit", [O.CRIT_GLOBAL, O.CRIT_HYDROSTATIC])
def test_fp32_state_fp64_solve_fixed_mask(crit):
    """NH_MIXED_FP64_SOLVE: FP32 state and predictor, FP64 operator and Krylov
    (rtol 1e-12, no refinement passes); same tolerance as the mixed path."""
    wl = _slide()
    n = 300
    ref = run_oracle(wl, n, crit=crit)
    G = make_gpu(wl, crit, precision=N.NH_MIXED_FP64_SOLVE, rtol=1e-12)
    st, info = G.run(wl.dt, n)
    if crit == O.CRIT_GLOBAL:
        assert info["last"]["ir_passes"] == 0
        assert info["last"]["rel_res"] <= 1e-12
    worst = compare(wl, G, ref, tol_eta=1e-4, what=f"fp32 state crit={crit}")
    print(f"fp32 state / fp64 solve crit={crit}: max |d eta| / a = {worst:.2e}")
    G.close()


def test_fp32_state_fp64_solve_graph_equals_steps():
    """The captured-graph run of NH_MIXED_FP64_SOLVE equals its step-by-step run."""
    wl = _slide()
    out = []
    for graphs in (False, True):
        G = make_gpu(wl, O.CRIT_ETA_D, knh=1e-5, precision=N.NH_MIXED_FP64_SOLVE, rtol=1e-12)
        G.set_run_mode(graphs)
        st, info = G.run(wl.dt, 40)
        out.append((G.get_state(), info["iters_total"]))
        G.close()
    (s0, i0), (s1, i1) = out
    assert i0 > 0 and i0 == i1
    for k in range(3):
        a, b = np.asarray(s0[k]), np.asarray(s1[k])
        assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.max(np.abs(a)))
