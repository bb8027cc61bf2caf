"""Shared helpers: run the same seeded 1D workload through the CUDA library and
through the FP64 oracle, member by member."""
import numpy as np

import oracle as O
from paper_2505_17025_gb300 import nhswe as N


def oracle_params(m, crit, knh=1e-3, enlarge=1, first=0, solver=O.SOLVER_AUTO, rtol=1e-12,
                  max_iter=20000, guess=O.GUESS_PREV, bc=O.BC_WALL, limiter=O.LIM_CENTRAL):
    return O.Params(nx=m.nx, dx=m.dx, xl=m.xl, bc=bc, limiter=limiter, slide=m.slide, A=m.A, L=m.L,
                    xc0=m.xc0, s0=m.s0, t0=m.t0, t2=m.t2, crit=crit, knh=knh, enlarge=enlarge,
                    first_step_global=first, solver=solver, rtol=rtol, max_iter=max_iter, guess=guess)


def run_oracle(wl, n_steps, members=None, **kw):
    """Final states (h, hu, hw, q), per-step infos and last masks of the oracle."""
    out = []
    for b in (range(len(wl.members)) if members is None else members):
        m = wl.members[b]
        p = oracle_params(m, **kw)
        s = O.State(m.h, m.hu, m.hw)
        infos = []
        mask = None
        for k in range(n_steps):
            st, info, mask = O.step(p, m.d0, k * wl.dt, k, wl.dt, s, want_mask=True)
            assert st == O.OK, (b, k, info)
            infos.append(info)
        out.append((s, infos, mask))
    return out


_CRIT = {O.CRIT_GLOBAL: N.NH_CRIT_GLOBAL, O.CRIT_HYDROSTATIC: N.NH_CRIT_HYDROSTATIC,
         O.CRIT_ETA_D: N.NH_CRIT_ETA_D, O.CRIT_ETA_X: N.NH_CRIT_ETA_X, O.CRIT_U: N.NH_CRIT_U,
         O.CRIT_U_X: N.NH_CRIT_U_X, O.CRIT_W: N.NH_CRIT_W, O.CRIT_W_X: N.NH_CRIT_W_X}


def make_gpu(wl, crit, knh=1e-3, enlarge=1, first=0, solver=O.SOLVER_AUTO, rtol=1e-12,
             max_iter=20000, guess=O.GUESS_PREV, bc=O.BC_WALL, limiter=O.LIM_CENTRAL,
             precision=N.NH_FP64, members=None, precond=N.NH_PRECOND_LINE):
    import copy
    if members is not None:
        wl = copy.copy(wl)
        wl.members = [wl.members[b] for b in members]
    G = N.grid_from_workload(wl, precision=precision, limiter=limiter, bc=bc)
    G.set_criterion(_CRIT[crit], knh, enlarge, bool(first))
    G.set_solver({O.SOLVER_AUTO: N.NH_SOLVER_AUTO, O.SOLVER_CG: N.NH_SOLVER_CG,
                  O.SOLVER_BICGSTAB: N.NH_SOLVER_BICGSTAB}[solver], rtol, max_iter,
                 N.NH_GUESS_PREV if guess == O.GUESS_PREV else N.NH_GUESS_ZERO)
    G.set_preconditioner(precond)
    return G


def compare(wl, G, ref, tol_eta=1e-9, what=""):
    """max |d eta| <= tol_eta * a and max |d hu|, |d hw| <= tol_eta * a * sqrt(g h_max)
    (a = the workload's amplitude; a sqrt(g h) is the momentum scale of a wave
    of that amplitude).  Returns the worst |d eta| / a."""
    h, hu, hw, p = G.get_state()
    worst = 0.0
    for b, (s, infos, mask) in enumerate(ref):
        a = wl.amplitude
        m = wl.members[b]
        qscale = a * np.sqrt(9.81 * float(np.max(m.d0)))
        d_eta = float(np.max(np.abs(h[b] - s.h)))
        d_hu = float(np.max(np.abs(hu[b] - s.hu)))
        d_hw = float(np.max(np.abs(hw[b] - s.hw)))
        worst = max(worst, d_eta / a)
        assert d_eta <= tol_eta * a, (what, b, "eta", d_eta / a)
        assert d_hu <= tol_eta * qscale, (what, b, "hu", d_hu / qscale)
        assert d_hw <= tol_eta * qscale, (what, b, "hw", d_hw / qscale)
    return worst
