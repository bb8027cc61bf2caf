"""nh_predict_static -- the predictor for callers that cannot allocate device
memory (its scratch is a fixed array inside the library) -- must give what the
regular handle-based path gives for the same step, and what the FP64 oracle's
predictor gives.

The regular path is nh_step with the HYDROSTATIC criterion (no
non-hydrostatic cell, so a step is exactly the predictor).  Two calls in a
row are compared, the second starting from the first's output, within the
FP64 tolerance of the parity tests: |d eta| <= 1e-9 a and |d hu|, |d hw| <=
1e-9 a sqrt(g h_max), over the smallest grid, a ragged one and the largest
the scratch array holds, walled and periodic, with and without a slide.  The
first call is also checked against the oracle's Heun predictor (Sec. 3.1).
This file is collected last on purpose.
"""
import ctypes as C
import math

import numpy as np
import pytest

import oracle as O
from paper_2505_17025_gb300 import nhswe as N

pytestmark = pytest.mark.gpu


def _member(nx, with_slide):
    """A seeded slope with a wave on it; the slide (if any) sits inside."""
    length = 4.0 if nx <= 4096 else 40.0
    dx = length / nx
    x = (np.arange(nx) + 0.5) * dx
    d0 = np.minimum(0.05 + 0.25 * x, 1.0)
    rng = np.random.default_rng(nx)
    a = 0.01
    eta = a * np.exp(-((x - 0.6 * length) / (0.1 * length)) ** 2) + 1e-4 * a * rng.standard_normal(nx)
    h = d0 + eta
    hu = 0.3 * eta * np.sqrt(9.81 * d0)
    hw = 1e-3 * eta
    slide = None
    if with_slide:
        slide = dict(A=0.02, L=0.15 * length, xc0=0.3 * length, s0=0.5, t0=1.0)
    return dict(nx=nx, dx=dx, d0=d0, h=h, hu=hu, hw=hw, slide=slide, a=a)


@pytest.mark.parametrize("nx", [8, 33, 3001, N.NH_STATIC_MAX_CELLS])
@pytest.mark.parametrize("bc", [N.NH_BC_WALL, N.NH_BC_PERIODIC])
@pytest.mark.parametrize("with_slide", [False, True])
def test_predict_static_matches_nh_step_and_oracle(nx, bc, with_slide):
    import torch

    L = N.load()
    m = _member(nx, with_slide)
    a = m["a"]
    qscale = a * math.sqrt(9.81 * float(np.max(m["d0"])))
    dt = 0.2 * m["dx"] / math.sqrt(9.81)
    t0 = 0.3

    # regular path: a handle with its own workspace, hydrostatic criterion
    G = N.Grid(nx, m["dx"], m["d0"], bc=bc)
    if with_slide:
        G.set_bottom_motion([dict(m["slide"], shape=N.NH_SLIDE_GAUSS_LNCOSH)])
    G.set_criterion(N.NH_CRIT_HYDROSTATIC, 1e-3, 1, False)
    G.set_state(m["h"], m["hu"], m["hw"], t=t0)
    ref = []
    for _ in range(2):
        st, info = G.step(dt)
        h, hu, hw, _ = G.get_state()
        ref.append((h[0].copy(), hu[0].copy(), hw[0].copy(), info["mass"]))
    G.close()

    # the oracle's predictor for the first step
    sl = m["slide"] or {}
    p = O.Params(nx=nx, dx=m["dx"], bc=O.BC_PERIODIC if bc == N.NH_BC_PERIODIC else O.BC_WALL,
                 slide=O.SLIDE_GAUSS_LNCOSH if with_slide else O.SLIDE_NONE,
                 A=sl.get("A", 0.0), L=sl.get("L", 1.0), xc0=sl.get("xc0", 0.0), s0=sl.get("s0", 0.0),
                 t0=sl.get("t0", 1.0))
    oh, ohu, ohw = O.predict(p, m["d0"], t0, dt, m["h"], m["hu"], m["hw"])

    # no-allocation path on caller buffers
    dev = torch.device("cuda")
    cur = [torch.tensor(v, dtype=torch.float64, device=dev) for v in (m["h"], m["hu"], m["hw"])]
    nxt = [torch.empty(nx, dtype=torch.float64, device=dev) for _ in range(3)]
    d0 = torch.tensor(m["d0"], dtype=torch.float64, device=dev)
    slide = (C.byref(N.nh_slide_desc(N.NH_SLIDE_GAUSS_LNCOSH, sl["A"], sl["L"], sl["xc0"], sl["s0"], sl["t0"]))
             if with_slide else None)
    stream = torch.cuda.current_stream()
    for k in range(2):
        mass = C.c_double(0.0)
        t = t0 + k * dt
        st = L.nh_predict_static(*(C.c_void_p(x.data_ptr()) for x in cur), C.c_void_p(d0.data_ptr()),
                                 *(C.c_void_p(x.data_ptr()) for x in nxt), nx, m["dx"], 0.0,
                                 bc, N.NH_LIM_CENTRAL, 9.81, slide, t, dt,
                                 C.byref(mass), C.c_void_p(stream.cuda_stream))
        assert st == N.NH_OK, L.nh_status_string(st)
        torch.cuda.synchronize()
        h, hu, hw = (x.cpu().numpy() for x in nxt)
        rh, rhu, rhw, rmass = ref[k]
        assert np.max(np.abs(h - rh)) <= 1e-9 * a
        assert np.max(np.abs(hu - rhu)) <= 1e-9 * qscale
        assert np.max(np.abs(hw - rhw)) <= 1e-9 * qscale
        assert abs(mass.value - rmass) <= 1e-12 * rmass
        if k == 0:
            assert np.max(np.abs(h - oh)) <= 1e-9 * a
            assert np.max(np.abs(hu - ohu)) <= 1e-9 * qscale
            assert np.max(np.abs(hw - ohw)) <= 1e-9 * qscale
        cur, nxt = nxt, cur


def test_predict_static_rejects_bad_arguments():
    import torch

    L = N.load()
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = C.c_void_p(x.data_ptr())
    q = C.c_void_p(x.data_ptr() + 64)
    n = N.NH_STATIC_MAX_CELLS + 1
    st = L.nh_predict_static(p, p, p, p, q, q, q, n, 0.1, 0.0, N.NH_BC_WALL, N.NH_LIM_CENTRAL, 9.81,
                             None, 0.0, 0.01, None, None)
    assert st == N.NH_ERR_ARG
    bad = N.nh_slide_desc(N.NH_SLIDE_GAUSS_LNCOSH, float("nan"), 0.5, 1.0, 1.0, 1.0)
    st = L.nh_predict_static(p, p, p, p, q, q, q, 8, 0.1, 0.0, N.NH_BC_WALL, N.NH_LIM_CENTRAL, 9.81,
                             C.byref(bad), 0.0, 0.01, None, None)
    assert st == N.NH_ERR_ARG
