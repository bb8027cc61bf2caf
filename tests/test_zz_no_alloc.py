"""nh_predict_static -- the predictor for callers that cannot allocate device
memory (its scratch is a fixed array inside the library) -- must give what the
regular handle-based path gives for the same step.

The regular path is nh_step with the HYDROSTATIC criterion (no
non-hydrostatic cell, so a step is exactly the predictor).  Two calls in a
row are compared, the second starting from the first's output, within the
FP64 tolerance of the parity tests: |d eta| <= 1e-9 a and |d hu|, |d hw| <=
1e-9 a sqrt(g h_max).  This file is collected last on purpose.
"""
import ctypes as C
import math

import numpy as np
import pytest

from paper_2505_17025_gb300 import nhswe as N
from paper_2505_17025_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_predict_static_matches_nh_step_twice():
    import torch

    L = N.load()
    wl = W.slide_1d(n_members=1, nx=3001, length=6.0, xc0=1.0, T=0.5, seed0=4)
    m = wl.members[0]
    a = wl.amplitude
    qscale = a * math.sqrt(9.81 * float(np.max(m.d0)))
    dt = wl.dt
    t0 = 0.3

    # regular path: a handle with its own workspace, hydrostatic criterion
    G = N.grid_from_workload(wl)
    G.set_criterion(N.NH_CRIT_HYDROSTATIC, 1e-3, 1, False)
    G.set_state(m.h, m.hu, m.hw, t=t0)
    ref = []
    for _ in range(2):
        st, info = G.step(dt)
        h, hu, hw, _ = G.get_state()
        ref.append((h[0].copy(), hu[0].copy(), hw[0].copy(), info["mass"]))
    G.close()

    # no-allocation path on caller buffers
    dev = torch.device("cuda")
    cur = [torch.tensor(v, dtype=torch.float64, device=dev) for v in (m.h, m.hu, m.hw)]
    nxt = [torch.empty(m.nx, dtype=torch.float64, device=dev) for _ in range(3)]
    d0 = torch.tensor(m.d0, dtype=torch.float64, device=dev)
    slide = N.nh_slide_desc(N.NH_SLIDE_GAUSS_LNCOSH, m.A, m.L, m.xc0, m.s0, m.t0)
    stream = torch.cuda.current_stream()
    for k in range(2):
        mass = C.c_double(0.0)
        t = t0 + k * dt
        st = L.nh_predict_static(*(C.c_void_p(x.data_ptr()) for x in cur), C.c_void_p(d0.data_ptr()),
                                 *(C.c_void_p(x.data_ptr()) for x in nxt), m.nx, m.dx, m.xl,
                                 N.NH_BC_WALL, N.NH_LIM_CENTRAL, 9.81, C.byref(slide), t, dt,
                                 C.byref(mass), C.c_void_p(stream.cuda_stream))
        assert st == N.NH_OK, L.nh_status_string(st)
        torch.cuda.synchronize()
        h, hu, hw = (x.cpu().numpy() for x in nxt)
        rh, rhu, rhw, rmass = ref[k]
        assert np.max(np.abs(h - rh)) <= 1e-9 * a
        assert np.max(np.abs(hu - rhu)) <= 1e-9 * qscale
        assert np.max(np.abs(hw - rhw)) <= 1e-9 * qscale
        assert abs(mass.value - rmass) <= 1e-12 * rmass
        cur, nxt = nxt, cur


def test_predict_static_rejects_oversize():
    import torch

    L = N.load()
    n = N.NH_STATIC_MAX_CELLS + 1
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = C.c_void_p(x.data_ptr())
    q = C.c_void_p(x.data_ptr() + 8)
    st = L.nh_predict_static(p, p, p, p, q, q, q, n, 0.1, 0.0, N.NH_BC_WALL, N.NH_LIM_CENTRAL, 9.81,
                             None, 0.0, 0.01, None, None)
    assert st == N.NH_ERR_ARG
