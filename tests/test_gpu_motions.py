"""The paper's own moving bottoms on the GPU against the FP64 oracle: the
impulsively moved plate of Sec. 4.2 (upward and downward, the paper's dx and
dt) and the sliding block of Sec. 4.3 (the table's Fr = 0.25 row), adaptive
|eta/d| criterion; masks every step bit for bit, state within 1e-9 a."""
import numpy as np
import pytest

import oracle as O
from paper_2505_17025_gb300 import workloads as W

from _helpers import compare, make_gpu, run_oracle

pytestmark = pytest.mark.gpu


def _run(wl, n, knh):
    ref = run_oracle(wl, n, crit=O.CRIT_ETA_D, knh=knh)
    G = make_gpu(wl, O.CRIT_ETA_D, knh=knh)
    masks = []
    for k in range(n):
        G.step(wl.dt)
        masks.append(G.get_mask()[0][0].copy())
    return ref, G, masks


@pytest.mark.parametrize("up", [True, False])
def test_plate_matches_oracle(up):
    wl = W.plate_1d(up=up, nx=600)
    n = 60
    ref, G, masks = _run(wl, n, 1e-4)
    assert np.array_equal(masks[-1], ref[0][2])
    assert ref[0][2].sum() > 0
    compare(wl, G, ref, what=f"plate up={up}")
    G.close()


def test_block_matches_oracle_through_its_phases():
    """Runs through the acceleration (t < t1 = 0.218 s) into the glide."""
    wl = W.block_1d(row=1)
    n = 120
    ref, G, masks = _run(wl, n, 1e-4)
    assert np.array_equal(masks[-1], ref[0][2])
    assert ref[0][2].sum() > 0
    compare(wl, G, ref, what="block Fr=0.25")
    G.close()


def test_block_at_rest_after_t3_stays_at_rest():
    """Still water over the block after it has stopped: nothing moves."""
    wl = W.block_1d(row=0)
    m = wl.members[0]
    t3 = m.t2 + m.t0
    p = O.Params(nx=m.nx, dx=m.dx, slide=O.SLIDE_QUARTIC, A=m.A, L=m.L, xc0=m.xc0, s0=m.s0, t0=m.t0, t2=m.t2)
    d = O.bottom_all(p, m.d0, t3 + 0.1)[0]
    G = make_gpu(wl, O.CRIT_GLOBAL)
    z = np.zeros(m.nx)
    G.set_state(d[None, :], z[None, :], z[None, :], t=t3 + 0.1)
    G.run(wl.dt, 20)
    h, hu, hw, _ = G.get_state()
    assert np.max(np.abs(h[0] - d)) < 1e-14 and np.max(np.abs(hu)) < 1e-14 and np.max(np.abs(hw)) < 1e-14
    G.close()
