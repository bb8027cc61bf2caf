"""Pins of the oracle's two bottom motions from the paper (CPU).

* The impulsive plate (Sec. 4.2): d = h0 - zeta0 (1 - exp(-alpha t)) on
  |x - xc0| < b, with alpha = 1.11 / t_c and t_c sqrt(g h0) / b = 0.148 (up)
  or 0.093 (down).
* The sliding block (Sec. 4.3): d = h0 - H_s (1 - (2 (x - S(t)) / L_s)^4) on
  |x - S| < L_s / 2 with the piecewise-quadratic S(t) of the paper's table.

Checked against what the definitions fix independently of the oracle's code:
closed forms of S(t) at the phase boundaries (continuity, the total travel
a0 t1 t2 that the table's parameters imply), the time and space derivatives
the method needs against finite differences of the depth itself, the block's
volume 4/5 H_s L_s, lake at rest once the block stops, mass conservation
while the bottom moves, and the plate's limits."""
import math

import numpy as np
import pytest

import oracle as O

# the paper's sliding-block table (Fr = 0.125, 0.25, 0.375): a0, ut, t1, t2, t3
TABLE = [(1.5, 0.163, 0.109, 2.109, 2.218), (1.5, 0.327, 0.218, 2.218, 2.436), (1.5, 0.491, 0.327, 2.327, 2.654)]


def _block(nx=400, dx=0.01, row=1, xc0=1.5, h0=0.175):
    a0, ut, t1, t2, t3 = TABLE[row]
    p = O.Params(nx=nx, dx=dx, slide=O.SLIDE_QUARTIC, A=0.026, L=0.5, xc0=xc0, s0=a0, t0=t1, t2=t2)
    return p, np.full(nx, h0)


def _S(p, d0, t):
    """Block position from the depth: the centre of the bump's mass."""
    x = (np.arange(p.nx) + 0.5) * p.dx
    m = d0 - O.bottom_all(p, d0, t)[0]
    return float(np.sum(x * m) / np.sum(m)) - p.xc0


def test_table_is_consistent_with_continuous_velocity():
    """ut = a0 t1 and t3 = t2 + t1 in the paper's table (to its rounding):
    the reading that makes S' continuous and zero after t3."""
    for a0, ut, t1, t2, t3 in TABLE:
        assert abs(ut - a0 * t1) < 1e-3
        assert abs(t3 - (t2 + t1)) < 1e-9


@pytest.mark.parametrize("row", [0, 1, 2])
def test_block_position_closed_forms(row):
    a0, ut, t1, t2, t3 = TABLE[row]
    p, d0 = _block(row=row, nx=1200, dx=0.0025)
    # before motion and at the phase ends: a0 t^2 / 2, then glide, total travel a0 t1 t2
    assert abs(_S(p, d0, 0.0)) < 1e-12
    assert abs(_S(p, d0, t1) - 0.5 * a0 * t1 * t1) < 1e-6
    assert abs(_S(p, d0, t2) - (0.5 * a0 * t1 * t1 + a0 * t1 * (t2 - t1))) < 1e-6
    assert abs(_S(p, d0, t2 + t1) - a0 * t1 * t2) < 1e-6
    assert abs(_S(p, d0, t2 + t1 + 1.0) - a0 * t1 * t2) < 1e-6


@pytest.mark.parametrize("t", [0.05, 0.15, 0.6, 2.15, 2.3, 3.0])
def test_block_derivatives_match_finite_differences(t):
    """d_t, d_tt from differences in time of d; d_x, d_xx, d_xt from
    differences of d over shifted grids (the bump is smooth inside)."""
    p, d0 = _block(row=1)
    e = 1e-5
    b = O.bottom_all(p, d0, t)
    bp, bm = O.bottom_all(p, d0, t + e), O.bottom_all(p, d0, t - e)
    inside = np.abs(d0 - b[0]) > 1e-3 * p.A          # away from the bump's edges
    dt_fd = (bp[0] - bm[0]) / (2 * e)
    dtt_fd = (bp[0] - 2 * b[0] + bm[0]) / (e * e)
    assert np.max(np.abs(b[3] - dt_fd)[inside]) < 1e-6
    assert np.max(np.abs(b[5] - dtt_fd)[inside]) < 2e-2 * max(1.0, np.max(np.abs(b[5])))
    hx = 1e-5
    qp = O.Params(**{**p.__dict__, "xl": p.xl + hx})
    qm = O.Params(**{**p.__dict__, "xl": p.xl - hx})
    dp, dm = O.bottom_all(qp, d0, t), O.bottom_all(qm, d0, t)
    dx_fd = (dp[0] - dm[0]) / (2 * hx)
    dxx_fd = (dp[0] - 2 * b[0] + dm[0]) / (hx * hx)
    dxt_fd = (dp[3] - dm[3]) / (2 * hx)
    assert np.max(np.abs(b[1] - dx_fd)[inside]) < 1e-6
    assert np.max(np.abs(b[2] - dxx_fd)[inside]) < 1e-2 * np.max(np.abs(b[2]))
    assert np.max(np.abs(b[4] - dxt_fd)[inside]) < 1e-5


def test_block_volume_and_shape():
    """Volume of H_s (1 - xi^4) over |xi| < 1 is 4/5 H_s L_s; zero outside."""
    p, d0 = _block(nx=4000, dx=0.001)
    m = d0 - O.bottom_all(p, d0, 0.7)[0]
    assert abs(np.sum(m) * p.dx - 0.8 * p.A * p.L) < 1e-6
    assert np.min(m) >= 0.0 and abs(np.max(m) - p.A) < 1e-6


def test_lake_at_rest_after_block_stops_and_mass_while_moving():
    p, d0 = _block(nx=300, dx=0.02, xc0=2.0)
    p.crit, p.knh, p.enlarge, p.rtol = O.CRIT_GLOBAL, 1e-3, 1, 1e-13
    a0, ut, t1, t2, t3 = TABLE[1]
    t_rest = t3 + 0.2
    d = O.bottom_all(p, d0, t_rest)[0]
    s = O.State(d.copy(), np.zeros(p.nx), np.zeros(p.nx))
    st, info, _, _ = O.run(p, d0, t_rest, 1, 0.004, 40, s)
    assert st == O.OK
    assert np.max(np.abs(s.h - d)) < 1e-14 and np.max(np.abs(s.hu)) < 1e-14 and np.max(np.abs(s.hw)) < 1e-14
    # while it moves: walls keep sum(h) dx
    d = O.bottom_all(p, d0, 0.0)[0]
    s = O.State(d.copy(), np.zeros(p.nx), np.zeros(p.nx))
    st, info, _, _ = O.run(p, d0, 0.0, 0, 0.004, 200, s)
    assert st == O.OK
    assert abs(np.sum(s.h) - np.sum(d)) <= 1e-12 * np.sum(d)
    assert np.max(np.abs(s.hu)) > 1e-4                                  # the block made waves


@pytest.mark.parametrize("ratio", [0.148, 0.093])
def test_plate_displacement_and_rates(ratio):
    """The paper's plate: h0 = 0.05 m, zeta0 = 0.005 m, b = 0.61 m,
    alpha = 1.11 / t_c with t_c sqrt(g h0) / b = ratio."""
    h0, z0, b, g = 0.05, 0.005, 0.61, 9.81
    tc = ratio * b / math.sqrt(g * h0)
    t0 = tc / 1.11
    p = O.Params(nx=200, dx=0.01, slide=O.SLIDE_PLATE_EXP, A=z0, L=b, xc0=0.0, t0=t0)
    d0 = np.full(p.nx, h0)
    x = (np.arange(p.nx) + 0.5) * p.dx
    on = np.abs(x) < b
    for t in (0.0, 0.5 * t0, t0, 3 * t0, 50 * t0):
        bb = O.bottom_all(p, d0, t)
        e = math.exp(-t / t0)
        assert np.allclose(bb[0][on], h0 - z0 * (1 - e), atol=1e-16) and np.all(bb[0][~on] == h0)
        assert np.allclose(bb[3][on], -z0 * e / t0, rtol=1e-14) and np.all(bb[3][~on] == 0.0)
        assert np.allclose(bb[5][on], z0 * e / t0 ** 2, rtol=1e-14)
        assert np.all(bb[1] == 0.0) and np.all(bb[2] == 0.0) and np.all(bb[4] == 0.0)
    # finite difference in time of the depth
    tt, e = 0.7 * t0, 1e-7 * t0
    dfd = (O.bottom_all(p, d0, tt + e)[0] - O.bottom_all(p, d0, tt - e)[0]) / (2 * e)
    assert np.max(np.abs(dfd - O.bottom_all(p, d0, tt)[3])) < 1e-6
