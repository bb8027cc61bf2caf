"""The seeded input generators (CPU): reproducible, within their stated
ranges, and consistent with the quantities they fix (still water over the
slide, CFL time steps)."""
import math

import numpy as np

from paper_2505_17025_gb300 import workloads as W


def test_landslide_ensemble_2d_draws():
    a, dt_a = W.landslide_ensemble_2d()
    b, dt_b = W.landslide_ensemble_2d()
    assert dt_a == dt_b and len(a) == 32
    sizes = set(range(256, 1025, 64))
    for m, (x, y) in enumerate(zip(a, b)):
        assert (x.nx, x.ny) == (y.nx, y.ny) and x.slide == y.slide
        assert np.array_equal(x.h, y.h)
        assert x.nx in sizes and x.ny in sizes
        assert x.d0.shape == (x.ny, x.nx) and x.h.shape == (x.ny, x.nx)
        s = x.slide
        assert 0.05 <= s["A"] <= 0.15 and 0.5 <= s["Lx"] <= 1.5 and s["Ly"] == s["Lx"] / 2
        assert 1.0 <= s["s0"] <= 3.0 and 0.1 <= x.meta["slope"] <= 0.3
        # still water over the slide: the surface h - (d0 - mound) is zero
        xc = (np.arange(x.nx) + 0.5) * x.dx
        yc = (np.arange(x.ny) + 0.5) * x.dy
        X, Y = np.meshgrid(xc, yc)
        mound = s["A"] * np.exp(-((X - s["xc0"]) / s["Lx"]) ** 2 - ((Y - s["yc0"]) / s["Ly"]) ** 2)
        assert np.max(np.abs(x.h - (x.d0 - mound))) < 1e-15
        assert np.all(x.h > 0)
        # member m is drawn from its own seed: the same member alone gives the same draw
        one, _ = W.landslide_ensemble_2d(n_members=m + 1)
        assert one[m].slide == s and (one[m].nx, one[m].ny) == (x.nx, x.ny)
    # one step for all: CFL 0.5 at 2 m depth on the 0.02 m spacing
    assert abs(dt_a - 0.5 / (math.sqrt(9.81 * 2.0) * 2 / 0.02)) < 1e-15
    assert 1.0e7 < sum(x.nx * x.ny for x in a) < 2.5e7


def test_two_dimensional_workloads_shapes():
    sol = W.line_soliton_2d(nx=64, ny=16, dx=0.5)
    assert sol.h.shape == (16, 64) and np.all(sol.h >= 1.0)
    # uniform in y, the wave's crest a/h = 0.2 above the still depth
    assert np.allclose(sol.h, sol.h[0:1, :]) and abs(sol.h.max() - 1.2) < 0.01   # crest between cell centres
    assert not np.any(sol.hv)
    ls = W.landslide_2d(n=64, dx=0.2)
    assert ls.h.shape == (64, 64) and ls.slide["A"] == 0.1
    assert np.min(ls.d0) >= 0.1 and np.max(ls.d0) <= 2.0


def test_dg_slide_workload():
    """The DG slide batch: linear nodal depths from 0.05 m to 1.05 m, still
    water over each member's mound, members drawn from their own seeds, dt at
    Courant 0.2 on the deepest water."""
    w = W.slide_dg_1d(n_members=3, ne=1000)
    assert len(w.members) == 3
    for k, m in enumerate(w.members):
        x = m.nodes()
        assert x.shape == (2000,) and x[0] == 0.0 and abs(x[-1] - 40.0) < 1e-12
        assert np.all(x[1::2] - x[0::2] > 0) and np.array_equal(x[1:-1:2], x[2::2])   # shared end points
        d0 = m.d0()
        assert abs(d0[0] - 0.05) < 1e-15 and abs(d0[-1] - 1.05) < 1e-12
        mound = m.A * np.exp(-((x - m.xc0) / m.L) ** 2)
        assert np.max(np.abs(m.h - (d0 - mound))) < 1e-15 and np.all(m.h > 0)
        assert not np.any(m.hu) and not np.any(m.hw)
        assert 0.7 * 0.05 <= m.A <= 1.3 * 0.05 and 0.7 * 2.0 <= m.s0 <= 1.3 * 2.0
        one = W.slide_dg_1d(n_members=k + 1, ne=1000).members[k]
        assert (one.A, one.L, one.s0) == (m.A, m.L, m.s0)
    assert abs(w.dt - 0.2 * w.members[0].dx / math.sqrt(9.81 * 1.05)) < 1e-15


def test_dg_cyclic_reduction_byte_count():
    """The bench's algorithmic bytes of the DG p-system solve: no global level
    below 513 rows (all in shared memory: rows in, x out), otherwise each
    level reads its rows and writes half as many, and the total grows with
    the marked elements."""
    import bench
    red, back = bench._dg_cr_bytes(300, 300)
    assert back == 0.0 and red == (112.0 + 16.0) * 300
    red1, back1 = bench._dg_cr_bytes(50000, 50000)
    red2, back2 = bench._dg_cr_bytes(25000, 50000)
    assert red1 > red2 > 0 and back1 > back2 > 0
    # 7 global levels at 50 000 elements (50 000 / 2^7 = 391 <= 512)
    n, lev = 50000, 0
    while -(-50000 // (1 << lev)) > 512:
        lev += 1
    assert lev == 7
    assert red1 < 4.0 * 112.0 * 50000 and back1 < 2.0 * 112.0 * 50000
