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
