"""Seeded synthetic inputs shared by the CUDA path, the oracle, tests and bench.

This module only builds inputs: grids, bathymetry, slide parameters, initial
states and time steps.  It holds none of the method's arithmetic (no fluxes,
criteria, elliptic coefficients or corrections) and imports neither the CUDA
binding nor the oracle.

Workloads (sizes are those of the synthetic configurations the library is
measured on; the paper's own runs are quoted where they are used):

* ``solitary_1d`` -- Green-Naghdi / Serre solitary wave over a flat bottom
  (Sec. 4.1, Eq. 18): eta = a sech^2(K (x - c t - x0)), u = c eta / (d + eta),
  c = sqrt(g (d + a)), K = sqrt(3 a / (4 d^2 (d + a))); the initial hw follows
  from the constraint (Eq. 4) for a flat, static bottom, hw = -h^2 u_x / 2.
* ``slide_1d`` -- still water over a plane slope d0 = min(h_min + s x, h_max)
  with a Gaussian mound of height A and width L moving down-slope as
  s(t) = s0 ln cosh(t / t0); per-member A, L, s0 drawn from a seeded uniform
  +-30 % band around the nominal values.
* ``ensemble_1d`` -- uneven 1D slide members with drawn sizes and parameters.
* ``line_soliton_2d`` -- the solitary wave in x, uniform in y, periodic.
* ``landslide_2d`` -- an elliptic Gaussian slide on a plane slope, walls.
* ``landslide_ensemble_2d`` -- uneven 2D landslide grids with drawn sizes,
  slopes and slide parameters, one time step for all.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

G = 9.81


# ---------------------------------------------------------------- closed form

def solitary_fields(x, t, a, d, x0, g=G):
    """(eta, u, hw) of the solitary wave of Eq. 18 at positions x, time t."""
    c = math.sqrt(g * (d + a))
    K = math.sqrt(3.0 * a / (4.0 * d * d * (d + a)))
    xi = K * (np.asarray(x, dtype=np.float64) - c * t - x0)
    sech2 = 1.0 / np.cosh(xi) ** 2
    eta = a * sech2
    u = c * eta / (d + eta)
    eta_x = -2.0 * K * eta * np.tanh(xi)
    u_x = c * d * eta_x / (d + eta) ** 2
    h = d + eta
    hw = -0.5 * h * h * u_x
    return eta, u, hw


def solitary_speed(a, d, g=G):
    return math.sqrt(g * (d + a))


def cfl_dt(T, cfl, dx, speed):
    """Fixed step dt = T / ceil(T / dt_cfl), dt_cfl = cfl dx / speed."""
    n = int(math.ceil(T / (cfl * dx / speed) - 1e-9))
    return T / n, n


# ------------------------------------------------------------------ workloads

@dataclass
class Member1D:
    """One 1D problem: grid, bottom, slide and initial state."""
    nx: int
    dx: float
    xl: float
    d0: np.ndarray
    h: np.ndarray
    hu: np.ndarray
    hw: np.ndarray
    slide: int = 0           # 0 static, 1 Gaussian mound, 2 impulsive plate, 3 sliding block
    A: float = 0.0
    L: float = 1.0
    xc0: float = 0.0
    s0: float = 0.0
    t0: float = 1.0
    t2: float = 0.0          # sliding block: end of the glide

    @property
    def x(self):
        return self.xl + (np.arange(self.nx) + 0.5) * self.dx


@dataclass
class Workload1D:
    name: str
    members: list
    dt: float
    n_steps: int
    T: float
    bc: int = 0              # 0 wall, 1 periodic
    amplitude: float = 0.0   # wave amplitude a used in error bounds
    meta: dict = field(default_factory=dict)

    @property
    def nx(self):
        return self.members[0].nx


def solitary_1d(nx=2000, length=200.0, depth=1.0, a=0.1, x0=None, T=20.0, cfl=0.5, g=G):
    """1D solitary wave, flat bottom, walls (default: h = 1 m, a/h = 0.1,
    [0, 200] m, dx = 0.1 m, CFL 0.5, T = 20 s)."""
    dx = length / nx
    x0 = length / 4.0 if x0 is None else x0
    x = (np.arange(nx) + 0.5) * dx
    eta, u, hw = solitary_fields(x, 0.0, a, depth, x0, g)
    h = depth + eta
    d0 = np.full(nx, depth)
    speed = float(np.max(np.abs(u) + np.sqrt(g * h)))
    dt, n = cfl_dt(T, cfl, dx, speed)
    m = Member1D(nx=nx, dx=dx, xl=0.0, d0=d0, h=h, hu=h * u, hw=hw)
    return Workload1D("solitary_1d", [m], dt, n, T, amplitude=a,
                      meta={"depth": depth, "a": a, "x0": x0, "length": length})


def slide_1d(n_members=64, nx=50000, length=40.0, h_min=0.05, h_max=1.0, slope=0.25,
             A=0.05, L=0.5, s0=2.0, t0=1.0, xc0=1.0, spread=0.3, T=2.0, cfl=0.5,
             seed0=0, g=G):
    """Batch of 1D moving-bottom slides; member k uses numpy default_rng(seed0 + k)
    to scale A, L, s0 by U(1 - spread, 1 + spread)."""
    dx = length / nx
    x = (np.arange(nx) + 0.5) * dx
    d0 = np.minimum(h_min + slope * x, h_max)
    members = []
    for k in range(n_members):
        rng = np.random.default_rng(seed0 + k)
        fa, fl, fs = rng.uniform(1.0 - spread, 1.0 + spread, size=3)
        Ak, Lk, sk = A * fa, L * fl, s0 * fs
        xi = (x - xc0) / Lk
        d = d0 - Ak * np.exp(-xi * xi)
        members.append(Member1D(nx=nx, dx=dx, xl=0.0, d0=d0.copy(), h=d.copy(),
                                hu=np.zeros(nx), hw=np.zeros(nx), slide=1,
                                A=Ak, L=Lk, xc0=xc0, s0=sk, t0=t0))
    speed = math.sqrt(g * h_max)
    dt, n = cfl_dt(T, cfl, dx, speed)
    return Workload1D("slide_1d", members, dt, n, T, amplitude=A,
                      meta={"h_min": h_min, "h_max": h_max, "slope": slope, "A": A, "L": L,
                            "s0": s0, "t0": t0, "xc0": xc0, "spread": spread, "seed0": seed0})


# The paper's sliding-block table (Sec. 4.3), one row per Froude number
# 0.125, 0.25, 0.375: acceleration a0 (m/s^2), t1, t2 (s); the glide speed
# is a0 t1 and the block stops at t2 + t1 (the table's ut and t3 to rounding).
BLOCK_TABLE = ((1.5, 0.109, 2.109), (1.5, 0.218, 2.218), (1.5, 0.327, 2.327))


def plate_1d(up=True, nx=1200, dx=0.025, h0=0.05, zeta0=0.005, b=0.61, T=2.0, cfl=None, dt=0.01, g=G):
    """The impulsively moved plate of Sec. 4.2 on a flat bottom h0 = 0.05 m:
    d = h0 - zeta0 (1 - exp(-alpha t)) on 0 <= x < b next to the wall at x = 0
    (mirror of |x| < b), b = 0.61 m, |zeta0| = 0.005 m (positive: the plate
    rises), alpha = 1.11 / t_c with t_c sqrt(g h0) / b = 0.148 (up) or 0.093
    (down); the paper's dx = 0.025 m and dt = 0.01 s; still water, walls (the
    far wall stands in for the paper's absorbing end)."""
    ratio = 0.148 if up else 0.093
    tc = ratio * b / math.sqrt(g * h0)
    z0 = zeta0 if up else -zeta0
    d0 = np.full(nx, h0)
    m = Member1D(nx=nx, dx=dx, xl=0.0, d0=d0, h=d0.copy(), hu=np.zeros(nx), hw=np.zeros(nx), slide=2,
                 A=z0, L=b, xc0=0.0, s0=0.0, t0=tc / 1.11)
    n = int(math.ceil(T / dt))
    return Workload1D("plate_1d", [m], T / n, n, T, amplitude=abs(z0),
                      meta={"up": up, "t_c": tc, "alpha": 1.11 / tc})


def block_1d(row=1, nx=400, length=10.0, h0=0.175, Hs=0.026, Ls=0.5, xc0=2.0, T=3.0, dt=0.005):
    """The sliding block of Sec. 4.3 over a flat bottom h0 = 0.175 m: the
    bump H_s (1 - (2 (x - S)/L_s)^4), H_s = 0.026 m, L_s = 0.5 m, centred at
    xc0 + S(t) with S(t) from BLOCK_TABLE[row]; still water over it, walls;
    the paper's dt = 0.005 s and dx = 0.025 m (a third of the paper's).  The
    bump's edges are kinks of the depth: at spacings far below the paper's
    the reaction term gamma turns negative next to them and the elliptic
    problem loses definiteness (seen at dx = 5 mm)."""
    a0, t1, t2 = BLOCK_TABLE[row]
    dx = length / nx
    x = (np.arange(nx) + 0.5) * dx
    d0 = np.full(nx, h0)
    xi = 2.0 * (x - xc0) / Ls
    mound = np.where(np.abs(xi) < 1.0, Hs * (1.0 - xi ** 4), 0.0)
    m = Member1D(nx=nx, dx=dx, xl=0.0, d0=d0, h=d0 - mound, hu=np.zeros(nx), hw=np.zeros(nx), slide=3,
                 A=Hs, L=Ls, xc0=xc0, s0=a0, t0=t1, t2=t2)
    n = int(math.ceil(T / dt))
    return Workload1D("block_1d", [m], T / n, n, T, amplitude=Hs,
                      meta={"a0": a0, "t1": t1, "t2": t2, "travel": a0 * t1 * t2})


def ensemble_1d(n_members=32, nx_min=16384, nx_max=131072, dx=0.002, h_min=0.1, h_max=2.0,
                slope=(0.1, 0.3), A=(0.05, 0.15), L=(0.5, 1.5), s0=(1.0, 3.0), t0=1.0,
                d_start=0.6, T=1.0, cfl=0.5, g=G):
    """Ensemble of uneven 1D landslide runs: member k draws, from
    numpy default_rng(k), its cell count (uniform in [nx_min, nx_max], a
    multiple of 256), slope tan(theta), mound height A, width L and travel s0
    from the given uniform ranges; d0 = min(h_min + tan(theta) x, h_max), the
    mound starts where d0 = d_start.  One dt for the whole ensemble."""
    members = []
    for k in range(n_members):
        rng = np.random.default_rng(k)
        nx = int(rng.integers(nx_min // 256, nx_max // 256 + 1)) * 256
        tan, Ak, Lk, sk = (rng.uniform(*slope), rng.uniform(*A), rng.uniform(*L), rng.uniform(*s0))
        x = (np.arange(nx) + 0.5) * dx
        d0 = np.minimum(h_min + tan * x, h_max)
        xc0 = (d_start - h_min) / tan
        xi = (x - xc0) / Lk
        d = d0 - Ak * np.exp(-xi * xi)
        members.append(Member1D(nx=nx, dx=dx, xl=0.0, d0=d0, h=d.copy(), hu=np.zeros(nx),
                                hw=np.zeros(nx), slide=1, A=Ak, L=Lk, xc0=xc0, s0=sk, t0=t0))
    dt, n = cfl_dt(T, cfl, dx, math.sqrt(g * h_max))
    return Workload1D("ensemble_1d", members, dt, n, T, amplitude=A[1],
                      meta={"nx_range": (nx_min, nx_max), "dx": dx, "slope": slope, "A": A, "L": L,
                            "s0": s0, "t0": t0})


def standing_wave_1d(nx=128, depth=1.0, kh=1.0, amp=1e-4, modes=1, g=G):
    """Small-amplitude standing wave eta = amp cos(k x) in a walled basin of
    length modes * pi / k (k = kh / depth), at rest."""
    k = kh / depth
    length = modes * math.pi / k
    dx = length / nx
    x = (np.arange(nx) + 0.5) * dx
    h = depth + amp * np.cos(k * x)
    m = Member1D(nx=nx, dx=dx, xl=0.0, d0=np.full(nx, depth), h=h,
                 hu=np.zeros(nx), hw=np.zeros(nx))
    return m, k, length


# ------------------------------------------------------------------- 2D grids

@dataclass
class Workload2D:
    """One 2D grid: arrays (ny, nx), x fastest."""
    name: str
    nx: int
    ny: int
    dx: float
    dy: float
    d0: np.ndarray
    h: np.ndarray
    hu: np.ndarray
    hv: np.ndarray
    hw: np.ndarray
    dt: float
    bc_x: int = 0
    bc_y: int = 0
    amplitude: float = 0.0
    slide: dict = None
    meta: dict = field(default_factory=dict)


def cfl_dt_2d(cfl, dx, dy, speed):
    """dt = cfl / (speed (1/dx + 1/dy))."""
    return cfl / (speed * (1.0 / dx + 1.0 / dy))


def line_soliton_2d(nx=1024, ny=1024, dx=0.05, depth=1.0, a=0.2, x0=None, cfl=0.5, g=G):
    """Line soliton (Eq. 18 in x, uniform in y) on a flat bottom, periodic in
    x and y (default: h = 1 m, a/h = 0.2, 1024 x 1024 cells, dx = 0.05 m)."""
    length = nx * dx
    x0 = length / 4.0 if x0 is None else x0
    x = (np.arange(nx) + 0.5) * dx
    eta, u, hw = solitary_fields(x, 0.0, a, depth, x0, g)
    h1 = depth + eta
    tile = lambda v: np.tile(v, (ny, 1))
    speed = float(np.max(np.abs(u) + np.sqrt(g * h1)))
    dt = cfl_dt_2d(cfl, dx, dx, speed)
    return Workload2D("line_soliton_2d", nx, ny, dx, dx, np.full((ny, nx), depth), tile(h1), tile(h1 * u),
                      np.zeros((ny, nx)), tile(hw), dt, bc_x=1, bc_y=1, amplitude=a,
                      meta={"depth": depth, "a": a, "x0": x0})


def landslide_2d(n=2048, dx=0.02, h_min=0.1, h_max=2.0, slope=0.2, A=0.1, Lx=1.0, Ly=0.5, s0=2.0, t0=1.0,
                 d_start=0.6, cfl=0.5, g=G):
    """Elliptic Gaussian slide on a plane slope d0 = min(h_min + slope x, h_max)
    (default: 2048 x 2048 cells, dx = 0.02 m, A = 0.1 m, Lx = 1 m, Ly = 0.5 m,
    s0 = 2 m, t0 = 1 s), starting where d0 = d_start, centred in y; still
    water, walls."""
    x = (np.arange(n) + 0.5) * dx
    d0 = np.tile(np.minimum(h_min + slope * x, h_max), (n, 1))
    xc0 = (d_start - h_min) / slope
    yc0 = n * dx / 2.0
    X, Y = np.meshgrid(x, x)
    h = d0 - A * np.exp(-((X - xc0) / Lx) ** 2 - ((Y - yc0) / Ly) ** 2)
    dt = cfl_dt_2d(cfl, dx, dx, math.sqrt(g * h_max))
    z = np.zeros((n, n))
    return Workload2D("landslide_2d", n, n, dx, dx, d0, h, z, z.copy(), z.copy(), dt, amplitude=A,
                      slide=dict(A=A, Lx=Lx, Ly=Ly, xc0=xc0, yc0=yc0, s0=s0, t0=t0),
                      meta={"h_min": h_min, "h_max": h_max, "slope": slope})


def landslide_ensemble_2d(n_members=32, sizes=tuple(range(256, 1025, 64)), dx=0.02, h_min=0.1, h_max=2.0,
                          slope=(0.1, 0.3), A=(0.05, 0.15), L=(0.5, 1.5), s0=(1.0, 3.0), t0=1.0,
                          d_start=0.6, x_frac_max=0.3, cfl=0.5, g=G, seed0=0):
    """Ensemble of uneven 2D landslide runs: member m draws, from
    numpy.random.default_rng(m), nx and ny independently from `sizes`, the
    plane slope tan(theta), the mound amplitude A, its length Lx (Ly = Lx / 2)
    and run-out s0 uniformly from the given ranges; d0 = min(h_min + slope x,
    h_max) at spacing dx in x and y; the slide starts where d0 = d_start (at
    most x_frac_max of the basin length), centred in y; still water, walls.
    One dt for all members: CFL cfl at depth h_max.  Member m is drawn from
    default_rng(seed0 + m).  Returns (members, dt)."""
    out = []
    for m in range(n_members):
        rng = np.random.default_rng(seed0 + m)
        nx = int(rng.choice(sizes))
        ny = int(rng.choice(sizes))
        sl_m = float(rng.uniform(*slope))
        A_m = float(rng.uniform(*A))
        Lx = float(rng.uniform(*L))
        s0_m = float(rng.uniform(*s0))
        x = (np.arange(nx) + 0.5) * dx
        y = (np.arange(ny) + 0.5) * dx
        d0 = np.tile(np.minimum(h_min + sl_m * x, h_max), (ny, 1))
        xc0 = min((d_start - h_min) / sl_m, x_frac_max * nx * dx)
        yc0 = ny * dx / 2.0
        X, Y = np.meshgrid(x, y)
        h = d0 - A_m * np.exp(-((X - xc0) / Lx) ** 2 - ((Y - yc0) / (Lx / 2.0)) ** 2)
        z = np.zeros((ny, nx))
        out.append(Workload2D(f"landslide_ens_{seed0 + m}", nx, ny, dx, dx, d0, h, z, z.copy(), z.copy(), 0.0,
                              amplitude=A_m,
                              slide=dict(A=A_m, Lx=Lx, Ly=Lx / 2.0, xc0=xc0, yc0=yc0, s0=s0_m, t0=t0),
                              meta={"h_min": h_min, "h_max": h_max, "slope": sl_m}))
    dt = cfl_dt_2d(cfl, dx, dx, math.sqrt(g * h_max))
    for w in out:
        w.dt = dt
    return out, dt


# ------------------------------------------------------------- DG workloads

@dataclass
class MemberDG:
    """One 1D member in the DG-P1 discretisation: ne elements of width dx
    from xl, static depth b0 + b1 (x - xl) (the form the DG oracle takes),
    a moving bottom and the nodal initial state (2 ne values per field, node
    2i = element i's left end)."""
    ne: int
    dx: float
    xl: float
    b0: float
    b1: float
    h: np.ndarray
    hu: np.ndarray
    hw: np.ndarray
    slide: int = 0
    A: float = 0.0
    L: float = 1.0
    xc0: float = 0.0
    s0: float = 0.0
    t0: float = 1.0
    t2: float = 0.0

    def nodes(self):
        i = np.arange(self.ne)
        x = np.empty(2 * self.ne)
        x[0::2] = self.xl + i * self.dx
        x[1::2] = self.xl + (i + 1) * self.dx
        return x

    def d0(self):
        return self.b0 + self.b1 * (self.nodes() - self.xl)


@dataclass
class WorkloadDG:
    name: str
    members: list
    dt: float
    amplitude: float
    meta: dict = field(default_factory=dict)


def slide_dg_1d(n_members=64, ne=50000, length=40.0, b0=0.05, b1=0.025, A=0.05, L=0.5, s0=2.0, t0=1.0,
                xc0=1.0, spread=0.3, courant=0.2, seed0=0, g=G):
    """Batch of 1D moving-bottom slides in DG-P1 form: ne elements over
    [0, length] on the plane slope d0 = b0 + b1 x (0.05 m to 1.05 m), a
    Gaussian mound moving as s0 ln cosh(t/t0) from xc0, member k drawing A,
    L, s0 scaled by U(1 - spread, 1 + spread) from default_rng(seed0 + k);
    still water at t = 0; dt at Courant number `courant` on the deepest
    water (the P1 / Heun limit is 1/3)."""
    dx = length / ne
    members = []
    for k in range(n_members):
        rng = np.random.default_rng(seed0 + k)
        fa, fl, fs = rng.uniform(1.0 - spread, 1.0 + spread, size=3)
        m = MemberDG(ne=ne, dx=dx, xl=0.0, b0=b0, b1=b1, h=None, hu=None, hw=None, slide=1,
                     A=A * fa, L=L * fl, xc0=xc0, s0=s0 * fs, t0=t0)
        x = m.nodes()
        xi = (x - xc0) / m.L
        m.h = m.d0() - m.A * np.exp(-xi * xi)
        m.hu = np.zeros(2 * ne)
        m.hw = np.zeros(2 * ne)
        members.append(m)
    dt = courant * dx / math.sqrt(g * (b0 + b1 * length))
    return WorkloadDG("slide_dg_1d", members, dt, A,
                      meta={"b0": b0, "b1": b1, "A": A, "L": L, "s0": s0, "t0": t0, "xc0": xc0,
                            "spread": spread, "courant": courant, "seed0": seed0, "length": length})
