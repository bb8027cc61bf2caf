"""ctypes marshalling of the 2D oracle (``nh_oracle2d.c``).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the arithmetic is in
the C source; this module only passes numpy arrays (row-major, x fastest:
cell (i, j) at j * nx + i, shape (ny, nx) on the Python side).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field, fields

import numpy as np

from . import (BC_WALL, CRIT_GLOBAL, GUESS_PREV, LIM_CENTRAL, SLIDE_NONE, SOLVER_AUTO,
               StepInfo, lib)

NCOEF = 9   # C, W, E, S, N, SW, SE, NW, NE


class _Params2(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("bcx", C.c_int), ("bcy", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double), ("x0", C.c_double), ("y0", C.c_double),
        ("g", C.c_double), ("rho", C.c_double), ("limiter", C.c_int),
        ("slide", C.c_int), ("A", C.c_double), ("Lx", C.c_double), ("Ly", C.c_double),
        ("xc0", C.c_double), ("yc0", C.c_double), ("s0", C.c_double), ("t0", C.c_double),
        ("crit", C.c_int), ("knh", C.c_double), ("enlarge", C.c_int), ("first_step_global", C.c_int),
        ("solver", C.c_int), ("rtol", C.c_double), ("max_iter", C.c_int), ("guess", C.c_int),
    ]


@dataclass
class Params2D:
    """Problem description of one 2D grid (mirrors ``or2_params``)."""
    nx: int
    ny: int
    dx: float
    dy: float
    x0: float = 0.0
    y0: float = 0.0
    bcx: int = BC_WALL
    bcy: int = BC_WALL
    g: float = 9.81
    rho: float = 1000.0
    limiter: int = LIM_CENTRAL
    slide: int = SLIDE_NONE
    A: float = 0.0
    Lx: float = 1.0
    Ly: float = 1.0
    xc0: float = 0.0
    yc0: float = 0.0
    s0: float = 0.0
    t0: float = 1.0
    crit: int = CRIT_GLOBAL
    knh: float = 1e-3
    enlarge: int = 1
    first_step_global: int = 0
    solver: int = SOLVER_AUTO
    rtol: float = 1e-13
    max_iter: int = 100000
    guess: int = GUESS_PREV

    def c(self) -> _Params2:
        return _Params2(**{f.name: getattr(self, f.name) for f in fields(self)})


_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_U8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_PP = C.POINTER(_Params2)


def _bind(L):
    L.or2_bottom.argtypes = [_PP, _D, C.c_int, C.c_int, C.c_double, _D]
    L.or2_rhs.argtypes = [_PP, _D, C.c_double] + [_D] * 8
    L.or2_predict.argtypes = [_PP, _D, C.c_double, C.c_double] + [_D] * 8
    L.or2_criterion.argtypes = [_PP, _D, C.c_double] + [_D] * 5
    L.or2_mask.argtypes = [_PP, _D, C.c_double, C.c_long, _D, _D, _D, _D, _U8]
    L.or2_mask.restype = C.c_int
    L.or2_assemble.argtypes = [_PP, _D, C.c_double, C.c_double] + [_D] * 7
    L.or2_apply.argtypes = [_PP, _U8, _D, _D, _D]
    L.or2_solve.argtypes = [_PP, _U8, _D, _D, _D, _D, C.POINTER(StepInfo)]
    L.or2_solve.restype = C.c_int
    L.or2_correct.argtypes = [_PP, _D, C.c_double, C.c_double, _U8, _D] + [_D] * 8
    L.or2_step.argtypes = [_PP, _D, C.c_double, C.c_long, C.c_double, _D, _D, _D, _D, _D,
                           C.c_void_p, C.POINTER(StepInfo)]
    L.or2_step.restype = C.c_int
    L.or2_run.argtypes = [_PP, _D, C.c_double, C.c_long, C.c_double, C.c_long,
                          _D, _D, _D, _D, _D, C.POINTER(StepInfo),
                          C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
    L.or2_run.restype = C.c_int


def _f(a):
    return np.ascontiguousarray(a, dtype=np.float64).reshape(-1)


def _shape(p, a):
    return a.reshape(p.ny, p.nx)


def bottom(p: Params2D, d0, i, j, t):
    """d, d_x, d_y, d_xx, d_yy, d_xy, d_t, d_xt, d_yt, d_tt at cell (i, j)."""
    out = np.zeros(10)
    lib().or2_bottom(C.byref(p.c()), _f(d0), int(i), int(j), float(t), out)
    return out


def rhs(p: Params2D, d0, t, h, hu, hv, hw):
    n = p.nx * p.ny
    out = [np.zeros(n) for _ in range(4)]
    lib().or2_rhs(C.byref(p.c()), _f(d0), float(t), _f(h), _f(hu), _f(hv), _f(hw), *out)
    return [_shape(p, o) for o in out]


def predict(p: Params2D, d0, t, dt, h, hu, hv, hw):
    n = p.nx * p.ny
    out = [np.zeros(n) for _ in range(4)]
    lib().or2_predict(C.byref(p.c()), _f(d0), float(t), float(dt), _f(h), _f(hu), _f(hv), _f(hw), *out)
    return [_shape(p, o) for o in out]


def criterion(p: Params2D, d0, t, ht, hut, hvt, hwt):
    c = np.zeros(p.nx * p.ny)
    lib().or2_criterion(C.byref(p.c()), _f(d0), float(t), _f(ht), _f(hut), _f(hvt), _f(hwt), c)
    return _shape(p, c)


def mask(p: Params2D, d0, t, step, ht, hut, hvt, hwt):
    m = np.zeros(p.nx * p.ny, dtype=np.uint8)
    lib().or2_mask(C.byref(p.c()), _f(d0), float(t), int(step), _f(ht), _f(hut), _f(hvt), _f(hwt), m)
    return _shape(p, m)


def assemble(p: Params2D, d0, t1, dt, ht, hut, hvt, hwt):
    """(coef [9, ny, nx], gamma, R)."""
    n = p.nx * p.ny
    coef, gam, R = np.zeros(NCOEF * n), np.zeros(n), np.zeros(n)
    lib().or2_assemble(C.byref(p.c()), _f(d0), float(t1), float(dt), _f(ht), _f(hut), _f(hvt), _f(hwt),
                       coef, gam, R)
    return coef.reshape(NCOEF, p.ny, p.nx), _shape(p, gam), _shape(p, R)


def apply(p: Params2D, m, coef, x):
    y = np.zeros(p.nx * p.ny)
    lib().or2_apply(C.byref(p.c()), np.ascontiguousarray(m, dtype=np.uint8).reshape(-1), _f(coef), _f(x), y)
    return _shape(p, y)


def solve(p: Params2D, m, coef, gam, R, q0=None):
    q = np.zeros(p.nx * p.ny) if q0 is None else _f(q0).copy()
    info = StepInfo()
    st = lib().or2_solve(C.byref(p.c()), np.ascontiguousarray(m, dtype=np.uint8).reshape(-1), _f(coef),
                         _f(gam), _f(R), q, C.byref(info))
    return _shape(p, q), st, info.as_dict()


def correct(p: Params2D, d0, t1, dt, m, q, ht, hut, hvt, hwt):
    n = p.nx * p.ny
    out = [np.zeros(n) for _ in range(4)]
    lib().or2_correct(C.byref(p.c()), _f(d0), float(t1), float(dt),
                      np.ascontiguousarray(m, dtype=np.uint8).reshape(-1), _f(q),
                      _f(ht), _f(hut), _f(hvt), _f(hwt), *out)
    return [_shape(p, o) for o in out]


@dataclass
class State2D:
    h: np.ndarray
    hu: np.ndarray
    hv: np.ndarray
    hw: np.ndarray
    q: np.ndarray = field(default=None)

    def __post_init__(self):
        self.h = _f(self.h).copy()
        self.hu = _f(self.hu).copy()
        self.hv = _f(self.hv).copy()
        self.hw = _f(self.hw).copy()
        self.q = np.zeros_like(self.h) if self.q is None else _f(self.q).copy()

    def fields(self, p):
        return [_shape(p, a) for a in (self.h, self.hu, self.hv, self.hw, self.q)]


def step(p: Params2D, d0, t, step_index, dt, s: State2D, want_mask=False):
    info = StepInfo()
    m = np.zeros(p.nx * p.ny, dtype=np.uint8) if want_mask else None
    st = lib().or2_step(C.byref(p.c()), _f(d0), float(t), int(step_index), float(dt),
                        s.h, s.hu, s.hv, s.hw, s.q, m.ctypes.data if want_mask else None, C.byref(info))
    return (st, info.as_dict(), _shape(p, m)) if want_mask else (st, info.as_dict())


def run(p: Params2D, d0, t_start, step0, dt, n_steps, s: State2D):
    info = StepInfo()
    ti, ta = C.c_longlong(0), C.c_longlong(0)
    st = lib().or2_run(C.byref(p.c()), _f(d0), float(t_start), int(step0), float(dt), int(n_steps),
                       s.h, s.hu, s.hv, s.hw, s.q, C.byref(info), C.byref(ti), C.byref(ta))
    return st, info.as_dict(), ti.value, ta.value
