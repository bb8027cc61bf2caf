"""ctypes marshalling of the DG-P1 / LDG oracle (``nh_oracle_dg.c``).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the arithmetic is in
the C source; this module only passes numpy arrays.  Per-node arrays hold
2 ne values: node 2i is element i's left end, node 2i+1 its right end.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field, fields

import numpy as np

from . import CRIT_GLOBAL, SLIDE_NONE, lib


class _ParamsDG(C.Structure):
    _fields_ = [
        ("ne", C.c_int), ("dx", C.c_double), ("xl", C.c_double), ("g", C.c_double), ("rho", C.c_double),
        ("b0", C.c_double), ("b1", C.c_double),
        ("slide", C.c_int), ("A", C.c_double), ("L", C.c_double), ("xc0", C.c_double), ("s0", C.c_double),
        ("t0", C.c_double), ("t2", C.c_double),
        ("crit", C.c_int), ("knh", C.c_double), ("enlarge", C.c_int), ("first_step_global", C.c_int),
        ("c11", C.c_double),
    ]


class InfoDG(C.Structure):
    _fields_ = [("n_active", C.c_int), ("status", C.c_int), ("rel_res", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


@dataclass
class ParamsDG:
    """One 1D grid of ne P1 elements (mirrors ``or_dg_params``)."""
    ne: int
    dx: float
    xl: float = 0.0
    g: float = 9.81
    rho: float = 1000.0
    b0: float = 1.0
    b1: float = 0.0
    slide: int = SLIDE_NONE
    A: float = 0.0
    L: float = 1.0
    xc0: float = 0.0
    s0: float = 0.0
    t0: float = 1.0
    t2: float = 0.0
    crit: int = CRIT_GLOBAL
    knh: float = 1e-3
    enlarge: int = 1
    first_step_global: int = 0
    c11: float = 0.5

    def c(self) -> _ParamsDG:
        return _ParamsDG(**{f.name: getattr(self, f.name) for f in fields(self)})

    def nodes(self) -> np.ndarray:
        """Node positions (2 ne)."""
        i = np.arange(self.ne)
        x = np.empty(2 * self.ne)
        x[0::2] = self.xl + i * self.dx
        x[1::2] = self.xl + (i + 1) * self.dx
        return x


_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_U8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_PP = C.POINTER(_ParamsDG)


def _bind(L):
    L.or_dg_bottom.argtypes = [_PP, C.c_double, C.c_double, _D]
    L.or_dg_rhs.argtypes = [_PP, C.c_double] + [_D] * 6
    L.or_dg_predict.argtypes = [_PP, C.c_double, C.c_double] + [_D] * 6
    L.or_dg_mask.argtypes = [_PP, C.c_double, C.c_long, _D, _D, _D, _U8]
    L.or_dg_mask.restype = C.c_int
    L.or_dg_assemble.argtypes = [_PP, C.c_double, C.c_double, _D, _D, _D, _U8, _D, _D]
    L.or_dg_solve.argtypes = [_PP, _D, _D, _D, C.POINTER(C.c_double)]
    L.or_dg_solve.restype = C.c_int
    L.or_dg_correct.argtypes = [_PP, C.c_double, C.c_double, _U8, _D, _D, _D, _D, _D, _D, _D, _D]
    L.or_dg_step.argtypes = [_PP, C.c_double, C.c_long, C.c_double, _D, _D, _D, _D, C.c_void_p,
                             C.POINTER(InfoDG)]
    L.or_dg_step.restype = C.c_int


def _f(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def bottom(p: ParamsDG, x, t):
    """d, d_x, d_xx, d_t, d_xt, d_tt at position x."""
    out = np.zeros(6)
    lib().or_dg_bottom(C.byref(p.c()), float(x), float(t), out)
    return out


def rhs(p: ParamsDG, t, h, hu, hw):
    n = 2 * p.ne
    out = [np.zeros(n) for _ in range(3)]
    lib().or_dg_rhs(C.byref(p.c()), float(t), _f(h), _f(hu), _f(hw), *out)
    return out


def predict(p: ParamsDG, t, dt, h, hu, hw):
    n = 2 * p.ne
    out = [np.zeros(n) for _ in range(3)]
    lib().or_dg_predict(C.byref(p.c()), float(t), float(dt), _f(h), _f(hu), _f(hw), *out)
    return out


def mask(p: ParamsDG, t1, step, ht, hut, hwt):
    m = np.zeros(p.ne, dtype=np.uint8)
    lib().or_dg_mask(C.byref(p.c()), float(t1), int(step), _f(ht), _f(hut), _f(hwt), m)
    return m


def assemble(p: ParamsDG, t1, dt, ht, hut, hwt, m):
    """(blocks [ne, 3, 4, 4] = couplings to element i-1, i, i+1; rhs [ne, 4])."""
    blk = np.zeros(48 * p.ne)
    r = np.zeros(4 * p.ne)
    lib().or_dg_assemble(C.byref(p.c()), float(t1), float(dt), _f(ht), _f(hut), _f(hwt),
                         np.ascontiguousarray(m, dtype=np.uint8), blk, r)
    return blk.reshape(p.ne, 3, 4, 4), r.reshape(p.ne, 4)


def solve(p: ParamsDG, blk, r):
    x = np.zeros(4 * p.ne)
    rel = C.c_double(0.0)
    st = lib().or_dg_solve(C.byref(p.c()), _f(np.asarray(blk).reshape(-1)), _f(np.asarray(r).reshape(-1)), x,
                           C.byref(rel))
    return x.reshape(p.ne, 4), st, rel.value


def dense(p: ParamsDG, blk):
    """The block-tridiagonal matrix as a dense (4 ne, 4 ne) array."""
    n = 4 * p.ne
    A = np.zeros((n, n))
    for i in range(p.ne):
        for q in range(3):
            e = i + q - 1
            if 0 <= e < p.ne:
                A[4 * i:4 * i + 4, 4 * e:4 * e + 4] = blk[i, q]
    return A


@dataclass
class StateDG:
    h: np.ndarray
    hu: np.ndarray
    hw: np.ndarray
    p: np.ndarray = field(default=None)

    def __post_init__(self):
        self.h = _f(self.h).copy()
        self.hu = _f(self.hu).copy()
        self.hw = _f(self.hw).copy()
        self.p = np.zeros_like(self.h) if self.p is None else _f(self.p).copy()


def step(p: ParamsDG, t, step_index, dt, s: StateDG, want_mask=False):
    info = InfoDG()
    m = np.zeros(p.ne, dtype=np.uint8) if want_mask else None
    st = lib().or_dg_step(C.byref(p.c()), float(t), int(step_index), float(dt), s.h, s.hu, s.hw, s.p,
                          m.ctypes.data if want_mask else None, C.byref(info))
    return (st, info.as_dict(), m) if want_mask else (st, info.as_dict())
