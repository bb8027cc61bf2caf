"""FP64 CPU oracle of the locally adaptive non-hydrostatic SWE method.

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow definition that the
CUDA library is checked against: only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA path (``paper_2505_17025_gb300``) and never imports it.

The C source (``nh_oracle.c``) holds the arithmetic, each function citing the
paper's section or equation it follows; this module only compiles it with gcc
and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIB = None

# enums (mirror nh_oracle.h)
BC_WALL, BC_PERIODIC = 0, 1
LIM_NONE, LIM_CENTRAL, LIM_MINMOD, LIM_MC = 0, 1, 2, 3
SLIDE_NONE, SLIDE_GAUSS_LNCOSH, SLIDE_PLATE_EXP, SLIDE_QUARTIC = 0, 1, 2, 3
CRIT_GLOBAL, CRIT_HYDROSTATIC, CRIT_ETA_D, CRIT_ETA_X, CRIT_U, CRIT_U_X, CRIT_W, CRIT_W_X = range(8)
SOLVER_AUTO, SOLVER_CG, SOLVER_BICGSTAB, SOLVER_DENSE, SOLVER_BANDED = 0, 1, 2, 3, 4
GUESS_ZERO, GUESS_PREV = 0, 1
OK, NOT_CONVERGED, BAD_ARG, SINGULAR = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/_build/libnh_oracle.so``.

    ``-ffp-contract=off`` keeps every multiply and add separately rounded on
    both x86 and Arm hosts, so results do not depend on FMA contraction.
    """
    os.makedirs(_BUILD, exist_ok=True)
    src = [os.path.join(_HERE, f) for f in ("nh_oracle.c", "nh_oracle2d.c", "nh_oracle_dg.c")]
    src = [s for s in src if os.path.exists(s)]
    out = os.path.join(_BUILD, "libnh_oracle.so")
    hdrs = [os.path.join(_HERE, h) for h in ("nh_oracle.h", "nh_oracle2d.h", "nh_oracle_dg.h")
            if os.path.exists(os.path.join(_HERE, h))]
    newest = max(os.path.getmtime(s) for s in src + hdrs)
    if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
               "-Wall", "-Wno-unused-variable", "-Wno-unused-but-set-variable",
               *src, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


class _Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("bc", C.c_int), ("dx", C.c_double), ("xl", C.c_double),
        ("g", C.c_double), ("rho", C.c_double), ("limiter", C.c_int),
        ("slide", C.c_int), ("A", C.c_double), ("L", C.c_double), ("xc0", C.c_double),
        ("s0", C.c_double), ("t0", C.c_double), ("t2", C.c_double),
        ("crit", C.c_int), ("knh", C.c_double), ("enlarge", C.c_int),
        ("first_step_global", C.c_int),
        ("solver", C.c_int), ("rtol", C.c_double), ("max_iter", C.c_int), ("guess", C.c_int),
    ]


class StepInfo(C.Structure):
    _fields_ = [("n_active", C.c_int), ("iters", C.c_int), ("solver_used", C.c_int),
                ("status", C.c_int), ("rel_res", C.c_double), ("min_gamma", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


@dataclass
class Params:
    """Problem description for one 1D member (mirrors ``or_params``)."""
    nx: int
    dx: float
    xl: float = 0.0
    bc: int = BC_WALL
    g: float = 9.81
    rho: float = 1000.0
    limiter: int = LIM_CENTRAL
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
    solver: int = SOLVER_AUTO
    rtol: float = 1e-13
    max_iter: int = 100000
    guess: int = GUESS_PREV

    def c(self) -> _Params:
        return _Params(**{f.name: getattr(self, f.name) for f in fields(self)})


_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_U8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_PP = C.POINTER(_Params)


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = C.CDLL(build())
            L.or_bottom.argtypes = [_PP, _D, C.c_int, C.c_double, _D]
            L.or_rhs.argtypes = [_PP, _D, C.c_double, _D, _D, _D, _D, _D, _D]
            L.or_predict.argtypes = [_PP, _D, C.c_double, C.c_double, _D, _D, _D, _D, _D, _D]
            L.or_criterion.argtypes = [_PP, _D, C.c_double, _D, _D, _D, _D]
            L.or_mask.argtypes = [_PP, _D, C.c_double, C.c_long, _D, _D, _D, _U8]
            L.or_mask.restype = C.c_int
            L.or_assemble.argtypes = [_PP, _D, C.c_double, C.c_double, _D, _D, _D, _D, _D, _D]
            L.or_apply.argtypes = [_PP, _U8, _D, _D, _D, _D]
            L.or_solve.argtypes = [_PP, _U8, _D, _D, _D, _D, C.POINTER(StepInfo)]
            L.or_solve.restype = C.c_int
            L.or_correct.argtypes = [_PP, _D, C.c_double, C.c_double, _U8, _D, _D, _D, _D, _D, _D, _D]
            L.or_step.argtypes = [_PP, _D, C.c_double, C.c_long, C.c_double, _D, _D, _D, _D,
                                  C.c_void_p, C.POINTER(StepInfo)]
            L.or_step.restype = C.c_int
            L.or_run.argtypes = [_PP, _D, C.c_double, C.c_long, C.c_double, C.c_long,
                                 _D, _D, _D, _D, C.POINTER(StepInfo),
                                 C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
            L.or_run.restype = C.c_int
            if hasattr(L, "or2_step"):
                from . import oracle2d  # noqa: F401  (binds the 2D entry points)
                oracle2d._bind(L)
            if hasattr(L, "or_dg_step"):
                from . import oracle_dg  # noqa: F401  (binds the DG / LDG entry points)
                oracle_dg._bind(L)
            _LIB = L
    return _LIB


def _f(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------- 1D wrappers

def bottom(p: Params, d0, i: int, t: float) -> np.ndarray:
    out = np.zeros(6)
    lib().or_bottom(C.byref(p.c()), _f(d0), int(i), float(t), out)
    return out


def bottom_all(p: Params, d0, t: float) -> np.ndarray:
    """(6, nx): d, d_x, d_xx, d_t, d_xt, d_tt at every cell centre."""
    d0 = _f(d0)
    return np.stack([bottom(p, d0, i, t) for i in range(p.nx)], axis=1)


def rhs(p: Params, d0, t, h, hu, hw):
    n = p.nx
    out = [np.zeros(n) for _ in range(3)]
    lib().or_rhs(C.byref(p.c()), _f(d0), float(t), _f(h), _f(hu), _f(hw), *out)
    return out


def predict(p: Params, d0, t, dt, h, hu, hw):
    n = p.nx
    out = [np.zeros(n) for _ in range(3)]
    lib().or_predict(C.byref(p.c()), _f(d0), float(t), float(dt), _f(h), _f(hu), _f(hw), *out)
    return out


def criterion(p: Params, d0, t, ht, hut, hwt):
    c = np.zeros(p.nx)
    lib().or_criterion(C.byref(p.c()), _f(d0), float(t), _f(ht), _f(hut), _f(hwt), c)
    return c


def mask(p: Params, d0, t, step, ht, hut, hwt):
    m = np.zeros(p.nx, dtype=np.uint8)
    lib().or_mask(C.byref(p.c()), _f(d0), float(t), int(step), _f(ht), _f(hut), _f(hwt), m)
    return m


def assemble(p: Params, d0, t1, dt, ht, hut, hwt):
    n = p.nx
    Kf, gam, R = np.zeros(n + 1), np.zeros(n), np.zeros(n)
    lib().or_assemble(C.byref(p.c()), _f(d0), float(t1), float(dt), _f(ht), _f(hut), _f(hwt),
                      Kf, gam, R)
    return Kf, gam, R


def apply(p: Params, m, Kf, gam, x):
    y = np.zeros(p.nx)
    lib().or_apply(C.byref(p.c()), np.ascontiguousarray(m, dtype=np.uint8), _f(Kf), _f(gam), _f(x), y)
    return y


def solve(p: Params, m, Kf, gam, R, q0=None):
    q = np.zeros(p.nx) if q0 is None else _f(q0).copy()
    info = StepInfo()
    st = lib().or_solve(C.byref(p.c()), np.ascontiguousarray(m, dtype=np.uint8), _f(Kf), _f(gam),
                        _f(R), q, C.byref(info))
    return q, st, info.as_dict()


def correct(p: Params, d0, t1, dt, m, q, ht, hut, hwt):
    n = p.nx
    out = [np.zeros(n) for _ in range(3)]
    lib().or_correct(C.byref(p.c()), _f(d0), float(t1), float(dt),
                     np.ascontiguousarray(m, dtype=np.uint8), _f(q), _f(ht), _f(hut), _f(hwt), *out)
    return out


@dataclass
class State:
    h: np.ndarray
    hu: np.ndarray
    hw: np.ndarray
    q: np.ndarray = field(default=None)

    def __post_init__(self):
        self.h = _f(self.h).copy()
        self.hu = _f(self.hu).copy()
        self.hw = _f(self.hw).copy()
        self.q = np.zeros_like(self.h) if self.q is None else _f(self.q).copy()

    def copy(self):
        return State(self.h, self.hu, self.hw, self.q)


def step(p: Params, d0, t, step_index, dt, s: State, want_mask=False):
    """One step in place on ``s``; returns (status, info dict[, mask])."""
    info = StepInfo()
    m = np.zeros(p.nx, dtype=np.uint8) if want_mask else None
    st = lib().or_step(C.byref(p.c()), _f(d0), float(t), int(step_index), float(dt),
                       s.h, s.hu, s.hw, s.q, m.ctypes.data if want_mask else None, C.byref(info))
    return (st, info.as_dict(), m) if want_mask else (st, info.as_dict())


def run(p: Params, d0, t_start, step0, dt, n_steps, s: State):
    """``n_steps`` steps in place; returns (status, last info, total iters, total active)."""
    info = StepInfo()
    ti, ta = C.c_longlong(0), C.c_longlong(0)
    st = lib().or_run(C.byref(p.c()), _f(d0), float(t_start), int(step0), float(dt), int(n_steps),
                      s.h, s.hu, s.hw, s.q, C.byref(info), C.byref(ti), C.byref(ta))
    return st, info.as_dict(), ti.value, ta.value
