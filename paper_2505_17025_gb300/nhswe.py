"""Thin ctypes binding of the C ABI in ``include/nhswe.h`` and ``include/nhswe_cnn.h``.

Argument marshalling only: every step of the method runs in the CUDA library.
The functions keep the C names (``nh_create_grid``, ``nh_step``, ...); the
``Grid`` class adds the one thing Python must supply -- device memory for the
workspace and the CUDA stream, both taken from PyTorch.

``load()`` raises ``RuntimeError`` if the library is missing or no CUDA device
is present: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

# enums (mirror include/nhswe.h)
NH_OK, NH_ERR_ARG, NH_ERR_CUDA, NH_ERR_NOT_CONVERGED, NH_ERR_NONFINITE, NH_ERR_TIMEOUT, NH_ERR_STATE = range(7)
NH_BC_WALL, NH_BC_PERIODIC = 0, 1
NH_FP64, NH_MIXED, NH_MIXED_FP64_SOLVE = 0, 1, 2
NH_LIM_NONE, NH_LIM_CENTRAL, NH_LIM_MINMOD, NH_LIM_MC = range(4)
(NH_CRIT_GLOBAL, NH_CRIT_HYDROSTATIC, NH_CRIT_ETA_D, NH_CRIT_ETA_X, NH_CRIT_U, NH_CRIT_U_X,
 NH_CRIT_W, NH_CRIT_W_X) = range(8)
NH_SOLVER_AUTO, NH_SOLVER_CG, NH_SOLVER_BICGSTAB = range(3)
NH_GUESS_ZERO, NH_GUESS_PREV, NH_GUESS_CNN = 0, 1, 2
NH_PRECOND_NONE, NH_PRECOND_LINE, NH_PRECOND_MG = 0, 1, 2
NH_SLIDE_NONE, NH_SLIDE_GAUSS_LNCOSH, NH_SLIDE_PLATE_EXP, NH_SLIDE_QUARTIC = 0, 1, 2, 3

# every exported symbol of the ABI (checked by the CPU test suite)
EXPORTS = ("nh_workspace_bytes", "nh_create_grid", "nh_set_bottom_motion", "nh_set_criterion",
           "nh_set_solver", "nh_set_preconditioner", "nh_set_state", "nh_put_state", "nh_get_state",
           "nh_get_mask", "nh_step", "nh_run", "nh_set_profiling", "nh_get_profile", "nh_destroy",
           "nh_status_string", "nh_predict_static", "nh_workspace_bytes_ensemble", "nh_create_ensemble",
           "nh_set_run_mode", "nh_set_tile", "nh_set_wait_budget", "nh_cnn_forward", "nh_cnn_workspace_bytes",
           "nh_cnn_loss_grad", "nh_cnn_adam", "nh_cnn_attach_bytes", "nh_cnn_attach",
           "nh_cnn_set_params", "nh_cnn_record", "nh_cnn_harvest", "nh_cnn_choices",
           "nh2d_workspace_bytes", "nh2d_create", "nh2d_set_bottom_motion", "nh2d_set_criterion",
           "nh2d_set_solver", "nh2d_set_state", "nh2d_get_state", "nh2d_get_mask", "nh2d_step",
           "nh2d_run", "nh2d_destroy", "nh2d_ensemble_workspace_bytes", "nh2d_create_ensemble", "nh2d_members",
           "nh2d_set_member_bottom_motion", "nh2d_set_graphs", "nh2d_set_member_state", "nh2d_get_member_state",
           "nh2d_get_member_mask", "nh2d_get_member_info", "nh2d_graph_runs", "nh2d_set_precision",
           "nh2d_set_wait_budget", "nh2d_set_preconditioner", "nh2d_set_profiling", "nh2d_get_profile",
           "nh2d_put_member_state", "nh2d_set_tile",
           "nh_dg_workspace_bytes", "nh_dg_create", "nh_dg_set_bottom_motion", "nh_dg_set_criterion",
           "nh_dg_set_check", "nh_dg_set_state", "nh_dg_get_state", "nh_dg_get_mask", "nh_dg_step",
           "nh_dg_run", "nh_dg_set_profiling", "nh_dg_get_profile", "nh_dg_destroy")
NH_CNN_PARAMS = 9328
NH_CNN_IN = 16
NH_STATIC_MAX_CELLS = 262144
KERNEL_CLASSES_2D = ("kin", "depth", "stage", "marks", "dilate", "compact", "assemble", "mass", "solve_init",
                     "solve", "summary", "clear", "correct")
KERNEL_CLASSES_DG = ("kinematics", "predict", "mark", "compact", "local", "form", "reduce", "back", "correct",
                     "finish")
KERNEL_CLASSES = ("kinematics", "predict", "compact", "assemble", "solve_init", "precond", "pcg_a",
                  "pcg_b", "cg_a", "cg_b", "bi_1", "bi_2", "bi_3", "summary", "clear", "correct",
                  "pcg_loop", "cnn")


class nh_grid_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("nbatch", C.c_int), ("bc", C.c_int),
                ("precision", C.c_int), ("limiter", C.c_int), ("dx", C.c_double),
                ("x0", C.c_double), ("g", C.c_double), ("rho", C.c_double)]


class nh_slide_desc(C.Structure):
    _fields_ = [("shape", C.c_int), ("A", C.c_double), ("L", C.c_double), ("xc0", C.c_double),
                ("s0", C.c_double), ("t0", C.c_double), ("t2", C.c_double)]


class nh_step_info(C.Structure):
    _fields_ = [("step", C.c_longlong), ("t", C.c_double), ("n_active", C.c_longlong),
                ("n_active_max", C.c_int), ("iters", C.c_int), ("ir_passes", C.c_int),
                ("solver", C.c_int), ("status", C.c_int), ("rel_res", C.c_double),
                ("min_gamma", C.c_double), ("mass", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class nh_grid2d_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("bc_x", C.c_int), ("bc_y", C.c_int),
                ("limiter", C.c_int), ("dx", C.c_double), ("dy", C.c_double), ("x0", C.c_double),
                ("y0", C.c_double), ("g", C.c_double), ("rho", C.c_double)]


class nh_slide2d_desc(C.Structure):
    _fields_ = [("shape", C.c_int), ("A", C.c_double), ("Lx", C.c_double), ("Ly", C.c_double),
                ("xc0", C.c_double), ("yc0", C.c_double), ("s0", C.c_double), ("t0", C.c_double)]


class nh_dg_desc(C.Structure):
    _fields_ = [("ne", C.c_int), ("nbatch", C.c_int), ("dx", C.c_double), ("x0", C.c_double),
                ("g", C.c_double), ("rho", C.c_double), ("c11", C.c_double)]


class nh_run_info(C.Structure):
    _fields_ = [("steps", C.c_longlong), ("iters_total", C.c_longlong),
                ("active_total", C.c_longlong), ("last", nh_step_info)]


_LIB = None
_LOCK = threading.Lock()
_D = C.POINTER(C.c_double)


def library_path() -> str:
    return _build.LIB


def load_symbols_only(path: str | None = None):
    """Open the shared library without touching a GPU (symbol checks)."""
    return C.CDLL(path or _build.build())


def load():
    """Build (if needed) and load the CUDA library; raises without a GPU."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2505_17025_gb300 needs a CUDA GPU; no CPU fallback exists")
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library missing: {path}")
        L = C.CDLL(path)
        L.nh_workspace_bytes.argtypes = [C.POINTER(nh_grid_desc)]
        L.nh_workspace_bytes.restype = C.c_size_t
        L.nh_create_grid.argtypes = [C.POINTER(nh_grid_desc), _D, C.c_void_p, C.c_size_t, C.c_void_p,
                                     C.POINTER(C.c_void_p)]
        L.nh_workspace_bytes_ensemble.argtypes = [C.POINTER(nh_grid_desc), C.POINTER(C.c_int)]
        L.nh_workspace_bytes_ensemble.restype = C.c_size_t
        L.nh_create_ensemble.argtypes = [C.POINTER(nh_grid_desc), C.POINTER(C.c_int), _D, C.c_void_p,
                                         C.c_size_t, C.c_void_p, C.POINTER(C.c_void_p)]
        L.nh_set_bottom_motion.argtypes = [C.c_void_p, C.POINTER(nh_slide_desc)]
        L.nh_set_criterion.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_int]
        L.nh_set_solver.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int,
                                    C.c_double]
        L.nh_set_preconditioner.argtypes = [C.c_void_p, C.c_int]
        L.nh_set_state.argtypes = [C.c_void_p, _D, _D, _D, C.c_double]
        L.nh_get_state.argtypes = [C.c_void_p, _D, _D, _D, _D]
        L.nh_put_state.argtypes = [C.c_void_p, _D, _D, _D]
        L.nh_set_profiling.argtypes = [C.c_void_p, C.c_int]
        L.nh_set_run_mode.argtypes = [C.c_void_p, C.c_int]
        L.nh_set_wait_budget.argtypes = [C.c_void_p, C.c_longlong]
        L.nh2d_set_wait_budget.argtypes = [C.c_void_p, C.c_longlong]
        L.nh2d_set_preconditioner.argtypes = [C.c_void_p, C.c_int]
        L.nh2d_set_profiling.argtypes = [C.c_void_p, C.c_int]
        L.nh2d_put_member_state.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.nh2d_put_member_state.restype = C.c_int
        L.nh2d_set_tile.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int)]
        L.nh2d_set_tile.restype = C.c_int
        L.nh2d_get_profile.argtypes = [C.c_void_p, _D, C.POINTER(C.c_longlong)]
        L.nh_set_tile.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int)]
        L.nh_get_profile.argtypes = [C.c_void_p, _D, C.POINTER(C.c_longlong)]
        L.nh_get_mask.argtypes = [C.c_void_p, C.POINTER(C.c_ubyte), C.POINTER(C.c_int), _D]
        L.nh_step.argtypes = [C.c_void_p, C.c_double, C.POINTER(nh_step_info)]
        L.nh_run.argtypes = [C.c_void_p, C.c_double, C.c_longlong, C.POINTER(nh_run_info)]
        L.nh_destroy.argtypes = [C.c_void_p]
        L.nh_destroy.restype = None
        L.nh_predict_static.argtypes = [C.c_void_p] * 7 + [C.c_int, C.c_double, C.c_double, C.c_int,
                                                           C.c_int, C.c_double,
                                                           C.POINTER(nh_slide_desc), C.c_double,
                                                           C.c_double, _D, C.c_void_p]
        L.nh_predict_static.restype = C.c_int
        vp, sz = C.c_void_p, C.c_size_t
        L.nh_cnn_forward.argtypes = [vp, vp, C.c_int, C.c_int, vp, vp, C.c_float, vp, vp]
        L.nh_cnn_workspace_bytes.argtypes = [C.c_int, C.c_int]
        L.nh_cnn_workspace_bytes.restype = sz
        L.nh_cnn_loss_grad.argtypes = [vp, vp, C.c_int, C.c_int, vp, vp, vp, C.c_longlong, vp, _D, vp, sz, vp]
        L.nh_cnn_adam.argtypes = [vp, vp, vp, vp, C.c_int, C.c_float, vp]
        L.nh_cnn_attach_bytes.argtypes = [vp]
        L.nh_cnn_attach_bytes.restype = sz
        L.nh_cnn_attach.argtypes = [vp, vp, sz]
        L.nh_cnn_set_params.argtypes = [vp, vp]
        L.nh_cnn_record.argtypes = [vp, C.c_int]
        L.nh_cnn_harvest.argtypes = [vp, vp, vp, vp, _D, C.POINTER(C.c_int)]
        L.nh_cnn_choices.argtypes = [vp, C.POINTER(C.c_longlong)]
        L.nh2d_workspace_bytes.argtypes = [C.POINTER(nh_grid2d_desc)]
        L.nh2d_workspace_bytes.restype = sz
        L.nh2d_create.argtypes = [C.POINTER(nh_grid2d_desc), _D, vp, sz, vp, C.POINTER(C.c_void_p)]
        L.nh2d_set_bottom_motion.argtypes = [vp, C.POINTER(nh_slide2d_desc)]
        L.nh2d_set_criterion.argtypes = [vp, C.c_int, C.c_double, C.c_int, C.c_int]
        L.nh2d_set_solver.argtypes = [vp, C.c_double, C.c_int, C.c_int]
        L.nh2d_set_state.argtypes = [vp, _D, _D, _D, _D, C.c_double]
        L.nh2d_get_state.argtypes = [vp, _D, _D, _D, _D, _D]
        L.nh2d_get_mask.argtypes = [vp, C.POINTER(C.c_ubyte)]
        L.nh2d_step.argtypes = [vp, C.c_double, C.POINTER(nh_step_info)]
        L.nh2d_run.argtypes = [vp, C.c_double, C.c_longlong, C.POINTER(nh_run_info)]
        L.nh2d_destroy.argtypes = [vp]
        L.nh2d_destroy.restype = None
        L.nh2d_ensemble_workspace_bytes.argtypes = [C.c_int, C.POINTER(nh_grid2d_desc)]
        L.nh2d_ensemble_workspace_bytes.restype = sz
        L.nh2d_create_ensemble.argtypes = [C.c_int, C.POINTER(nh_grid2d_desc), C.POINTER(_D), vp, sz, vp,
                                           C.POINTER(C.c_void_p)]
        L.nh2d_members.argtypes = [vp]
        L.nh2d_members.restype = C.c_int
        L.nh2d_set_member_bottom_motion.argtypes = [vp, C.c_int, C.POINTER(nh_slide2d_desc)]
        L.nh2d_set_graphs.argtypes = [vp, C.c_int]
        L.nh2d_set_member_state.argtypes = [vp, C.c_int, _D, _D, _D, _D, C.c_double]
        L.nh2d_get_member_state.argtypes = [vp, C.c_int, _D, _D, _D, _D, _D]
        L.nh2d_get_member_mask.argtypes = [vp, C.c_int, C.POINTER(C.c_ubyte)]
        L.nh2d_get_member_info.argtypes = [vp, C.c_int, C.POINTER(nh_step_info)]
        L.nh2d_set_precision.argtypes = [vp, C.c_int]
        L.nh2d_graph_runs.argtypes = [vp]
        L.nh2d_graph_runs.restype = C.c_longlong
        for f in ("nh2d_create", "nh2d_set_bottom_motion", "nh2d_set_criterion", "nh2d_set_solver",
                  "nh2d_set_state", "nh2d_get_state", "nh2d_get_mask", "nh2d_step", "nh2d_run",
                  "nh2d_create_ensemble", "nh2d_set_member_bottom_motion", "nh2d_set_graphs",
                  "nh2d_set_member_state", "nh2d_get_member_state", "nh2d_get_member_mask",
                  "nh2d_get_member_info", "nh2d_set_precision"):
            getattr(L, f).restype = C.c_int
        L.nh_dg_workspace_bytes.argtypes = [C.POINTER(nh_dg_desc)]
        L.nh_dg_workspace_bytes.restype = sz
        L.nh_dg_create.argtypes = [C.POINTER(nh_dg_desc), _D, vp, sz, vp, C.POINTER(C.c_void_p)]
        L.nh_dg_set_bottom_motion.argtypes = [vp, C.POINTER(nh_slide_desc)]
        L.nh_dg_set_criterion.argtypes = [vp, C.c_int, C.c_double, C.c_int, C.c_int]
        L.nh_dg_set_check.argtypes = [vp, C.c_int]
        L.nh_dg_set_state.argtypes = [vp, _D, _D, _D, C.c_double]
        L.nh_dg_get_state.argtypes = [vp, _D, _D, _D, _D]
        L.nh_dg_get_mask.argtypes = [vp, C.POINTER(C.c_ubyte), _D]
        L.nh_dg_step.argtypes = [vp, C.c_double, C.POINTER(nh_step_info)]
        L.nh_dg_run.argtypes = [vp, C.c_double, C.c_longlong, C.POINTER(nh_run_info)]
        L.nh_dg_set_profiling.argtypes = [vp, C.c_int]
        L.nh_dg_get_profile.argtypes = [vp, _D, C.POINTER(C.c_longlong)]
        L.nh_dg_destroy.argtypes = [vp]
        L.nh_dg_destroy.restype = None
        for f in ("nh_dg_create", "nh_dg_set_bottom_motion", "nh_dg_set_criterion", "nh_dg_set_check",
                  "nh_dg_set_state", "nh_dg_get_state", "nh_dg_get_mask", "nh_dg_step", "nh_dg_run",
                  "nh_dg_set_profiling", "nh_dg_get_profile"):
            getattr(L, f).restype = C.c_int
        L.nh_status_string.argtypes = [C.c_int]
        L.nh_status_string.restype = C.c_char_p
        for f in ("nh_create_grid", "nh_create_ensemble", "nh_set_bottom_motion", "nh_set_criterion", "nh_set_solver",
                  "nh_set_preconditioner", "nh_put_state", "nh_set_profiling", "nh_get_profile",
                  "nh_set_run_mode", "nh_set_tile", "nh_set_wait_budget", "nh2d_set_wait_budget",
                  "nh2d_set_preconditioner", "nh2d_set_profiling", "nh2d_get_profile", "nh_set_state", "nh_get_state", "nh_get_mask", "nh_step", "nh_run",
                  "nh_cnn_forward", "nh_cnn_loss_grad", "nh_cnn_adam", "nh_cnn_attach",
                  "nh_cnn_set_params", "nh_cnn_record", "nh_cnn_harvest", "nh_cnn_choices"):
            getattr(L, f).restype = C.c_int
        _LIB = L
        return L


class NHError(RuntimeError):
    def __init__(self, status, where):
        msg = load().nh_status_string(status).decode()
        super().__init__(f"{where}: {msg}")
        self.status = status


def _check(status, where):
    if status != NH_OK:
        raise NHError(status, where)
    return status


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


class Grid:
    """A batch of 1D members on one GPU, stepping through the C ABI.

    ``nx`` is one cell count for every member, or a sequence of per-member
    counts (an uneven ensemble, ``nh_create_ensemble``).  ``d0`` is (nbatch, nx),
    (nx,) or, for an ensemble, a sequence of per-member arrays.  The workspace
    is a ``torch.uint8`` tensor on the current CUDA device and the stream is
    ``torch.cuda.current_stream()`` unless one is given.
    """

    def __init__(self, nx, dx, d0, nbatch=1, x0=0.0, bc=NH_BC_WALL, precision=NH_FP64,
                 limiter=NH_LIM_CENTRAL, g=9.81, rho=1000.0, stream=None):
        import torch
        self.L = load()
        if np.ndim(nx) == 0:
            self.nxs = [int(nx)] * int(nbatch)
        else:
            self.nxs = [int(v) for v in nx]
            nbatch = len(self.nxs)
        self.uneven = len(set(self.nxs)) > 1 or np.ndim(nx) > 0
        self.nb = int(nbatch)
        self.nx = max(self.nxs)
        self.offsets = np.concatenate([[0], np.cumsum(self.nxs)]).astype(np.int64)
        self.ncells = int(self.offsets[-1])
        self.desc = nh_grid_desc(1, self.nx, self.nb, int(bc), int(precision), int(limiter),
                                 float(dx), float(x0), float(g), float(rho))
        nxa = (C.c_int * self.nb)(*self.nxs)
        nbytes = self.L.nh_workspace_bytes_ensemble(C.byref(self.desc), nxa)
        if nbytes == 0:
            raise NHError(NH_ERR_ARG, "nh_workspace_bytes_ensemble")
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.ws.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        d0c = self._concat(d0)
        h = C.c_void_p()
        _check(self.L.nh_create_ensemble(C.byref(self.desc), nxa, _dptr(d0c), C.c_void_p(self._ws_ptr),
                                         C.c_size_t(nbytes), C.c_void_p(self.stream.cuda_stream),
                                         C.byref(h)), "nh_create_ensemble")
        self.h = h
        self.workspace_bytes = nbytes

    def _concat(self, a):
        """Host layout: members concatenated (FP64, contiguous)."""
        if isinstance(a, (list, tuple)) and len(a) == self.nb and np.ndim(a[0]) == 1:
            out = np.concatenate([np.asarray(v, dtype=np.float64).reshape(-1) for v in a])
        else:
            arr = np.asarray(a, dtype=np.float64)
            if arr.ndim == 1 and arr.size == self.nx and not self.uneven:
                arr = np.broadcast_to(arr, (self.nb, self.nx))
            out = np.ascontiguousarray(arr).reshape(-1)
        if out.size != self.ncells:
            raise ValueError(f"expected {self.ncells} values, got {out.size}")
        return np.ascontiguousarray(out)

    def _split(self, a):
        if not self.uneven:
            return a.reshape(self.nb, self.nx)
        return [a[self.offsets[b]:self.offsets[b + 1]] for b in range(self.nb)]

    # -- configuration
    def set_bottom_motion(self, slides):
        """slides: list of dicts (shape, A, L, xc0, s0, t0[, t2]) per member, or None."""
        if slides is None:
            _check(self.L.nh_set_bottom_motion(self.h, None), "nh_set_bottom_motion")
            return
        arr = (nh_slide_desc * self.nb)()
        for b, s in enumerate(slides):
            arr[b] = nh_slide_desc(int(s.get("shape", NH_SLIDE_GAUSS_LNCOSH)), float(s["A"]),
                                   float(s["L"]), float(s["xc0"]), float(s["s0"]), float(s["t0"]),
                                   float(s.get("t2", 0.0)))
        _check(self.L.nh_set_bottom_motion(self.h, arr), "nh_set_bottom_motion")

    def set_criterion(self, kind, k_nh=1e-3, enlarge=1, first_step_global=False):
        _check(self.L.nh_set_criterion(self.h, int(kind), float(k_nh), int(enlarge),
                                       int(bool(first_step_global))), "nh_set_criterion")

    def set_solver(self, kind=NH_SOLVER_AUTO, rtol=1e-12, max_iter=20000, guess=NH_GUESS_PREV,
                   ir_max=30, inner_rtol=1e-5):
        _check(self.L.nh_set_solver(self.h, int(kind), float(rtol), int(max_iter), int(guess),
                                    int(ir_max), float(inner_rtol)), "nh_set_solver")

    def set_preconditioner(self, kind=NH_PRECOND_LINE):
        _check(self.L.nh_set_preconditioner(self.h, int(kind)), "nh_set_preconditioner")

    # -- state
    def set_state(self, h, hu, hw, t=0.0):
        h, hu, hw = self._concat(h), self._concat(hu), self._concat(hw)
        _check(self.L.nh_set_state(self.h, _dptr(h), _dptr(hu), _dptr(hw), float(t)), "nh_set_state")

    def set_state_ptr(self, h_ptr, hu_ptr, hw_ptr, t=0.0):
        """Same as set_state from raw host addresses (e.g. pinned tensors)."""
        _check(self.L.nh_set_state(self.h, C.cast(C.c_void_p(h_ptr), _D), C.cast(C.c_void_p(hu_ptr), _D),
                                   C.cast(C.c_void_p(hw_ptr), _D), float(t)), "nh_set_state")

    def put_state_ptr(self, h_ptr, hu_ptr, hw_ptr):
        """Replace the state from raw host addresses, keeping time and warm start."""
        cast = lambda p: C.cast(C.c_void_p(p), _D)
        _check(self.L.nh_put_state(self.h, cast(h_ptr), cast(hu_ptr), cast(hw_ptr)), "nh_put_state")

    def set_tile(self, tile=0):
        """Force the predictor tile (128/256/512) or, with 0, read the autotuned one."""
        out = C.c_int(0)
        _check(self.L.nh_set_tile(self.h, int(tile), C.byref(out)), "nh_set_tile")
        return out.value

    def set_run_mode(self, use_graphs=True):
        _check(self.L.nh_set_run_mode(self.h, int(bool(use_graphs))), "nh_set_run_mode")

    def set_wait_budget(self, cycles=0):
        """Spin limit of the solver's grid barrier in SM clock cycles (0: about one second)."""
        _check(self.L.nh_set_wait_budget(self.h, int(cycles)), "nh_set_wait_budget")

    def set_profiling(self, enable=True):
        _check(self.L.nh_set_profiling(self.h, int(bool(enable))), "nh_set_profiling")

    def get_profile(self):
        ms = np.zeros(len(KERNEL_CLASSES))
        n = np.zeros(len(KERNEL_CLASSES), dtype=np.int64)
        _check(self.L.nh_get_profile(self.h, _dptr(ms), n.ctypes.data_as(C.POINTER(C.c_longlong))),
               "nh_get_profile")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_CLASSES)}

    def get_state(self):
        n = self.ncells
        h, hu, hw, p = (np.empty(n) for _ in range(4))
        _check(self.L.nh_get_state(self.h, _dptr(h), _dptr(hu), _dptr(hw), _dptr(p)), "nh_get_state")
        return self._split(h), self._split(hu), self._split(hw), self._split(p)

    def get_state_ptr(self, h_ptr, hu_ptr=0, hw_ptr=0, p_ptr=0):
        cast = lambda p: C.cast(C.c_void_p(p), _D) if p else None
        _check(self.L.nh_get_state(self.h, cast(h_ptr), cast(hu_ptr), cast(hw_ptr), cast(p_ptr)),
               "nh_get_state")

    def get_mask(self):
        m = np.empty(self.ncells, dtype=np.uint8)
        it = np.empty(self.nb, dtype=np.int32)
        rr = np.empty(self.nb)
        _check(self.L.nh_get_mask(self.h, m.ctypes.data_as(C.POINTER(C.c_ubyte)),
                                  it.ctypes.data_as(C.POINTER(C.c_int)), _dptr(rr)), "nh_get_mask")
        return self._split(m), it, rr

    # -- learned guess (nhswe_cnn.h)
    def cnn_attach(self):
        """Allocate the guess buffers (a torch tensor kept by the Grid) and attach them."""
        import torch
        n = self.L.nh_cnn_attach_bytes(self.h)
        self.cnn_ws = torch.empty(n + 256, dtype=torch.uint8, device="cuda")
        ptr = (self.cnn_ws.data_ptr() + 255) // 256 * 256
        _check(self.L.nh_cnn_attach(self.h, C.c_void_p(ptr), C.c_size_t(n)), "nh_cnn_attach")

    def cnn_set_params(self, params):
        """params: CUDA float32 tensor of NH_CNN_PARAMS values (copied)."""
        _params_check(params)
        _check(self.L.nh_cnn_set_params(self.h, C.c_void_p(params.data_ptr())), "nh_cnn_set_params")

    def cnn_record(self, record=True):
        _check(self.L.nh_cnn_record(self.h, int(bool(record))), "nh_cnn_record")

    def cnn_harvest(self):
        """(features [nb, pitch, 16] bf16, target [nb, pitch] f32, mask [nb, pitch] u8, scale) of
        the last step, as CUDA tensors."""
        import torch
        pitch = C.c_int(0)
        scale = C.c_double(0.0)
        probe = (self.nx + 511) // 512 * 512
        feat = torch.empty((self.nb, probe, NH_CNN_IN), dtype=torch.bfloat16, device="cuda")
        target = torch.empty((self.nb, probe), dtype=torch.float32, device="cuda")
        mask = torch.empty((self.nb, probe), dtype=torch.uint8, device="cuda")
        _check(self.L.nh_cnn_harvest(self.h, C.c_void_p(feat.data_ptr()), C.c_void_p(target.data_ptr()),
                                     C.c_void_p(mask.data_ptr()), C.byref(scale), C.byref(pitch)),
               "nh_cnn_harvest")
        if pitch.value != probe:
            raise RuntimeError(f"row pitch {pitch.value} != {probe}")
        return feat, target, mask, scale.value

    def cnn_choices(self):
        """{previous, extrapolation, network}: solves started from each."""
        c = (C.c_longlong * 3)()
        _check(self.L.nh_cnn_choices(self.h, c), "nh_cnn_choices")
        return {"previous": c[0], "extrapolation": c[1], "network": c[2]}

    def nx_device(self):
        import torch
        return torch.tensor(self.nxs, dtype=torch.int32, device="cuda")

    # -- stepping
    def step(self, dt, check=True):
        info = nh_step_info()
        st = self.L.nh_step(self.h, float(dt), C.byref(info))
        if check:
            _check(st, "nh_step")
        return st, info.as_dict()

    def run(self, dt, n_steps, check=True):
        info = nh_run_info()
        st = self.L.nh_run(self.h, float(dt), int(n_steps), C.byref(info))
        if check:
            _check(st, "nh_run")
        return st, {"steps": info.steps, "iters_total": info.iters_total,
                    "active_total": info.active_total, "last": info.last.as_dict()}

    def close(self):
        if getattr(self, "h", None):
            self.L.nh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------ network calls (nhswe_cnn.h)

def _params_check(t):
    import torch
    if t.dtype != torch.float32 or not t.is_cuda or t.numel() != NH_CNN_PARAMS or not t.is_contiguous():
        raise ValueError("params must be a contiguous CUDA float32 tensor of NH_CNN_PARAMS values")


def _stream_ptr():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def nh_cnn_forward(feat, nx_dev, params, out_scale=1.0, status=None):
    """feat: CUDA bf16 [nb, pitch, 16]; nx_dev: CUDA int32 [nb]; returns y [nb, pitch] float32
    (entries at or beyond a member's cell count are 0)."""
    import torch
    L = load()
    _params_check(params)
    nb, pitch, ch = feat.shape
    if ch != NH_CNN_IN or feat.dtype != torch.bfloat16 or not feat.is_contiguous():
        raise ValueError("feat must be a contiguous bf16 tensor [nb, pitch, 16]")
    y = torch.zeros((nb, pitch), dtype=torch.float32, device=feat.device)
    sp = C.c_void_p(status.data_ptr()) if status is not None else None
    _check(L.nh_cnn_forward(C.c_void_p(feat.data_ptr()), C.c_void_p(nx_dev.data_ptr()), nb, pitch,
                            C.c_void_p(params.data_ptr()), C.c_void_p(y.data_ptr()), float(out_scale), sp,
                            _stream_ptr()), "nh_cnn_forward")
    return y


class CnnWorkspace:
    """Scratch of nh_cnn_loss_grad for nb x pitch cells (a torch tensor)."""

    def __init__(self, nb, pitch):
        import torch
        L = load()
        self.nbytes = L.nh_cnn_workspace_bytes(int(nb), int(pitch))
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device="cuda")
        self.ptr = (self.buf.data_ptr() + 255) // 256 * 256


def nh_cnn_loss_grad(feat, nx_dev, params, target, mask, grad, ws=None):
    """Loss (float) and gradient (written into ``grad``, CUDA float32 [NH_CNN_PARAMS])."""
    import torch
    L = load()
    _params_check(params)
    _params_check(grad)
    nb, pitch, _ = feat.shape
    ws = ws or CnnWorkspace(nb, pitch)
    # counted cells: mask set and inside the member (cells at or beyond nx are ignored)
    inside = torch.arange(pitch, device=mask.device)[None, :] < nx_dev.to(torch.int64)[:, None]
    count = int(((mask != 0) & inside).count_nonzero().item())
    loss = C.c_double(0.0)
    _check(L.nh_cnn_loss_grad(C.c_void_p(feat.data_ptr()), C.c_void_p(nx_dev.data_ptr()), nb, pitch,
                              C.c_void_p(params.data_ptr()), C.c_void_p(target.data_ptr()),
                              C.c_void_p(mask.data_ptr()), count, C.c_void_p(grad.data_ptr()),
                              C.byref(loss), C.c_void_p(ws.ptr), C.c_size_t(ws.nbytes), _stream_ptr()),
           "nh_cnn_loss_grad")
    return loss.value


def nh_cnn_adam(params, grad, m, v, step, lr):
    L = load()
    for t in (params, grad, m, v):
        _params_check(t)
    _check(L.nh_cnn_adam(C.c_void_p(params.data_ptr()), C.c_void_p(grad.data_ptr()), C.c_void_p(m.data_ptr()),
                         C.c_void_p(v.data_ptr()), int(step), float(lr), _stream_ptr()), "nh_cnn_adam")


class Grid2D:
    """2D grids (nhswe2d.h): one grid, or an ensemble of grids stepped
    together (``Grid2D.ensemble``).  Arrays are (ny, nx), x fastest; the
    workspace is a torch.uint8 tensor on the current CUDA device."""

    def __init__(self, nx, ny, dx, dy, d0, bc_x=NH_BC_WALL, bc_y=NH_BC_WALL, limiter=NH_LIM_CENTRAL,
                 x0=0.0, y0=0.0, g=9.81, rho=1000.0, stream=None):
        self._create([dict(nx=nx, ny=ny, dx=dx, dy=dy, d0=d0, bc_x=bc_x, bc_y=bc_y, limiter=limiter,
                           x0=x0, y0=y0, g=g, rho=rho)], stream)

    @classmethod
    def ensemble(cls, members, stream=None):
        """members: dicts with nx, ny, dx, dy, d0 and optionally bc_x, bc_y,
        limiter, x0, y0, g, rho (the single-grid constructor's arguments)."""
        self = cls.__new__(cls)
        self._create(list(members), stream)
        return self

    def _create(self, members, stream):
        import torch
        self.L = load()
        self.h = None
        self.shapes = [(int(m["ny"]), int(m["nx"])) for m in members]
        self.nx, self.ny = self.shapes[0][1], self.shapes[0][0]
        n_m = len(members)
        descs = (nh_grid2d_desc * n_m)()
        for i, m in enumerate(members):
            descs[i] = nh_grid2d_desc(int(m["nx"]), int(m["ny"]), int(m.get("bc_x", NH_BC_WALL)),
                                      int(m.get("bc_y", NH_BC_WALL)), int(m.get("limiter", NH_LIM_CENTRAL)),
                                      float(m["dx"]), float(m["dy"]), float(m.get("x0", 0.0)),
                                      float(m.get("y0", 0.0)), float(m.get("g", 9.81)), float(m.get("rho", 1000.0)))
        self.descs = descs
        self.desc = descs[0]
        n = self.L.nh2d_ensemble_workspace_bytes(n_m, descs)
        if n == 0:
            raise NHError(NH_ERR_ARG, "nh2d_ensemble_workspace_bytes")
        self.ws = torch.empty(n + 256, dtype=torch.uint8, device="cuda")
        ptr = (self.ws.data_ptr() + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        d0s = [self._f(m["d0"], i) for i, m in enumerate(members)]
        arr = (_D * n_m)(*[_dptr(v) for v in d0s])
        h = C.c_void_p()
        _check(self.L.nh2d_create_ensemble(n_m, descs, arr, C.c_void_p(ptr), C.c_size_t(n),
                                           C.c_void_p(self.stream.cuda_stream), C.byref(h)), "nh2d_create_ensemble")
        self.h = h

    @property
    def members(self):
        return self.L.nh2d_members(self.h)

    def _shape(self, member):
        # an out-of-range member reaches the library, which rejects it
        return self.shapes[member] if 0 <= member < len(self.shapes) else (1, 1)

    def _f(self, a, member=0):
        if not 0 <= member < len(self.shapes):
            return np.zeros(1)
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), self.shapes[member]))
        return a.reshape(-1)

    @staticmethod
    def _slide(slide):
        return nh_slide2d_desc(int(slide.get("shape", NH_SLIDE_GAUSS_LNCOSH)), float(slide["A"]),
                               float(slide["Lx"]), float(slide["Ly"]), float(slide["xc0"]), float(slide["yc0"]),
                               float(slide["s0"]), float(slide["t0"]))

    def set_bottom_motion(self, slide=None, member=None):
        """slide: dict (A, Lx, Ly, xc0, yc0, s0, t0) or None; member None = all."""
        ref = None if slide is None else C.byref(self._slide(slide))
        if member is None:
            _check(self.L.nh2d_set_bottom_motion(self.h, ref), "nh2d_set_bottom_motion")
        else:
            _check(self.L.nh2d_set_member_bottom_motion(self.h, int(member), ref), "nh2d_set_member_bottom_motion")

    def set_criterion(self, kind, k_nh=1e-3, enlarge=1, first_step_global=False):
        _check(self.L.nh2d_set_criterion(self.h, int(kind), float(k_nh), int(enlarge), int(bool(first_step_global))),
               "nh2d_set_criterion")

    def set_solver(self, rtol=1e-12, max_iter=20000, guess=NH_GUESS_PREV):
        _check(self.L.nh2d_set_solver(self.h, float(rtol), int(max_iter), int(guess)), "nh2d_set_solver")

    def set_graphs(self, on):
        _check(self.L.nh2d_set_graphs(self.h, int(bool(on))), "nh2d_set_graphs")

    def set_wait_budget(self, cycles=0):
        """Spin limit of the solver's grid barrier in SM clock cycles (0: about one second)."""
        _check(self.L.nh2d_set_wait_budget(self.h, int(cycles)), "nh2d_set_wait_budget")

    def set_preconditioner(self, kind=NH_PRECOND_MG):
        """NH_PRECOND_MG (default) or NH_PRECOND_LINE for the CG solve."""
        _check(self.L.nh2d_set_preconditioner(self.h, int(kind)), "nh2d_set_preconditioner")

    def set_tile(self, tile=-1):
        """FP32 predictor tile: 0..3 forces a candidate (32x16, 64x8, 32x8, 64x16), -2 re-times at
        the next step, -1 only reads.  Returns the candidate in use (-1: not chosen yet)."""
        out = C.c_int(-1)
        _check(self.L.nh2d_set_tile(self.h, int(tile), C.byref(out)), "nh2d_set_tile")
        return out.value

    def set_profiling(self, enable=True):
        """Event pairs around every launch of later (host-enqueued) steps."""
        _check(self.L.nh2d_set_profiling(self.h, int(bool(enable))), "nh2d_set_profiling")

    def get_profile(self):
        """{class: (device ms, launches)} since the last set_profiling."""
        ms = np.zeros(len(KERNEL_CLASSES_2D))
        n = np.zeros(len(KERNEL_CLASSES_2D), dtype=np.int64)
        _check(self.L.nh2d_get_profile(self.h, _dptr(ms), n.ctypes.data_as(C.POINTER(C.c_longlong))),
               "nh2d_get_profile")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_CLASSES_2D)}

    def set_precision(self, precision):
        """NH_FP64 or NH_MIXED_FP64_SOLVE (FP32 state); clears every member's state."""
        _check(self.L.nh2d_set_precision(self.h, int(precision)), "nh2d_set_precision")

    def set_state(self, h, hu, hv, hw, t=0.0, member=0):
        a = [self._f(v, member) for v in (h, hu, hv, hw)]
        _check(self.L.nh2d_set_member_state(self.h, int(member), *[_dptr(v) for v in a], float(t)),
               "nh2d_set_member_state")

    def get_state(self, member=0):
        ny, nx = self._shape(member)
        out = [np.empty(nx * ny) for _ in range(5)]
        _check(self.L.nh2d_get_member_state(self.h, int(member), *[_dptr(v) for v in out]), "nh2d_get_member_state")
        return [v.reshape(ny, nx) for v in out]

    def put_state_ptr(self, member, h_ptr, hu_ptr, hv_ptr, hw_ptr):
        """Member state from raw host addresses (e.g. pinned tensors), keeping time and warm start."""
        _check(self.L.nh2d_put_member_state(self.h, int(member), C.c_void_p(h_ptr), C.c_void_p(hu_ptr),
                                            C.c_void_p(hv_ptr), C.c_void_p(hw_ptr)), "nh2d_put_member_state")

    def get_state_ptr(self, member, h_ptr, hu_ptr=0, hv_ptr=0, hw_ptr=0):
        """Member state into raw host addresses (0 skips a field)."""
        cast = lambda p: C.cast(C.c_void_p(p), _D) if p else None
        _check(self.L.nh2d_get_member_state(self.h, int(member), cast(h_ptr), cast(hu_ptr), cast(hv_ptr),
                                            cast(hw_ptr), None), "nh2d_get_member_state")

    def get_mask(self, member=0):
        ny, nx = self._shape(member)
        m = np.empty(nx * ny, dtype=np.uint8)
        _check(self.L.nh2d_get_member_mask(self.h, int(member), m.ctypes.data_as(C.POINTER(C.c_ubyte))),
               "nh2d_get_member_mask")
        return m.reshape(ny, nx)

    def member_info(self, member):
        info = nh_step_info()
        _check(self.L.nh2d_get_member_info(self.h, int(member), C.byref(info)), "nh2d_get_member_info")
        return info.as_dict()

    @property
    def graph_runs(self):
        return self.L.nh2d_graph_runs(self.h)

    def step(self, dt, check=True):
        info = nh_step_info()
        st = self.L.nh2d_step(self.h, float(dt), C.byref(info))
        if check:
            _check(st, "nh2d_step")
        return st, info.as_dict()

    def run(self, dt, n_steps, check=True):
        info = nh_run_info()
        st = self.L.nh2d_run(self.h, float(dt), int(n_steps), C.byref(info))
        if check:
            _check(st, "nh2d_run")
        return st, {"steps": info.steps, "iters_total": info.iters_total,
                    "active_total": info.active_total, "last": info.last.as_dict()}

    def close(self):
        if getattr(self, "h", None):
            self.L.nh2d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def grid_from_workload(wl, precision=NH_FP64, limiter=NH_LIM_CENTRAL, bc=None, **kw):
    """A Grid holding every member of a ``workloads.Workload1D`` (uniform or
    uneven cell counts) with its bottom motion and initial state set."""
    ms = wl.members
    m0 = ms[0]
    nxs = [m.nx for m in ms]
    nx = nxs[0] if len(set(nxs)) == 1 else nxs
    G = Grid(nx, m0.dx, [m.d0 for m in ms], nbatch=len(ms), x0=m0.xl,
             bc=wl.bc if bc is None else bc, precision=precision, limiter=limiter, **kw)
    if any(m.slide for m in ms):
        G.set_bottom_motion([dict(shape=m.slide, A=m.A, L=m.L, xc0=m.xc0, s0=m.s0, t0=m.t0, t2=m.t2)
                             for m in ms])
    G.set_state([m.h for m in ms], [m.hu for m in ms], [m.hw for m in ms])
    return G


class GridDG:
    """A batch of 1D members in the paper's DG-P1 / LDG discretisation
    (``include/nhswe_dg.h``), stepping through the C ABI.

    Per-node arrays are (nbatch, 2 ne): node 2i is element i's left end, node
    2i+1 its right end.  ``d0`` holds the static nodal depths.  Workspace and
    stream come from PyTorch as for ``Grid``.
    """

    def __init__(self, ne, dx, d0, nbatch=1, x0=0.0, g=9.81, rho=1000.0, c11=0.5, stream=None):
        import torch
        self.L = load()
        self.ne, self.nb = int(ne), int(nbatch)
        self.nn = 2 * self.ne
        self.dx = float(dx)
        self.desc = nh_dg_desc(self.ne, self.nb, float(dx), float(x0), float(g), float(rho), float(c11))
        nbytes = self.L.nh_dg_workspace_bytes(C.byref(self.desc))
        if nbytes == 0:
            raise NHError(NH_ERR_ARG, "nh_dg_workspace_bytes")
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        self._ws_ptr = (self.ws.data_ptr() + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        d0c = self._nodes(d0)
        h = C.c_void_p()
        _check(self.L.nh_dg_create(C.byref(self.desc), _dptr(d0c), C.c_void_p(self._ws_ptr), C.c_size_t(nbytes),
                                   C.c_void_p(self.stream.cuda_stream), C.byref(h)), "nh_dg_create")
        self.h = h
        self.workspace_bytes = nbytes

    def _nodes(self, a):
        arr = np.asarray(a, dtype=np.float64)
        if arr.ndim == 1 and arr.size == self.nn:
            arr = np.broadcast_to(arr, (self.nb, self.nn))
        return _f64(np.ascontiguousarray(arr), self.nb * self.nn)

    def nodes(self):
        """Node positions (2 ne) of every member."""
        i = np.arange(self.ne)
        x = np.empty(self.nn)
        x[0::2] = self.desc.x0 + i * self.dx
        x[1::2] = self.desc.x0 + (i + 1) * self.dx
        return x

    def set_bottom_motion(self, slides):
        if slides is None:
            _check(self.L.nh_dg_set_bottom_motion(self.h, None), "nh_dg_set_bottom_motion")
            return
        arr = (nh_slide_desc * self.nb)()
        for b, s in enumerate(slides):
            arr[b] = nh_slide_desc(int(s.get("shape", NH_SLIDE_GAUSS_LNCOSH)), float(s.get("A", 0.0)),
                                   float(s.get("L", 1.0)), float(s.get("xc0", 0.0)), float(s.get("s0", 0.0)),
                                   float(s.get("t0", 1.0)), float(s.get("t2", 0.0)))
        _check(self.L.nh_dg_set_bottom_motion(self.h, arr), "nh_dg_set_bottom_motion")

    def set_criterion(self, kind, k_nh=1e-3, enlarge=1, first_step_global=False):
        _check(self.L.nh_dg_set_criterion(self.h, int(kind), float(k_nh), int(enlarge),
                                          int(bool(first_step_global))), "nh_dg_set_criterion")

    def set_check(self, check=True):
        _check(self.L.nh_dg_set_check(self.h, int(bool(check))), "nh_dg_set_check")

    def set_state(self, h, hu, hw, t=0.0):
        h, hu, hw = self._nodes(h), self._nodes(hu), self._nodes(hw)
        _check(self.L.nh_dg_set_state(self.h, _dptr(h), _dptr(hu), _dptr(hw), float(t)), "nh_dg_set_state")

    def get_state(self):
        n = self.nb * self.nn
        h, hu, hw, p = (np.empty(n) for _ in range(4))
        _check(self.L.nh_dg_get_state(self.h, _dptr(h), _dptr(hu), _dptr(hw), _dptr(p)), "nh_dg_get_state")
        return tuple(a.reshape(self.nb, self.nn) for a in (h, hu, hw, p))

    def get_mask(self):
        m = np.empty(self.nb * self.ne, dtype=np.uint8)
        rr = np.empty(self.nb)
        _check(self.L.nh_dg_get_mask(self.h, m.ctypes.data_as(C.POINTER(C.c_ubyte)), _dptr(rr)), "nh_dg_get_mask")
        return m.reshape(self.nb, self.ne), rr

    def step(self, dt):
        info = nh_step_info()
        st = self.L.nh_dg_step(self.h, float(dt), C.byref(info))
        return st, info.as_dict()

    def run(self, dt, n_steps):
        info = nh_run_info()
        st = self.L.nh_dg_run(self.h, float(dt), int(n_steps), C.byref(info))
        return st, {"steps": info.steps, "active_total": info.active_total, "last": info.last.as_dict()}

    def set_profiling(self, enable=True):
        _check(self.L.nh_dg_set_profiling(self.h, int(bool(enable))), "nh_dg_set_profiling")

    def get_profile(self):
        ms = np.zeros(len(KERNEL_CLASSES_DG))
        n = np.zeros(len(KERNEL_CLASSES_DG), dtype=np.int64)
        _check(self.L.nh_dg_get_profile(self.h, _dptr(ms), n.ctypes.data_as(C.POINTER(C.c_longlong))),
               "nh_dg_get_profile")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_CLASSES_DG)}

    def close(self):
        if getattr(self, "h", None):
            self.L.nh_dg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
