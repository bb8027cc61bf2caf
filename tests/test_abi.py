"""The C-ABI library builds for sm_103a and exports every entry point that
the headers in include/ declare (no GPU needed: symbols only, no compute
call)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2505_17025_gb300 import build as B
from paper_2505_17025_gb300 import nhswe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(nh[a-z0-9]*_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(B.build())
    declared = _declared()
    assert declared, "no declarations found"
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(nhswe.EXPORTS) <= declared


def test_workspace_size_needs_no_gpu():
    lib = ctypes.CDLL(B.build())
    lib.nh_workspace_bytes.argtypes = [ctypes.POINTER(nhswe.nh_grid_desc)]
    lib.nh_workspace_bytes.restype = ctypes.c_size_t
    d = nhswe.nh_grid_desc(1, 50000, 64, 0, 0, 1, 8e-4, 0.0, 9.81, 1000.0)
    n = lib.nh_workspace_bytes(ctypes.byref(d))
    assert n > 64 * 50000 * 8 * 20
    bad = nhswe.nh_grid_desc(1, 4, 1, 0, 0, 1, 8e-4, 0.0, 9.81, 1000.0)   # nx < 8
    assert lib.nh_workspace_bytes(ctypes.byref(bad)) == 0
    bad = nhswe.nh_grid_desc(1, 100, 1, 0, 0, 1, -1.0, 0.0, 9.81, 1000.0)  # dx <= 0
    assert lib.nh_workspace_bytes(ctypes.byref(bad)) == 0


def test_status_strings_need_no_gpu():
    lib = ctypes.CDLL(B.build())
    lib.nh_status_string.restype = ctypes.c_char_p
    for s in range(7):
        assert lib.nh_status_string(s).startswith(b"NH_")


def test_workspace_size_2d_needs_no_gpu():
    lib = ctypes.CDLL(B.build())
    lib.nh2d_workspace_bytes.argtypes = [ctypes.POINTER(nhswe.nh_grid2d_desc)]
    lib.nh2d_workspace_bytes.restype = ctypes.c_size_t
    d = nhswe.nh_grid2d_desc(1024, 1024, 1, 1, 1, 0.05, 0.05, 0.0, 0.0, 9.81, 1000.0)
    assert lib.nh2d_workspace_bytes(ctypes.byref(d)) > 1024 * 1024 * 8 * 40
    bad = nhswe.nh_grid2d_desc(2, 1024, 0, 0, 1, 0.05, 0.05, 0.0, 0.0, 9.81, 1000.0)   # nx < 3
    assert lib.nh2d_workspace_bytes(ctypes.byref(bad)) == 0


def test_ensemble_workspace_2d_needs_no_gpu():
    """Every member gets a slot of the largest member's cells (rounded up to
    256); an invalid member or an empty ensemble gives 0."""
    lib = ctypes.CDLL(B.build())
    lib.nh2d_ensemble_workspace_bytes.argtypes = [ctypes.c_int, ctypes.POINTER(nhswe.nh_grid2d_desc)]
    lib.nh2d_ensemble_workspace_bytes.restype = ctypes.c_size_t
    lib.nh2d_workspace_bytes.argtypes = [ctypes.POINTER(nhswe.nh_grid2d_desc)]
    lib.nh2d_workspace_bytes.restype = ctypes.c_size_t
    D = nhswe.nh_grid2d_desc
    big = D(512, 500, 0, 0, 1, 0.02, 0.02, 0.0, 0.0, 9.81, 1000.0)
    small = D(40, 30, 1, 0, 2, 0.05, 0.04, 0.0, 0.0, 9.81, 1000.0)
    one = lib.nh2d_workspace_bytes(ctypes.byref(big))
    arr = (D * 3)(small, big, small)
    three = lib.nh2d_ensemble_workspace_bytes(3, arr)
    assert 2.9 * one < three < 3.1 * one
    assert lib.nh2d_ensemble_workspace_bytes(1, arr) < lib.nh2d_ensemble_workspace_bytes(2, arr)
    assert lib.nh2d_ensemble_workspace_bytes(0, arr) == 0
    arr[2] = D(40, 2, 1, 0, 2, 0.05, 0.04, 0.0, 0.0, 9.81, 1000.0)   # ny < 3
    assert lib.nh2d_ensemble_workspace_bytes(3, arr) == 0


def test_product_path_fails_loudly_without_a_gpu():
    """No CPU fallback: on a machine without CUDA every product entry point
    raises instead of computing anything (the oracle is never consulted)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2505_17025_gb300 import workloads as W
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        nhswe.load()
    with pytest.raises(RuntimeError):
        nhswe.grid_from_workload(W.slide_1d(n_members=1, nx=64, length=1.0, T=0.01))
    with pytest.raises(RuntimeError):
        nhswe.Grid2D(8, 8, 0.1, 0.1, np.ones((8, 8)))


def test_workspace_size_dg_needs_no_gpu():
    """The DG handle's workspace grows with members x elements; invalid
    descriptors (ne < 2, dx <= 0, negative c11) give 0."""
    lib = ctypes.CDLL(B.build())
    lib.nh_dg_workspace_bytes.argtypes = [ctypes.POINTER(nhswe.nh_dg_desc)]
    lib.nh_dg_workspace_bytes.restype = ctypes.c_size_t
    D = nhswe.nh_dg_desc
    small = lib.nh_dg_workspace_bytes(ctypes.byref(D(200, 1, 4.0, 0.0, 9.81, 1000.0, 0.5)))
    big = lib.nh_dg_workspace_bytes(ctypes.byref(D(50000, 64, 1e-3, 0.0, 9.81, 1000.0, 0.5)))
    assert small > 200 * 8 * 30 and big > 64 * 50000 * 8 * 60
    for bad in (D(1, 1, 4.0, 0.0, 9.81, 1000.0, 0.5), D(200, 1, 0.0, 0.0, 9.81, 1000.0, 0.5),
                D(200, 1, 4.0, 0.0, 9.81, 1000.0, -0.5), D(200, 0, 4.0, 0.0, 9.81, 1000.0, 0.5)):
        assert lib.nh_dg_workspace_bytes(ctypes.byref(bad)) == 0
