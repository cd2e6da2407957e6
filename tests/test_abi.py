"""The C-ABI library builds, loads and exports every symbol include/ps.h
declares; host-side argument checks work without a GPU (no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_2005_13193_gb300 import _abi, make_grid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(ps_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    lib = _abi.load()
    declared = header_symbols()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(lib, name), name
    # and the Python binding describes each of them
    assert declared == set(_abi.SIGNATURES), declared ^ set(_abi.SIGNATURES)


def test_version_and_error_strings():
    lib = _abi.load()
    assert b"sm_103a" in lib.ps_version()
    assert isinstance(lib.ps_last_error(), bytes)


def test_workspace_queries_on_host():
    lib = _abi.load()
    g = make_grid((512, 512, 512))
    brick = (ctypes.c_int32 * 3)(8, 8, 8)
    nbins = 64 ** 3
    np_ = 1 << 24
    ws = lib.ps_bin_workspace_size(ctypes.byref(g), brick, np_)
    assert ws >= 4 * (nbins + 1) + 4 * np_
    ws_rk = lib.ps_rk2_workspace_size(ctypes.byref(g), brick, np_)
    assert ws_rk >= 24 * np_ + 8 * np_
    assert lib.ps_rk2_workspace_size(ctypes.byref(g), None, np_) == 0
    # planar FP32: the two-pass solve's unpadded intermediate where it applies
    # (optional: without it the three passes run in place)
    assert lib.ps_spline_coeffs_workspace_size(ctypes.byref(g), 3, _abi.PS_F32) >= 3 * 4 * 512 ** 3
    g_odd = make_grid((37, 20, 9))
    assert lib.ps_spline_coeffs_workspace_size(ctypes.byref(g_odd), 3, _abi.PS_F32) == 0
    assert lib.ps_spline_coeffs_workspace_size(ctypes.byref(g), 3, _abi.PS_BF16) >= 3 * 4 * 512 ** 3


@pytest.mark.parametrize("n", [(2, 8, 8), (8, 8, 4096), (0, 1, 1)])
def test_bad_grid_rejected_on_host(n):
    lib = _abi.load()
    g = make_grid(n)
    rc = lib.ps_spline_coeffs(ctypes.byref(g), 3, _abi.PS_F32, ctypes.c_void_p(16), _abi.PS_F32,
                              ctypes.c_void_p(16), None, None, 0, None)
    assert rc == _abi.PS_ERR_INVALID_ARG
    assert b"grid" in lib.ps_last_error()


def test_bad_arguments_rejected_on_host():
    lib = _abi.load()
    g = make_grid((16, 16, 16))
    P = ctypes.c_void_p(256)
    # missing scale for quantised coefficients
    rc = lib.ps_spline_coeffs(ctypes.byref(g), 3, _abi.PS_F32, P, _abi.PS_BF16, P, None, P,
                              1 << 20, None)
    assert rc == _abi.PS_ERR_INVALID_ARG
    # workspace too small
    s = ctypes.c_void_p(512)
    rc = lib.ps_spline_coeffs(ctypes.byref(g), 3, _abi.PS_F32, P, _abi.PS_BF16, P, s, P, 16, None)
    assert rc == _abi.PS_ERR_WORKSPACE
    # ncomp 2 is not an interpolation width
    rc = lib.ps_interp(ctypes.byref(g), 2, _abi.PS_F32, P, None, 10, P, None, None, None, P, None,
                       None, None)
    assert rc == _abi.PS_ERR_INVALID_ARG
    # brick of zero cells
    brick = (ctypes.c_int32 * 3)(8, 0, 8)
    rc = lib.ps_bin_particles(ctypes.byref(g), brick, 10, P, P, P, None, None, P, 1 << 20, None,
                              None)
    assert rc == _abi.PS_ERR_INVALID_ARG
    # rebin=0 without offsets
    brick = (ctypes.c_int32 * 3)(8, 8, 8)
    rc = lib.ps_rk2_step(ctypes.byref(g), _abi.PS_F32, P, None, None, None, 10, P, None, None,
                         1e-3, brick, 0, None, None, 0, None, None)
    assert rc == _abi.PS_ERR_INVALID_ARG
    # non-finite dt
    rc = lib.ps_rk2_step(ctypes.byref(g), _abi.PS_F32, P, None, None, None, 10, P, None, None,
                         float("nan"), None, 0, None, None, 0, None, None)
    assert rc == _abi.PS_ERR_INVALID_ARG
    # rebin outside 0..3
    for bad in (-1, 4):
        rc = lib.ps_rk2_step(ctypes.byref(g), _abi.PS_F32, P, None, None, None, 10, P, None,
                             None, 1e-3, brick, bad, P, P, 1 << 30, None, None)
        assert rc == _abi.PS_ERR_INVALID_ARG
        assert b"rebin" in lib.ps_last_error()
    # rebin 2 and 3 need the workspace like rebin 1
    for mode in (1, 2, 3):
        rc = lib.ps_rk2_step(ctypes.byref(g), _abi.PS_F32, P, None, None, None, 10, P, None,
                             None, 1e-3, brick, mode, P, None, 0, None, None)
        assert rc == _abi.PS_ERR_WORKSPACE


# every tune key: its documented values are taken and read back, anything
# else is refused and leaves the value unchanged (host only, no GPU)
TUNE_KEYS = {
    "brick_kernel": ([-1, 0, 2, 5], [1, 3, 4, 6, -2]),
    "brick_min_stage": ([0, 8, 1 << 20], [-1, (1 << 20) + 1]),
    "node_tma": ([0, 1], [2, -1]),
    "solve_xw": ([0, 8, 16, 32], [4, 24, 64]),
    "solve_stream": ([0, 1], [2, -1]),
    "solve_zt": ([0, 16, 32, 64, 128, 256], [8, 48, 512]),
    "solve_stages": ([0, 2, 3, 4], [1, 5]),
    "batch_run_below": ([0, 16, 1 << 20], [-1, (1 << 20) + 1]),
    "batch_persistent": ([0, 1], [2, -1]),
    "wait_probe": ([0, 1000, 1 << 30], [-1, (1 << 30) + 1]),
}


@pytest.mark.parametrize("key", sorted(TUNE_KEYS))
def test_tune_keys_on_host(key):
    lib = _abi.load()
    k = key.encode()
    good, bad = TUNE_KEYS[key]
    old = lib.ps_tune_get(k)
    try:
        for v in good:
            assert lib.ps_tune_set(k, v) == _abi.PS_OK, (key, v)
            assert lib.ps_tune_get(k) == v
        last = lib.ps_tune_get(k)
        for v in bad:
            assert lib.ps_tune_set(k, v) == _abi.PS_ERR_INVALID_ARG, (key, v)
            assert lib.ps_tune_get(k) == last
    finally:
        lib.ps_tune_set(k, old)
    assert lib.ps_tune_set(b"no_such_key", 1) == _abi.PS_ERR_INVALID_ARG
    assert lib.ps_tune_get(b"no_such_key") == -1
