"""FP64 CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``oracle.c`` (plain C, built
with ``-ffp-contract=off``) through ctypes and shares nothing with the CUDA
library: no code, no header, no constant.

Each wrapper states the passage of Buaria & Yeung (arXiv 2005.13193) it
follows; the C file carries the full statement and the readings taken where
the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_ARG = 1
ERR_NONFINITE = 2
ERR_NOMEM = 3


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            i32 = ctypes.c_int
            d = ctypes.c_double
            lib.ora_cyclic_solve.argtypes = [i32, P, P]
            lib.ora_spline_coeffs.argtypes = [P, i32, P, P]
            lib.ora_interp.argtypes = [P, P, i32, P, i64, P, P, P]
            lib.ora_bin.argtypes = [P, P, P, i64, P, P, P, P]
            lib.ora_interp_backward.argtypes = [P, P, i32, P, i64, P, P, P, P]
            lib.ora_rk2_step.argtypes = [P, P, P, P, i64, P, d, P]
            lib.ora_interp_windowed.argtypes = [P, P, P, i64, P, P]
            lib.ora_interp_hessian.argtypes = [P, P, i32, P, i64, P, P]
            lib.ora_lagrangian_accel.argtypes = [P, P, P, P, d, i64, P, P]
            lib.ora_basis.argtypes = [d, P, P]
            lib.ora_basis.restype = None
            lib.ora_locate.argtypes = [d, d, i32, P, P]
            lib.ora_spline_coeffs_truncated.argtypes = [P, i32, i32, P, P]
            lib.ora_green.argtypes = [i64, i64, P]
            lib.ora_green.restype = None
            lib.ora_set_num_threads.argtypes = [i32]
            lib.ora_set_num_threads.restype = None
            lib.ora_num_threads.restype = i32
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _grid(n, L):
    n_arr = np.ascontiguousarray(n, dtype=np.int32)
    L_arr = np.ascontiguousarray(L, dtype=np.float64)
    assert n_arr.shape == (3,) and L_arr.shape == (3,)
    return n_arr, L_arr


def _check(rc, allow_nonfinite=False):
    if rc == OK or (allow_nonfinite and rc == ERR_NONFINITE):
        return rc
    raise OracleError(f"oracle returned {rc}")


def set_num_threads(n: int) -> None:
    _load().ora_set_num_threads(int(n))


def num_threads() -> int:
    return int(_load().ora_num_threads())


def cyclic_solve(g) -> np.ndarray:
    """Sec. 2.2: periodic (1/6, 4/6, 1/6) system by Thomas + Sherman-Morrison."""
    g = _f64(g)
    c = np.empty_like(g)
    _check(_load().ora_cyclic_solve(len(g), _p(g), _p(c)))
    return c


def spline_coeffs(field, n=None) -> np.ndarray:
    """Sec. 2.2 Operation 1: field [ncomp][nz][ny][nx] -> padded [ncomp][nz+3][ny+3][nx+3]."""
    field = _f64(field)
    assert field.ndim == 4
    ncomp, nz, ny, nx = field.shape
    n_arr = np.array([nx, ny, nz], dtype=np.int32)
    coef = np.empty((ncomp, nz + 3, ny + 3, nx + 3), dtype=np.float64)
    _check(_load().ora_spline_coeffs(_p(n_arr), ncomp, _p(field), _p(coef)))
    return coef


def spline_coeffs_truncated(field, K) -> np.ndarray:
    """Sec. 2.2 Operation 1 through the periodic inverse's entries G_N(d), cut to
    |d| <= K (2K + 1 <= N): field [ncomp][nz][ny][nx] -> padded coefficients."""
    field = _f64(field)
    assert field.ndim == 4
    ncomp, nz, ny, nx = field.shape
    n_arr = np.array([nx, ny, nz], dtype=np.int32)
    coef = np.empty((ncomp, nz + 3, ny + 3, nx + 3), dtype=np.float64)
    _check(_load().ora_spline_coeffs_truncated(_p(n_arr), ncomp, int(K), _p(field), _p(coef)))
    return coef


def interp(coef, pos, L=(2 * np.pi,) * 3, grad=False, allow_nonfinite=False):
    """Sec. 2.2 Eq. (spline): coef [ncomp][nz+3][ny+3][nx+3], pos [3][np] -> vel [ncomp][np]
    (and grad [ncomp][3][np] when asked)."""
    coef = _f64(coef)
    pos = _f64(pos)
    ncomp = coef.shape[0]
    n_arr, L_arr = _grid([coef.shape[3] - 3, coef.shape[2] - 3, coef.shape[1] - 3], L)
    npart = pos.shape[1]
    vel = np.empty((ncomp, npart), dtype=np.float64)
    g = np.empty((ncomp, 3, npart), dtype=np.float64) if grad else None
    rc = _load().ora_interp(_p(n_arr), _p(L_arr), ncomp, _p(coef), npart, _p(pos),
                            _p(vel), _p(g) if grad else None)
    _check(rc, allow_nonfinite)
    return (vel, g) if grad else vel


def interp_hessian(coef, pos, L=(2 * np.pi,) * 3, allow_nonfinite=False):
    """Second derivatives of Eq. (spline): hess [ncomp][6][np] (xx, yy, zz, xy, xz, yz)."""
    coef = _f64(coef)
    pos = _f64(pos)
    ncomp = coef.shape[0]
    n_arr, L_arr = _grid([coef.shape[3] - 3, coef.shape[2] - 3, coef.shape[1] - 3], L)
    npart = pos.shape[1]
    hess = np.empty((ncomp, 6, npart), dtype=np.float64)
    _check(_load().ora_interp_hessian(_p(n_arr), _p(L_arr), ncomp, _p(coef), npart, _p(pos),
                                      _p(hess)), allow_nonfinite)
    return hess


def lagrangian_accel(coef_n, pos, coef_np1=None, dt_field=1.0, L=(2 * np.pi,) * 3):
    """a = du/dt + (u . grad) u at the particles ([3][np]); du/dt by the two-field
    difference when coef_np1 is given."""
    coef_n = _f64(coef_n)
    pos = _f64(pos)
    n_arr, L_arr = _grid([coef_n.shape[3] - 3, coef_n.shape[2] - 3, coef_n.shape[1] - 3], L)
    npart = pos.shape[1]
    acc = np.empty((3, npart), dtype=np.float64)
    c1 = _f64(coef_np1) if coef_np1 is not None else None
    _check(_load().ora_lagrangian_accel(_p(n_arr), _p(L_arr), _p(coef_n),
                                        _p(c1) if c1 is not None else None, float(dt_field),
                                        npart, _p(pos), _p(acc)))
    return acc


def bin_particles(n, brick, pos, L=(2 * np.pi,) * 3):
    """Sec. 3 dynamic mapping, read as a stable counting sort into bricks.
    Returns bin_of [np] int32, bin_offsets [nbins+1] int32, perm [np] int64."""
    n_arr, L_arr = _grid(n, L)
    br = np.ascontiguousarray(brick, dtype=np.int32)
    pos = _f64(pos)
    npart = pos.shape[1]
    nb = [(int(n_arr[d]) + int(br[d]) - 1) // int(br[d]) for d in range(3)]
    nbins = nb[0] * nb[1] * nb[2]
    bin_of = np.empty(npart, dtype=np.int32)
    offs = np.empty(nbins + 1, dtype=np.int32)
    perm = np.empty(npart, dtype=np.int64)
    _check(_load().ora_bin(_p(n_arr), _p(L_arr), _p(br), npart, _p(pos), _p(bin_of),
                           _p(offs), _p(perm)))
    return bin_of, offs, perm


def interp_backward(coef, pos, g_vel, n=None, L=(2 * np.pi,) * 3, want_pos=True,
                    want_field=True):
    """Adjoint of Eq. (spline) and of the coefficient solve (transpose = same
    symmetric solves applied to the folded scatter)."""
    coef = _f64(coef)
    pos = _f64(pos)
    g_vel = _f64(g_vel)
    ncomp = coef.shape[0]
    nz, ny, nx = coef.shape[1] - 3, coef.shape[2] - 3, coef.shape[3] - 3
    n_arr, L_arr = _grid([nx, ny, nz], L)
    npart = pos.shape[1]
    g_pos = np.empty((3, npart)) if want_pos else None
    g_field = np.empty((ncomp, nz, ny, nx)) if want_field else None
    rc = _load().ora_interp_backward(
        _p(n_arr), _p(L_arr), ncomp, _p(coef), npart, _p(pos), _p(g_vel),
        _p(g_pos) if want_pos else None, _p(g_field) if want_field else None)
    _check(rc)
    return g_pos, g_field


def rk2_step(coef_n, pos, dt, coef_np1=None, L=(2 * np.pi,) * 3):
    """Sec. 2.1 / 4.3 second-order Runge-Kutta, read as Heun. Returns (new pos, u1)."""
    coef_n = _f64(coef_n)
    assert coef_n.shape[0] == 3
    pos = np.array(pos, dtype=np.float64, copy=True, order="C")
    nz, ny, nx = coef_n.shape[1] - 3, coef_n.shape[2] - 3, coef_n.shape[3] - 3
    n_arr, L_arr = _grid([nx, ny, nz], L)
    c1 = _f64(coef_np1) if coef_np1 is not None else None
    npart = pos.shape[1]
    vel = np.empty((3, npart))
    _check(_load().ora_rk2_step(_p(n_arr), _p(L_arr), _p(coef_n),
                                _p(c1) if c1 is not None else None, npart, _p(pos),
                                float(dt), _p(vel)))
    return pos, vel


def interp_windowed(field_f32, pos, L=(2 * np.pi,) * 3):
    """Eq. (spline) with coefficients from the truncated exact periodic inverse
    (for grids whose FP64 coefficients do not fit in host memory)."""
    field = np.ascontiguousarray(field_f32, dtype=np.float32)
    assert field.ndim == 4 and field.shape[0] == 3
    _, nz, ny, nx = field.shape
    n_arr, L_arr = _grid([nx, ny, nz], L)
    pos = _f64(pos)
    npart = pos.shape[1]
    vel = np.empty((3, npart))
    _check(_load().ora_interp_windowed(_p(n_arr), _p(L_arr), _p(field), npart, _p(pos),
                                       _p(vel)))
    return vel


def basis(t):
    """Uniform cubic B-spline basis and its derivative at local coordinate t."""
    b = np.empty(4)
    db = np.empty(4)
    _load().ora_basis(float(t), _p(b), _p(db))
    return b, db


def locate(x, L, n):
    cell = np.zeros(1, dtype=np.int64)
    t = np.zeros(1)
    rc = _load().ora_locate(float(x), float(L), int(n), _p(cell), _p(t))
    _check(rc)
    return int(cell[0]), float(t[0])


def green(n, d):
    out = np.zeros(1)
    _load().ora_green(int(n), int(d), _p(out))
    return float(out[0])
