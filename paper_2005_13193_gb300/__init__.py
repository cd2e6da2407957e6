"""Periodic cubic-spline particle interpolation on one GB300.

Python binding of the C ABI in include/ps.h (Buaria & Yeung, arXiv
2005.13193, Sec. 2.2 Eq. (spline), Sec. 3, Sec. 4.3).  The ``ps_*``
functions carry the C names and only marshal torch tensors into pointers and
sizes; every step of the computation runs in the CUDA library libps.so.  If
that library cannot be loaded the calls raise: there is no CPU path.

Higher-level helpers (`SplineField`, `Tracker`, `InterpFn`) allocate with
torch and call the same entry points.
"""
from __future__ import annotations

import ctypes
import math
from typing import Optional, Sequence

import torch

from . import _abi
from ._abi import (PS_BF16, PS_BF16X4, PS_F16, PS_F16X4, PS_F32, PS_F32X4, PS_F64, PS_OK,
                   PsGrid)

TWO_PI = 2.0 * math.pi
DEFAULT_L = (TWO_PI, TWO_PI, TWO_PI)

_DT = {torch.float32: PS_F32, torch.float64: PS_F64, torch.bfloat16: PS_BF16,
       torch.float16: PS_F16}

# Coefficient storage with the three components of a node interleaved
# (u, v, w, 0): a tensor [nz+3][ny+3][pitch][4], float32 (PS_F32X4) or 16-bit
# values scaled per component and x-line (PS_BF16X4, PS_F16X4; the scales are
# a float32 tensor [nz+3][ny+3][4]).
F32X4 = "f32x4"
BF16X4 = "bf16x4"
F16X4 = "f16x4"
_NODE = {F32X4: (PS_F32X4, torch.float32), BF16X4: (PS_BF16X4, torch.bfloat16),
         F16X4: (PS_F16X4, torch.float16)}
_NODE_OF = {v[1]: k for k, v in _NODE.items()}


def _is_token(dtype) -> bool:
    return isinstance(dtype, str)


def _dt_code(dtype) -> int:
    return _NODE[dtype][0] if _is_token(dtype) else _DT[dtype]


def _is_node4(coef: torch.Tensor) -> bool:
    # planar rows hold >= 8 elements, so a last extent of 4 is a node array
    return coef.dtype in _NODE_OF and coef.dim() == 4 and coef.shape[-1] == 4


def _coef_type(coef: torch.Tensor) -> int:
    return _dt_code(coef_kind(coef))


def coef_kind(coef: torch.Tensor):
    """The coefficient dtype argument a tensor corresponds to (a node token or a torch dtype)."""
    return _NODE_OF[coef.dtype] if _is_node4(coef) else coef.dtype


def _ncomp_of(coef: torch.Tensor) -> int:
    return 3 if _is_node4(coef) else coef.shape[0]


class PSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libps error {code}: {msg}")
        self.code = code


def _lib():
    return _abi.load()


def _check(rc: int):
    if rc != PS_OK:
        raise PSError(rc, _lib().ps_last_error().decode())


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _dev(t: Optional[torch.Tensor], name: str, dtype=None, numel=None):
    if t is None:
        return
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, needs {numel}")


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def make_grid(n: Sequence[int], L: Sequence[float] = DEFAULT_L) -> PsGrid:
    """n = (nx, ny, nz) nodes; L = box lengths."""
    g = PsGrid()
    for d in range(3):
        g.n[d] = int(n[d])
        g.L[d] = float(L[d])
    return g


def _brick_arr(brick):
    if brick is None:
        return None
    if isinstance(brick, int):
        brick = (brick, brick, brick)
    return (ctypes.c_int32 * 3)(*[int(b) for b in brick])


def coef_row_pitch(nx: int, dtype: torch.dtype) -> int:
    """Row pitch (elements) of a padded coefficient array: nx+3 rounded up to
    16 bytes (ps_coef_row_pitch)."""
    return int(_lib().ps_coef_row_pitch(int(nx), _dt_code(dtype)))


def coef_shape(n, ncomp: int, dtype):
    """Storage shape [ncomp][nz+3][ny+3][pitch] of padded coefficients, or
    [nz+3][ny+3][nx+3][4] for F32X4 (ncomp 3)."""
    if _is_token(dtype):
        if ncomp != 3:
            raise ValueError("node coefficients hold three components")
        return (n[2] + 3, n[1] + 3, coef_row_pitch(n[0], dtype), 4)
    return (ncomp, n[2] + 3, n[1] + 3, coef_row_pitch(n[0], dtype))


def scale_shape(n, ncomp: int, dtype):
    """Shape of the per-x-line scales of 16-bit coefficients (None otherwise)."""
    if dtype in (BF16X4, F16X4):
        return (n[2] + 3, n[1] + 3, 4)
    if dtype in (torch.bfloat16, torch.float16):
        return (ncomp, n[2] + 3, n[1] + 3)
    return None


def _storage_dtype(dtype) -> torch.dtype:
    return _NODE[dtype][1] if _is_token(dtype) else dtype


def _check_coef_shape(coef: torch.Tensor, n):
    want = coef_shape(n, _ncomp_of(coef), coef_kind(coef))
    if tuple(coef.shape) != want:
        raise ValueError(f"coef has shape {tuple(coef.shape)}, grid {tuple(n)} needs {want}")


def grid_of_field(field: torch.Tensor):
    return (field.shape[3], field.shape[2], field.shape[1])


# ------------------------------------------------------------- C entry points ----

def ps_last_error() -> str:
    return _lib().ps_last_error().decode()


def ps_version() -> str:
    return _lib().ps_version().decode()


def ps_tune_set(key: str, value: int):
    _check(_lib().ps_tune_set(key.encode(), int(value)))


def ps_tune_get(key: str) -> int:
    return int(_lib().ps_tune_get(key.encode()))


def ps_status_clear(status: torch.Tensor, stream=None):
    _dev(status, "status", torch.int32, 4)
    _check(_lib().ps_status_clear(_ptr(status), _stream(stream)))


def ps_status_read(status: torch.Tensor, stream=None, raise_on_error: bool = False):
    """Returns [code, index_lo, index_hi, count]."""
    _dev(status, "status", torch.int32, 4)
    out = (ctypes.c_int32 * 4)()
    rc = _lib().ps_status_read(_ptr(status), ctypes.cast(out, ctypes.c_void_p), _stream(stream))
    if rc not in (PS_OK, _abi.PS_ERR_DEVICE_STATUS) or (raise_on_error and rc != PS_OK):
        _check(rc)
    return list(out)


def ps_spline_coeffs_workspace_size(n, ncomp: int, coef_dtype: torch.dtype,
                                    L=DEFAULT_L) -> int:
    g = make_grid(n, L)
    return int(_lib().ps_spline_coeffs_workspace_size(ctypes.byref(g), ncomp,
                                                       _dt_code(coef_dtype)))


def ps_spline_coeffs(field: torch.Tensor, coef: torch.Tensor, scale: Optional[torch.Tensor] = None,
                     ws: Optional[torch.Tensor] = None, L=DEFAULT_L, stream=None):
    """Operation 1 (Sec. 2.2): field [ncomp][nz][ny][nx] -> coef [ncomp][nz+3][ny+3][nx+3]."""
    n = grid_of_field(field)
    ncomp = field.shape[0]
    _dev(field, "field")
    _check_coef_shape(coef, n)
    _dev(coef, "coef")
    _dev(scale, "scale", torch.float32)
    _dev(ws, "ws")
    g = make_grid(n, L)
    ws_bytes = ws.numel() * ws.element_size() if ws is not None else 0
    _check(_lib().ps_spline_coeffs(ctypes.byref(g), ncomp, _DT[field.dtype], _ptr(field),
                                   _coef_type(coef), _ptr(coef), _ptr(scale), _ptr(ws), ws_bytes,
                                   _stream(stream)))


def ps_bin_workspace_size(n, brick, np_: int, L=DEFAULT_L) -> int:
    g = make_grid(n, L)
    return int(_lib().ps_bin_workspace_size(ctypes.byref(g), _brick_arr(brick), int(np_)))


def ps_bin_particles(n, brick, pos: torch.Tensor, bin_of: torch.Tensor, bin_offsets: torch.Tensor,
                     perm: Optional[torch.Tensor] = None, pos_sorted: Optional[torch.Tensor] = None,
                     ws: Optional[torch.Tensor] = None, status: Optional[torch.Tensor] = None,
                     L=DEFAULT_L, stream=None):
    """Sec. 3 dynamic mapping read as a bin sort into bricks of `brick` cells."""
    np_ = pos.shape[1]
    _dev(pos, "pos", torch.float64)
    _dev(bin_of, "bin_of", torch.int32, np_)
    _dev(bin_offsets, "bin_offsets", torch.int32)
    _dev(perm, "perm", torch.int64, np_)
    _dev(pos_sorted, "pos_sorted", torch.float64, 3 * np_)
    _dev(ws, "ws")
    _dev(status, "status", torch.int32, 4)
    g = make_grid(n, L)
    ws_bytes = ws.numel() * ws.element_size() if ws is not None else 0
    _check(_lib().ps_bin_particles(ctypes.byref(g), _brick_arr(brick), np_, _ptr(pos),
                                   _ptr(bin_of), _ptr(bin_offsets), _ptr(perm), _ptr(pos_sorted),
                                   _ptr(ws), ws_bytes, _ptr(status), _stream(stream)))


def ps_spline_truncated_workspace_size(n, ncomp: int, L=DEFAULT_L) -> int:
    g = make_grid(n, L)
    return int(_lib().ps_spline_truncated_workspace_size(ctypes.byref(g), ncomp))


def ps_spline_coeffs_truncated(field: torch.Tensor, coef: torch.Tensor, K: int = 15,
                               ws: Optional[torch.Tensor] = None, L=DEFAULT_L, stream=None):
    """Operation 1 (Sec. 2.2) through the periodic inverse cut to |d| <= K: field
    [ncomp][nz][ny][nx] F32 -> padded F32 coefficients (the layout of PS_F32)."""
    n = grid_of_field(field)
    ncomp = field.shape[0]
    _dev(field, "field", torch.float32)
    _dev(coef, "coef", torch.float32)
    if tuple(coef.shape) != coef_shape(n, ncomp, torch.float32):
        raise ValueError(f"coef shape {tuple(coef.shape)} != {coef_shape(n, ncomp, torch.float32)}")
    if ws is None:
        ws = workspace(ps_spline_truncated_workspace_size(n, ncomp, L), field.device)
    _dev(ws, "ws")
    g = make_grid(n, L)
    _check(_lib().ps_spline_coeffs_truncated(ctypes.byref(g), ncomp, _ptr(field), int(K),
                                             _ptr(coef), _ptr(ws), ws.numel() * ws.element_size(),
                                             _stream(stream)))


def ps_interp(coef: torch.Tensor, n, pos: torch.Tensor, vel: torch.Tensor,
              scale: Optional[torch.Tensor] = None, perm: Optional[torch.Tensor] = None,
              bin_offsets: Optional[torch.Tensor] = None, brick=None,
              grad: Optional[torch.Tensor] = None, status: Optional[torch.Tensor] = None,
              L=DEFAULT_L, stream=None):
    """Operations 2-3 (Sec. 2.2, Eq. (spline)) at positions pos [3][np] -> vel [ncomp][np].
    n = (nx, ny, nz) of the grid the coefficients belong to."""
    _check_coef_shape(coef, n)
    ncomp = _ncomp_of(coef)
    np_ = pos.shape[1]
    _dev(coef, "coef")
    _dev(pos, "pos", torch.float64)
    _dev(vel, "vel", torch.float32, ncomp * np_)
    _dev(scale, "scale", torch.float32)
    _dev(perm, "perm", torch.int64, np_)
    _dev(bin_offsets, "bin_offsets", torch.int32)
    _dev(grad, "grad", torch.float32, ncomp * 3 * np_)
    _dev(status, "status", torch.int32, 4)
    g = make_grid(n, L)
    _check(_lib().ps_interp(ctypes.byref(g), ncomp, _coef_type(coef), _ptr(coef), _ptr(scale), np_,
                            _ptr(pos), _ptr(perm), _ptr(bin_offsets), _brick_arr(brick),
                            _ptr(vel), _ptr(grad), _ptr(status), _stream(stream)))


def ps_interp_backward(coef: torch.Tensor, n, pos: torch.Tensor, g_vel: torch.Tensor,
                       g_pos: Optional[torch.Tensor] = None, g_field: Optional[torch.Tensor] = None,
                       scale: Optional[torch.Tensor] = None, status: Optional[torch.Tensor] = None,
                       L=DEFAULT_L, stream=None):
    """Adjoint of ps_interp and of the coefficient solve."""
    _check_coef_shape(coef, n)
    ncomp = _ncomp_of(coef)
    np_ = pos.shape[1]
    _dev(coef, "coef")
    _dev(pos, "pos", torch.float64)
    _dev(g_vel, "g_vel", torch.float32, ncomp * np_)
    _dev(g_pos, "g_pos", torch.float64, 3 * np_)
    _dev(g_field, "g_field", torch.float32, ncomp * n[0] * n[1] * n[2])
    _dev(status, "status", torch.int32, 4)
    g = make_grid(n, L)
    _check(_lib().ps_interp_backward(ctypes.byref(g), ncomp, _coef_type(coef), _ptr(coef),
                                     _ptr(scale), np_, _ptr(pos), _ptr(g_vel), _ptr(g_pos),
                                     _ptr(g_field), None, 0, _ptr(status), _stream(stream)))


def ps_interp_hessian(coef: torch.Tensor, n, pos: torch.Tensor, hess: torch.Tensor,
                      scale: Optional[torch.Tensor] = None, perm: Optional[torch.Tensor] = None,
                      bin_offsets: Optional[torch.Tensor] = None, brick=None,
                      status: Optional[torch.Tensor] = None, L=DEFAULT_L, stream=None):
    """Second derivatives of Eq. (spline): hess [ncomp][6][np] (xx, yy, zz, xy, xz, yz).
    With bin_offsets (and brick, perm as for ps_interp) the stencils come from each
    brick's staged halo."""
    _check_coef_shape(coef, n)
    ncomp = _ncomp_of(coef)
    np_ = pos.shape[1]
    _dev(coef, "coef")
    _dev(pos, "pos", torch.float64)
    _dev(hess, "hess", torch.float32, ncomp * 6 * np_)
    _dev(scale, "scale", torch.float32)
    _dev(perm, "perm", torch.int64, np_)
    _dev(bin_offsets, "bin_offsets", torch.int32)
    _dev(status, "status", torch.int32, 4)
    g = make_grid(n, L)
    _check(_lib().ps_interp_hessian(ctypes.byref(g), ncomp, _coef_type(coef), _ptr(coef),
                                    _ptr(scale), np_, _ptr(pos), _ptr(perm), _ptr(bin_offsets),
                                    _brick_arr(brick), _ptr(hess), _ptr(status),
                                    _stream(stream)))


def ps_lagrangian_accel(coef_n: torch.Tensor, n, pos: torch.Tensor, acc: torch.Tensor,
                        coef_np1: Optional[torch.Tensor] = None, dt_field: float = 1.0,
                        scale_n: Optional[torch.Tensor] = None,
                        scale_np1: Optional[torch.Tensor] = None,
                        vel: Optional[torch.Tensor] = None, perm: Optional[torch.Tensor] = None,
                        bin_offsets: Optional[torch.Tensor] = None, brick=None,
                        status: Optional[torch.Tensor] = None, L=DEFAULT_L, stream=None):
    """a = du/dt + (u . grad) u at pos [3][np] -> acc [3][np] (du/dt from two fields).
    With bin_offsets (and brick, perm as for ps_interp) the stencils of coef_n come from
    each brick's staged halo."""
    _check_coef_shape(coef_n, n)
    np_ = pos.shape[1]
    _dev(coef_n, "coef_n")
    _dev(coef_np1, "coef_np1", coef_n.dtype)
    if coef_np1 is not None and _coef_type(coef_np1) != _coef_type(coef_n):
        raise ValueError("coef_np1 must have the storage of coef_n")
    _dev(pos, "pos", torch.float64)
    _dev(acc, "acc", torch.float32, 3 * np_)
    _dev(vel, "vel", torch.float32, 3 * np_)
    _dev(perm, "perm", torch.int64, np_)
    _dev(bin_offsets, "bin_offsets", torch.int32)
    _dev(status, "status", torch.int32, 4)
    g = make_grid(n, L)
    _check(_lib().ps_lagrangian_accel(ctypes.byref(g), _coef_type(coef_n), _ptr(coef_n),
                                      _ptr(scale_n), _ptr(coef_np1), _ptr(scale_np1),
                                      float(dt_field), np_, _ptr(pos), _ptr(perm),
                                      _ptr(bin_offsets), _brick_arr(brick), _ptr(acc),
                                      _ptr(vel), _ptr(status), _stream(stream)))


def ps_rk2_workspace_size(n, brick, np_: int, L=DEFAULT_L) -> int:
    g = make_grid(n, L)
    return int(_lib().ps_rk2_workspace_size(ctypes.byref(g), _brick_arr(brick), int(np_)))


def ps_rk2_step(coef_n: torch.Tensor, n, pos: torch.Tensor, dt: float,
                coef_np1: Optional[torch.Tensor] = None, scale_n: Optional[torch.Tensor] = None,
                scale_np1: Optional[torch.Tensor] = None, ids: Optional[torch.Tensor] = None,
                vel_out: Optional[torch.Tensor] = None, brick=None, rebin: int = 1,
                bin_offsets: Optional[torch.Tensor] = None, ws: Optional[torch.Tensor] = None,
                status: Optional[torch.Tensor] = None, L=DEFAULT_L, stream=None):
    """One Heun RK2 step (Sec. 2.1 / 4.3) of positions pos [3][np] in place.
    rebin: 0/False (bins given), 1/True (sort first), 2 (sort, and count the new
    positions' bins into ws), 3 (sort from the counts a previous 2 or 3 step
    left in ws)."""
    _check_coef_shape(coef_n, n)
    rebin = int(rebin)
    if rebin not in (0, 1, 2, 3):
        raise ValueError("rebin is 0, 1, 2 or 3")
    np_ = pos.shape[1]
    _dev(coef_n, "coef_n")
    _dev(coef_np1, "coef_np1", coef_n.dtype)
    _dev(pos, "pos", torch.float64)
    _dev(ids, "ids", torch.int64, np_)
    _dev(vel_out, "vel_out", torch.float32, 3 * np_)
    _dev(bin_offsets, "bin_offsets", torch.int32)
    _dev(ws, "ws")
    _dev(status, "status", torch.int32, 4)
    g = make_grid(n, L)
    ws_bytes = ws.numel() * ws.element_size() if ws is not None else 0
    if coef_np1 is not None and _coef_type(coef_np1) != _coef_type(coef_n):
        raise ValueError("coef_np1 must have the storage of coef_n")
    _check(_lib().ps_rk2_step(ctypes.byref(g), _coef_type(coef_n), _ptr(coef_n), _ptr(coef_np1),
                              _ptr(scale_n), _ptr(scale_np1), np_, _ptr(pos), _ptr(ids),
                              _ptr(vel_out), float(dt), _brick_arr(brick), rebin,
                              _ptr(bin_offsets), _ptr(ws), ws_bytes, _ptr(status),
                              _stream(stream)))


def ps_rk2_sort(n, brick, pos: torch.Tensor, pos_sorted: torch.Tensor,
                bin_offsets: torch.Tensor, ws: torch.Tensor, ids: Optional[torch.Tensor] = None,
                ids_sorted: Optional[torch.Tensor] = None, counted: bool = False,
                status: Optional[torch.Tensor] = None, L=DEFAULT_L, stream=None):
    """The sort of a binned Heun step: pos [3][np] (and ids) copied in bin order to
    pos_sorted (and ids_sorted), bounds to bin_offsets.  counted=True starts from
    the counts the last ps_rk2_step on ws took of the positions it wrote."""
    np_ = pos.shape[1]
    _dev(pos, "pos", torch.float64)
    _dev(pos_sorted, "pos_sorted", torch.float64, 3 * np_)
    _dev(ids, "ids", torch.int64, np_)
    _dev(ids_sorted, "ids_sorted", torch.int64, np_)
    _dev(bin_offsets, "bin_offsets", torch.int32)
    _dev(ws, "ws")
    _dev(status, "status", torch.int32, 4)
    g = make_grid(n, L)
    _check(_lib().ps_rk2_sort(ctypes.byref(g), _brick_arr(brick), np_, _ptr(pos), _ptr(ids),
                              1 if counted else 0, _ptr(pos_sorted), _ptr(ids_sorted),
                              _ptr(bin_offsets), _ptr(ws), ws.numel() * ws.element_size(),
                              _ptr(status), _stream(stream)))


# ------------------------------------------------------------------ helpers ----

def workspace(nbytes: int, device="cuda") -> torch.Tensor:
    """A 256-byte-aligned byte buffer (torch's caching allocator aligns to 512)."""
    t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)
    assert t.data_ptr() % 256 == 0
    return t


class SplineField:
    """Padded spline coefficients of a periodic field (Sec. 2.2 Operation 1)."""

    def __init__(self, coef: torch.Tensor, scale: Optional[torch.Tensor], n, L=DEFAULT_L):
        self.coef = coef
        self.scale = scale
        self.L = tuple(float(v) for v in L)
        self.n = tuple(int(v) for v in n)
        self.ncomp = _ncomp_of(coef)
        _check_coef_shape(coef, self.n)

    def padded(self) -> torch.Tensor:
        """[ncomp][nz+3][ny+3][nx+3] view (the row pitch tail dropped; for F32X4
        the component-major view of the interleaved nodes)."""
        if _is_node4(self.coef):
            return self.coef.permute(3, 0, 1, 2)[:3, ..., : self.n[0] + 3]
        return self.coef[..., : self.n[0] + 3]

    @classmethod
    def from_field(cls, field: torch.Tensor, coef_dtype=torch.float32, L=DEFAULT_L,
                   out: Optional["SplineField"] = None, ws: Optional[torch.Tensor] = None,
                   stream=None) -> "SplineField":
        n = grid_of_field(field)
        ncomp = field.shape[0]
        if out is None:
            coef = torch.empty(coef_shape(n, ncomp, coef_dtype),
                               dtype=_storage_dtype(coef_dtype), device=field.device)
            shp = scale_shape(n, ncomp, coef_dtype)
            scale = (torch.empty(shp, dtype=torch.float32, device=field.device)
                     if shp is not None else None)
            out = cls(coef, scale, n, L)
        need = ps_spline_coeffs_workspace_size(n, ncomp, coef_kind(out.coef), L)
        if need and (ws is None or ws.numel() < need):
            ws = workspace(need, field.device)
        ps_spline_coeffs(field, out.coef, out.scale, ws if need else None, L=L, stream=stream)
        return out

    def hessian(self, pos: torch.Tensor, status: Optional[torch.Tensor] = None,
                bins: Optional["Bins"] = None, stream=None) -> torch.Tensor:
        """Second derivatives at pos: [ncomp][6][np] (xx, yy, zz, xy, xz, yz); with
        `bins` of these positions, from each brick's staged halo."""
        h = torch.empty((self.ncomp, 6, pos.shape[1]), dtype=torch.float32, device=pos.device)
        ps_interp_hessian(self.coef, self.n, pos, h, scale=self.scale,
                          perm=bins.perm if bins is not None else None,
                          bin_offsets=bins.offsets if bins is not None else None,
                          brick=bins.brick if bins is not None else None, status=status,
                          L=self.L, stream=stream)
        return h

    def acceleration(self, pos: torch.Tensor, later: Optional["SplineField"] = None,
                     dt_field: float = 1.0, status: Optional[torch.Tensor] = None,
                     bins: Optional["Bins"] = None, stream=None) -> torch.Tensor:
        """Lagrangian acceleration du/dt + (u . grad) u at pos ([3][np]); du/dt from
        `later` (the field dt_field later) when given; with `bins` of these positions,
        from each brick's staged halo."""
        a = torch.empty((3, pos.shape[1]), dtype=torch.float32, device=pos.device)
        ps_lagrangian_accel(self.coef, self.n, pos, a,
                            coef_np1=later.coef if later is not None else None,
                            dt_field=dt_field, scale_n=self.scale,
                            scale_np1=later.scale if later is not None else None,
                            perm=bins.perm if bins is not None else None,
                            bin_offsets=bins.offsets if bins is not None else None,
                            brick=bins.brick if bins is not None else None,
                            status=status, L=self.L, stream=stream)
        return a

    def interp(self, pos: torch.Tensor, grad: bool = False, bins: Optional["Bins"] = None,
               status: Optional[torch.Tensor] = None, stream=None):
        np_ = pos.shape[1]
        vel = torch.empty((self.ncomp, np_), dtype=torch.float32, device=pos.device)
        g = (torch.empty((self.ncomp, 3, np_), dtype=torch.float32, device=pos.device)
             if grad else None)
        ps_interp(self.coef, self.n, pos, vel, scale=self.scale,
                  perm=bins.perm if bins is not None else None,
                  bin_offsets=bins.offsets if bins is not None else None,
                  brick=bins.brick if bins is not None else None, grad=g, status=status,
                  L=self.L, stream=stream)
        return (vel, g) if grad else vel


class Bins:
    """Result of a bin sort: offsets per brick and (optionally) a permutation."""

    def __init__(self, brick, offsets, bin_of, perm=None):
        self.brick = brick
        self.offsets = offsets
        self.bin_of = bin_of
        self.perm = perm


def bin_particles(n, brick, pos: torch.Tensor, L=DEFAULT_L, want_perm=True,
                  want_sorted=False, status=None, stream=None):
    if isinstance(brick, int):
        brick = (brick, brick, brick)
    np_ = pos.shape[1]
    nb = [-(-int(n[d]) // int(brick[d])) for d in range(3)]
    dev = pos.device
    bin_of = torch.empty(np_, dtype=torch.int32, device=dev)
    offsets = torch.empty(nb[0] * nb[1] * nb[2] + 1, dtype=torch.int32, device=dev)
    perm = torch.empty(np_, dtype=torch.int64, device=dev) if want_perm else None
    pos_sorted = torch.empty_like(pos) if want_sorted else None
    ws = workspace(ps_bin_workspace_size(n, brick, np_, L), dev)
    ps_bin_particles(n, brick, pos, bin_of, offsets, perm, pos_sorted, ws, status, L, stream)
    b = Bins(tuple(brick), offsets, bin_of, perm)
    return (b, pos_sorted) if want_sorted else b


class Tracker:
    """Particles advanced by Heun RK2 through a (frozen or time-dependent)
    spline field, bin-sorted into bricks every step.  With incremental=True
    each step's kernel counts the bins of the positions it writes, and the
    next step's sort starts from those counts (ps_rk2_step rebin 2, then 3).
    Positions changed between steps keep results exact (a particle outside
    its brick's halo reads its stencil from global memory); call reset_bins()
    after such a change to sort them afresh."""

    def __init__(self, field: SplineField, pos: torch.Tensor, brick=(8, 8, 8),
                 ids: Optional[torch.Tensor] = None, keep_velocity: bool = True,
                 incremental: bool = True):
        self.field = field
        self.pos = pos
        self.incremental = incremental
        self._counted = False  # ws holds the counts of the current positions
        self.brick = brick if brick is None or not isinstance(brick, int) else (brick,) * 3
        np_ = pos.shape[1]
        self.ids = ids if ids is not None else torch.arange(np_, dtype=torch.int64,
                                                            device=pos.device)
        self.vel = (torch.empty((3, np_), dtype=torch.float32, device=pos.device)
                    if keep_velocity else None)
        self.status = torch.zeros(4, dtype=torch.int32, device=pos.device)
        self.ws = None
        self.offsets = None
        if self.brick is not None:
            nb = [-(-field.n[d] // self.brick[d]) for d in range(3)]
            self.offsets = torch.empty(nb[0] * nb[1] * nb[2] + 1, dtype=torch.int32,
                                       device=pos.device)
            self.ws = workspace(ps_rk2_workspace_size(field.n, self.brick, np_, field.L),
                                pos.device)

    def reset_bins(self) -> None:
        """Forget the counts left by the last step (the next step sorts from the
        positions themselves)."""
        self._counted = False

    def step(self, dt: float, field_np1: Optional[SplineField] = None, rebin: bool = True,
             stream=None):
        f1 = field_np1
        mode = 0
        if rebin:
            mode = (3 if self._counted else 2) if self.incremental else 1
        ps_rk2_step(self.field.coef, self.field.n, self.pos, dt,
                    coef_np1=f1.coef if f1 is not None else None, scale_n=self.field.scale,
                    scale_np1=f1.scale if f1 is not None else None, ids=self.ids,
                    vel_out=self.vel, brick=self.brick, rebin=mode, bin_offsets=self.offsets,
                    ws=self.ws, status=self.status, L=self.field.L, stream=stream)
        self._counted = mode >= 2 and self.brick is not None


class InterpFn(torch.autograd.Function):
    """u = I(pos; spline(field)) with the hand-written adjoint:
    d/dpos via the spline derivative, d/dfield via scatter-add + the transposed
    (= same, symmetric) periodic solves."""

    @staticmethod
    def forward(ctx, pos: torch.Tensor, field: torch.Tensor, L=DEFAULT_L):
        sf = SplineField.from_field(field.detach().float(), torch.float32, L)
        vel = sf.interp(pos.detach())
        ctx.save_for_backward(pos)
        ctx.sf = sf
        ctx.field_dtype = field.dtype
        return vel

    @staticmethod
    def backward(ctx, g_vel):
        (pos,) = ctx.saved_tensors
        sf = ctx.sf
        g_vel = g_vel.contiguous().float()
        want_pos = ctx.needs_input_grad[0]
        want_field = ctx.needs_input_grad[1]
        g_pos = torch.empty_like(pos) if want_pos else None
        g_field = (torch.empty((sf.ncomp, sf.n[2], sf.n[1], sf.n[0]), dtype=torch.float32,
                               device=pos.device) if want_field else None)
        if want_pos or want_field:
            ps_interp_backward(sf.coef, sf.n, pos.detach(), g_vel, g_pos, g_field,
                               scale=sf.scale, L=sf.L)
        if g_field is not None:
            g_field = g_field.to(ctx.field_dtype)
        return g_pos, g_field, None


class BatchPlan:
    """Many periodic fields and their particle sets advanced together
    (ps_batch_plan / ps_batch_run).  `grids` is a list of (n, L) or n tuples;
    particles of all fields are one concatenated [3][np_total] array."""

    def __init__(self, grids, nps, coef_dtype=torch.float32, brick=(8, 8, 8),
                 tune_cache: Optional[str] = None):
        gl = []
        for g in grids:
            n, L = (g if isinstance(g[0], (tuple, list)) else (g, DEFAULT_L))
            gl.append(make_grid(n, L))
        self.grids = [(tuple(g.n), tuple(g.L)) for g in gl]
        self.nfields = len(gl)
        arr = (PsGrid * self.nfields)(*gl)
        nps_arr = (ctypes.c_int64 * self.nfields)(*[int(v) for v in nps])
        self.coef_dtype = coef_dtype
        self._plan = ctypes.c_void_p()
        _check(_lib().ps_batch_plan(self.nfields, arr, ctypes.cast(nps_arr, ctypes.c_void_p),
                                    _dt_code(coef_dtype), _brick_arr(brick),
                                    tune_cache.encode() if tune_cache else None,
                                    ctypes.byref(self._plan)))
        self.np_total = int(_lib().ps_batch_num_particles(self._plan))
        self.base = [int(_lib().ps_batch_particle_base(self._plan, f))
                     for f in range(self.nfields + 1)]
        self.ws_bytes = int(_lib().ps_batch_workspace_size(self._plan))
        self._ws = None

    def workspace(self, device="cuda") -> torch.Tensor:
        if self._ws is None or self._ws.device != torch.device(device):
            self._ws = workspace(self.ws_bytes, device)
        return self._ws

    def run(self, fields, pos: torch.Tensor, nsteps: int, dt: float, solve: bool = True,
            ids: Optional[torch.Tensor] = None, vel: Optional[torch.Tensor] = None,
            use_graph: bool = True, status: Optional[torch.Tensor] = None, stream=None):
        """fields: list of (field tensor or None, SplineField) per field."""
        assert len(fields) == self.nfields
        _dev(pos, "pos", torch.float64, 3 * self.np_total)
        _dev(ids, "ids", torch.int64, self.np_total)
        _dev(vel, "vel", torch.float32, 3 * self.np_total)
        _dev(status, "status", torch.int32, 4)
        bf = (_abi.PsBatchField * self.nfields)()
        for f, (fld, sf) in enumerate(fields):
            if fld is not None:
                _dev(fld, "field", torch.float32)
            _check_coef_shape(sf.coef, self.grids[f][0])
            bf[f].field = fld.data_ptr() if fld is not None else None
            bf[f].coef = sf.coef.data_ptr()
            bf[f].scale = sf.scale.data_ptr() if sf.scale is not None else None
        ws = self.workspace(pos.device)
        _check(_lib().ps_batch_run(self._plan, ctypes.cast(bf, ctypes.c_void_p), 1 if solve else 0,
                                   _ptr(pos), _ptr(ids), _ptr(vel), int(nsteps), float(dt),
                                   1 if use_graph else 0, _ptr(ws), self.ws_bytes, _ptr(status),
                                   _stream(stream)))

    def __del__(self):
        plan = getattr(self, "_plan", None)
        if plan is not None and plan.value:
            try:
                _lib().ps_plan_destroy(plan)
            except Exception:
                pass
            self._plan = None


def interp_autograd(pos: torch.Tensor, field: torch.Tensor, L=DEFAULT_L) -> torch.Tensor:
    return InterpFn.apply(pos, field, L)
