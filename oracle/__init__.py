"""FP64 CPU oracle for the SO2DR stencil path (Sec. II-A definition of a stencil
update; Sec. IV only reorganises it, so the oracle is the plain definition).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product package.  It shares no code
with the CUDA path.

Parity: pinned by tests/test_oracle_pins.py against closed forms (sin-mode
eigenvalues of the Jacobi operator with a zero ring), invariants (constant
fields, linearity, first moments, the adjoint dot-product identity), a library
routine (scipy.ndimage.correlate for one step), brute-force matrix powers on
tiny grids and FP64 finite differences of the loss.
"""
import ctypes
import os

import numpy as np

from . import build as _build

STAR, BOX, VARCOEF_STAR = 0, 1, 2

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_num_offsets.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.oracle_offsets.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int)]
        lib.oracle_run_const.argtypes = [ctypes.c_int, i64p, ctypes.c_int, ctypes.c_int,
                                         dp, dp, ctypes.c_int64]
        lib.oracle_run_varcoef.argtypes = [ctypes.c_int, i64p, dp, dp, ctypes.c_int64]
        lib.oracle_apply_varcoef.argtypes = [ctypes.c_int, i64p, dp, dp, dp]
        lib.oracle_apply_varcoef_transpose.argtypes = [ctypes.c_int, i64p, dp, dp, dp]
        lib.oracle_adjoint_varcoef.argtypes = [ctypes.c_int, i64p, dp, dp, dp, ctypes.c_int64,
                                               ctypes.c_int64, dp, dp, dp]
        lib.oracle_loss.argtypes = [ctypes.c_int64, dp, dp]
        lib.oracle_loss.restype = ctypes.c_double
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dims(shape):
    return (ctypes.c_int64 * len(shape))(*shape)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def offsets(ndim: int, radius: int, kind: int) -> np.ndarray:
    """Offsets in coefficient-table order, shape (npts, ndim)."""
    lib = _load()
    n = lib.oracle_num_offsets(ndim, radius, kind)
    if n <= 0:
        raise ValueError("invalid stencil")
    buf = (ctypes.c_int * (3 * n))()
    lib.oracle_offsets(ndim, radius, kind, buf)
    return np.array(buf, dtype=np.int64).reshape(n, 3)[:, :ndim]


def run(u0, coeffs, radius: int, kind: int, steps: int) -> np.ndarray:
    """u_T of the constant-coefficient sweep with a fixed ring of width radius."""
    u = _f64(u0).copy()
    c = _f64(coeffs)
    lib = _load()
    if c.size != lib.oracle_num_offsets(u.ndim, radius, kind):
        raise ValueError("coefficient count does not match the stencil")
    rc = lib.oracle_run_const(u.ndim, _dims(u.shape), radius, kind, _dp(c), _dp(u), steps)
    if rc:
        raise RuntimeError("oracle_run_const failed: %d" % rc)
    return u


def run_varcoef(u0, faces, steps: int) -> np.ndarray:
    """u_T of the variable-coefficient 7-point (3D) / 5-point (2D) sweep.
    faces has shape (2*ndim,) + u0.shape."""
    u = _f64(u0).copy()
    f = _f64(faces)
    assert f.shape == (2 * u.ndim,) + u.shape
    rc = _load().oracle_run_varcoef(u.ndim, _dims(u.shape), _dp(f), _dp(u), steps)
    if rc:
        raise RuntimeError("oracle_run_varcoef failed: %d" % rc)
    return u


def apply_varcoef(u, faces) -> np.ndarray:
    u = _f64(u)
    f = _f64(faces)
    out = np.empty_like(u)
    _load().oracle_apply_varcoef(u.ndim, _dims(u.shape), _dp(f), _dp(u), _dp(out))
    return out


def apply_varcoef_transpose(lam, faces) -> np.ndarray:
    lam = _f64(lam)
    f = _f64(faces)
    out = np.empty_like(lam)
    _load().oracle_apply_varcoef_transpose(lam.ndim, _dims(lam.shape), _dp(f), _dp(lam), _dp(out))
    return out


def adjoint_varcoef(u0, faces, target, steps: int, ckpt_every: int = 8):
    """Returns (loss, dL/du0, dL/dfaces) for L = 1/2 ||u_T - target||^2."""
    u0 = _f64(u0)
    f = _f64(faces)
    tg = _f64(target)
    gu = np.empty_like(u0)
    gf = np.empty_like(f)
    loss = ctypes.c_double(0.0)
    rc = _load().oracle_adjoint_varcoef(u0.ndim, _dims(u0.shape), _dp(f), _dp(u0), _dp(tg),
                                        steps, ckpt_every, _dp(gu), _dp(gf), ctypes.byref(loss))
    if rc:
        raise RuntimeError("oracle_adjoint_varcoef failed: %d" % rc)
    return loss.value, gu, gf


def loss(u, target) -> float:
    u = _f64(u)
    tg = _f64(target)
    return _load().oracle_loss(u.size, _dp(u), _dp(tg))


def cone_box(shape, lo, hi, reach):
    """Sub-box [lo - reach, hi + reach) clipped to the grid, for the
    dependency-cone evaluation: by locality, a cell's value after T steps of a
    radius-r stencil depends only on cells within r*T of it (clipped at the
    fixed ring), so running the plain oracle on this machine (its own outer ring
    held fixed) gives exact values on [lo, hi) when reach >= r*T."""
    blo = [max(0, l - reach) for l in lo]
    bhi = [min(n, h + reach) for n, h in zip(shape, hi)]
    return blo, bhi


def run_cone(u0_box, coeffs, radius, kind, steps, box_lo, box_hi, shape, lo, hi):
    """Exact u_T on [lo, hi) from u0 restricted to the cone box (see cone_box).
    Only valid when the box was produced by cone_box(..., reach >= radius*steps)."""
    u = run(u0_box, coeffs, radius, kind, steps)
    sl = tuple(slice(l - bl, h - bl) for l, h, bl in zip(lo, hi, box_lo))
    return u[sl]
