"""Seeded synthetic inputs (no stencil arithmetic here).

Every array the tests, the smoke check and the benchmark feed to either the
CUDA path or the FP64 oracle comes from this module, so both sides see the
same bytes.  The draws come from a counter-based SplitMix64 stream (see
csrc/inputs_gen.c); storage rounding is double -> float32 (round to nearest
even), then float32 -> bfloat16 / float16 (round to nearest even).

Seeds used by the workloads: 1 = initial field, 2 = target field,
100 + f = face-coefficient field f, 7 = radius-4 coefficient table,
11 + r = box2d{r}r coefficient table,
1000 + k = finite-difference direction k.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "inputs_gen.c")
_LIB = os.path.join(_HERE, "libso2dr_inputs.so")
_lib = None

F64, F32, BF16, F16 = 0, 1, 2, 3
DTYPE_NAMES = {F64: "f64", F32: "f32", BF16: "bf16", F16: "f16"}
ITEMSIZE = {F64: 8, F32: 4, BF16: 2, F16: 2}


def build(force: bool = False) -> str:
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", _SRC,
                    "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.so2dr_gen_box.argtypes = [ctypes.c_uint64, i64p, i64p, i64p, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_void_p]
        lib.so2dr_gen_box.restype = None
        _lib = lib
    return _lib


def _pad3(v, fill):
    v = list(v)
    return v + [fill] * (3 - len(v))


def draw_box(seed, shape, lo=None, hi=None, dist="uniform", a=0.0, b=1.0,
             out=None, as_f32=False):
    """Values of the full grid `shape` on the sub-box [lo, hi) (default: all),
    as float64 (or float32 with as_f32).  dist 'uniform' -> [a, b);
    'normal' -> mean a, deviation b.  `out` may be a preallocated contiguous
    array (numpy or anything exposing a data pointer via __array_interface__)."""
    nd = len(shape)
    if nd > 3:
        raise ValueError("draw_box handles grids of up to 3 dimensions")
    lo = [0] * nd if lo is None else list(lo)
    hi = list(shape) if hi is None else list(hi)
    ext = tuple(h - l for l, h in zip(lo, hi))
    dt = np.float32 if as_f32 else np.float64
    if out is None:
        out = np.empty(ext, dtype=dt)
    assert out.dtype == dt and out.flags["C_CONTIGUOUS"] and out.size == int(np.prod(ext))
    dims3 = (ctypes.c_int64 * 3)(*_pad3(shape, 1))
    lo3 = (ctypes.c_int64 * 3)(*_pad3(lo, 0))
    hi3 = (ctypes.c_int64 * 3)(*_pad3(hi, 1))
    _load().so2dr_gen_box(seed, dims3, lo3, hi3, 0 if dist == "uniform" else 1,
                          a, b, 1 if as_f32 else 0, out.ctypes.data)
    return out


def f32_to_bf16_bits(x32: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 (nearest even); returns the uint16 bit patterns."""
    u = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return u.astype(np.uint16)


def bf16_bits_to_f64(b: np.ndarray) -> np.ndarray:
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def to_storage(x64: np.ndarray, dtype: int) -> np.ndarray:
    """Round float64 values to the storage dtype.  Returns the storage array
    (float64 / float32 / uint16 bit patterns for bf16 / float16)."""
    if dtype == F64:
        return np.ascontiguousarray(x64, dtype=np.float64)
    x32 = np.ascontiguousarray(x64, dtype=np.float64).astype(np.float32)
    if dtype == F32:
        return x32
    if dtype == BF16:
        return f32_to_bf16_bits(x32)
    if dtype == F16:
        return x32.astype(np.float16)
    raise ValueError(dtype)


def storage_to_f64(s: np.ndarray, dtype: int) -> np.ndarray:
    if dtype == BF16:
        return bf16_bits_to_f64(s)
    return np.asarray(s).astype(np.float64)


def zero_ring(x: np.ndarray, r: int) -> np.ndarray:
    """Set the boundary ring of width r to zero (the 2D Jacobi workload keeps a
    zero ring and draws only the interior)."""
    for a in range(x.ndim):
        sl = [slice(None)] * x.ndim
        sl[a] = slice(0, r)
        x[tuple(sl)] = 0
        sl[a] = slice(x.shape[a] - r, x.shape[a])
        x[tuple(sl)] = 0
    return x


def box2d_coeffs(r: int, seed: int = 11) -> np.ndarray:
    """(2r+1)^2 independent draws in [0.5, 1.5) normalised in FP64 to sum to 1,
    row-major from offset (-r, -r): the weights of the box2d{r}r workloads,
    whose values the paper does not give."""
    c = draw_box(seed + r, ((2 * r + 1) ** 2,), dist="uniform", a=0.5, b=1.5)
    return c / c.sum()


def radius4_star_coeffs(seed: int = 7, ndim: int = 3) -> np.ndarray:
    """25 independent draws in [0.5, 1.5) normalised in FP64 to sum to 1
    (coefficient-table order of the star stencil)."""
    n = 1 + 2 * 4 * ndim
    c = draw_box(seed, (n,), dist="uniform", a=0.5, b=1.5)
    return c / c.sum()
