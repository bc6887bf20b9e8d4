"""Host-side failure detection (no GPU needed): every entry point rejects bad
arguments with a status code and a message before any CUDA call, and never
aborts.  Pointers below are never dereferenced: the calls fail their
argument checks first."""
import ctypes

import pytest

from paper_2309_08864_gb300 import so2dr

C7 = [0.4] + [0.1] * 6
FAKE = ctypes.c_void_p(1 << 20)      # aligned, never dereferenced


def lib():
    return so2dr.load_library()


def _dims(*d):
    return (ctypes.c_int64 * len(d))(*d)


def _coeffs(c):
    return (ctypes.c_double * len(c))(*c)


def test_bind_rejects_null_misaligned_arena_and_stream_count():
    p = so2dr.Plan((40, 36, 44), 1, "star", C7, 4, min_chunks=3, budget_bytes=0)
    L = lib()
    assert L.so2dr_bind(p._h, None, 1 << 20, None, 4) == so2dr.E_INVAL
    assert L.so2dr_bind(p._h, FAKE, 1 << 20, None, 2) == so2dr.E_INVAL
    assert L.so2dr_bind(p._h, ctypes.c_void_p((1 << 20) + 8), 1 << 20, None, 4) == so2dr.E_INVAL
    assert "aligned" in L.so2dr_last_error().decode()


@pytest.mark.parametrize("change,code", [
    (dict(ndim=4), so2dr.E_INVAL),
    (dict(radius=5), so2dr.E_INVAL),
    (dict(kind=so2dr.BOX), so2dr.E_UNSUPPORTED),      # 3D box
    (dict(dtype=7), so2dr.E_INVAL),
    (dict(steps=-1), so2dr.E_INVAL),
    (dict(k_on=0), so2dr.E_INVAL),
    (dict(ncoeffs=6), so2dr.E_INVAL),
    (dict(same=True), so2dr.E_INVAL),                 # d_in == d_out
    (dict(out=(1 << 20) + 4096), so2dr.E_INVAL),      # d_out overlaps d_in
    (dict(out=(2 << 20) + 8), so2dr.E_INVAL),         # d_out not 16-byte aligned
    (dict(dims=(4096, 64, 64)), so2dr.E_INFEASIBLE),  # 64 MiB > the 32 MiB scratch (two launches)
])
def test_noalloc_argument_checks(change, code):
    a = dict(ndim=3, dims=(16, 16, 16), radius=1, kind=so2dr.STAR, ncoeffs=7, steps=4, k_on=2, dtype=so2dr.F32,
             same=False, out=1 << 40)
    a.update(change)
    d = a["dims"]
    rc = lib().so2dr_run_device_noalloc(a["ndim"], _dims(*d), a["radius"], a["kind"], _coeffs(C7), a["ncoeffs"],
                                        a["steps"], a["k_on"], a["dtype"], FAKE,
                                        FAKE if a["same"] else ctypes.c_void_p(a["out"]), None)
    assert rc == code, lib().so2dr_last_error().decode()


@pytest.mark.parametrize("change,code", [
    (dict(table_len=False), so2dr.E_INVAL),
    (dict(arena=None), so2dr.E_INVAL),
    (dict(max_candidates=0), so2dr.E_INVAL),
    (dict(repeats=0), so2dr.E_INVAL),
    (dict(kind=so2dr.VARCOEF_STAR), so2dr.E_UNSUPPORTED),
    (dict(budget=0), so2dr.E_INVAL),
    (dict(nstreams=2), so2dr.E_INVAL),
    (dict(budget=4096), so2dr.E_INFEASIBLE),          # the problem is checked before any device work
])
def test_autotune_argument_checks(change, code):
    a = dict(table_len=True, arena=FAKE, max_candidates=4, repeats=1, kind=so2dr.STAR, budget=16 << 20, nstreams=4)
    a.update(change)
    n = ctypes.c_int()
    tab = (so2dr.TuneEntry * 8)()
    rc = lib().so2dr_autotune(3, _dims(256, 128, 128), 1, a["kind"], _coeffs(C7), 7, 16, 1, 0, 0, a["budget"],
                              so2dr.F32, a["arena"], None, a["nstreams"], FAKE, a["max_candidates"], a["repeats"],
                              tab, 8, ctypes.byref(n) if a["table_len"] else None, None)
    assert rc == code, lib().so2dr_last_error().decode()


def test_plan_rejects_bad_problems_with_messages():
    L = lib()
    h = ctypes.c_void_p()
    assert L.so2dr_plan(ctypes.byref(h), 3, _dims(16, 16, 16), 1, so2dr.STAR, _coeffs(C7), 7, 4, 0, 0, 0, 0,
                        so2dr.F32) == so2dr.E_INVAL                               # min_chunks 0
    assert "min_chunks" in L.so2dr_last_error().decode()
    assert L.so2dr_plan(ctypes.byref(h), 3, _dims(16, 16, 16), 1, so2dr.STAR, _coeffs([float("nan")] * 7), 7, 4,
                        1, 0, 0, 0, so2dr.F32) == so2dr.E_INVAL                   # non-finite weight
    assert L.so2dr_plan(ctypes.byref(h), 3, _dims(512, 512, 512), 1, so2dr.STAR, _coeffs(C7), 7, 4, 1, 0, 0,
                        1 << 20, so2dr.F32) == so2dr.E_INFEASIBLE                 # 1 MiB cannot hold a 1 MiB plane
    assert not h.value
