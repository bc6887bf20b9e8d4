"""The C-ABI library loads and exports every entry point include/so2dr.h
declares; host-only calls behave as documented (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2309_08864_gb300 import build, so2dr

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "so2dr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(so2dr_\w+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(so2dr.SYMBOLS) | (set(names) - set(so2dr.SYMBOLS))
    for n in so2dr.SYMBOLS:
        assert n in names, n


def test_version_and_status_strings():
    lib = so2dr.load_library()
    assert lib.so2dr_abi_version() == 5
    for code in range(0, -10, -1):
        s = lib.so2dr_strerror(code).decode()
        assert s and s != "unknown status"
    assert lib.so2dr_strerror(-99).decode() == "unknown status"


def test_run_before_bind_is_an_error_not_a_crash():
    p = so2dr.Plan((32, 32), 1, "star", [0.2] * 5, 4, min_chunks=2, k_on=2, k_off=4, budget_bytes=0)
    buf = ctypes.create_string_buffer(32 * 32 * 4)
    rc = so2dr.load_library().so2dr_run(p._h, ctypes.cast(buf, ctypes.c_void_p), None, 0, None)
    assert rc == so2dr.E_NOT_BOUND
    assert "bound" in so2dr.load_library().so2dr_last_error().decode()


def test_null_arguments_are_rejected():
    lib = so2dr.load_library()
    assert lib.so2dr_plan_info(None, None) == so2dr.E_INVAL
    n = ctypes.c_int64()
    assert lib.so2dr_plan_ops(None, 0, None, 0, ctypes.byref(n)) == so2dr.E_INVAL
    lib.so2dr_destroy(None)  # no-op
