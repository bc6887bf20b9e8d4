"""so2dr_run_device_noalloc, the entry point for callers that cannot allocate
memory (graph capture, allocation-free real-time loops, runtimes that only
hand out pre-registered buffers): called through the C ABI twice in a row, it
must reproduce the in-core so2dr_run of the same problem bit for bit (the same
kernels run in the same launch depths).  Cases cover odd and even launch
counts (the first launch writes the scratch array or d_out), one launch (no
scratch, any size), zero steps (a copy), the 2D box stencil and FP64 / BF16
storage.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_2309_08864_gb300 import inputs, so2dr
from tests import gpu_util as gu
from tests.test_gpu_parity import _coeffs

pytestmark = pytest.mark.gpu

C7 = [0.4] + [0.1] * 6


def _noalloc(lib, dims, r, kind, coeffs, steps, k_on, dtype, d_in, d_out, stream):
    d = (ctypes.c_int64 * len(dims))(*dims)
    c = (ctypes.c_double * len(coeffs))(*coeffs)
    return lib.so2dr_run_device_noalloc(len(dims), d, r, kind, c, len(coeffs), steps, k_on, dtype,
                                        ctypes.c_void_p(d_in.data_ptr()), ctypes.c_void_p(d_out.data_ptr()),
                                        ctypes.c_void_p(stream))


@pytest.mark.parametrize("dims,r,kind,coeffs,steps,k_on,dtype", [
    ((48, 80, 132), 1, "star", C7, 10, 4, so2dr.F32),                 # launches 4, 4, 2
    ((48, 80, 132), 1, "star", C7, 8, 4, so2dr.F32),                  # launches 4, 4
    ((40, 56, 136), 1, "star", C7, 8, 3, so2dr.BF16),                 # launches 3, 3, 2 (16-bit)
    ((70, 300), 2, "box", _coeffs(2, 2, "box"), 6, 2, so2dr.F64),     # 2D box, generic FP64 kernel
    ((90, 300), 1, "star", [0.2] * 5, 4, 4, so2dr.F32),               # one launch: no scratch
    ((48, 80, 132), 1, "star", C7, 0, 4, so2dr.F32),                  # zero steps: a copy
])
def test_noalloc_matches_the_in_core_run_on_two_calls(dims, r, kind, coeffs, steps, k_on, dtype):
    import torch
    lib = so2dr.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    kcode = so2dr.STAR if kind == "star" else so2dr.BOX
    for call, seed in enumerate((1, 2)):
        st = inputs.to_storage(inputs.draw_box(seed, dims), dtype)
        ref = gu.pinned_from_storage(st.copy(), dtype)
        if steps > 0:
            plan = so2dr.Plan(dims, r, kind, coeffs, steps, min_chunks=1, k_on=k_on, k_off=steps,
                              budget_bytes=0, dtype=dtype)
            plan.run(ref, in_core=True)
            plan.close()
        src = gu.pinned_from_storage(st.copy(), dtype)
        d_in = src.cuda()
        d_out = torch.full_like(d_in, float("nan"))
        assert _noalloc(lib, dims, r, kcode, list(coeffs), steps, k_on, dtype, d_in, d_out, stream) == so2dr.OK, \
            lib.so2dr_last_error().decode()
        torch.cuda.synchronize()
        assert torch.equal(d_out.cpu().view(torch.uint8), ref.view(torch.uint8)), call
        assert torch.equal(d_in.cpu().view(torch.uint8), src.view(torch.uint8)), "d_in must not be modified"


def test_noalloc_one_launch_takes_grids_beyond_its_scratch():
    import torch
    lib = so2dr.load_library()
    dims, steps, k_on = (256, 256, 256), 3, 4     # 64 MiB of FP32 in one launch
    u0 = inputs.draw_box(5, dims, as_f32=True)
    ref = torch.from_numpy(u0.copy()).pin_memory()
    plan = so2dr.Plan(dims, 1, "star", C7, steps, min_chunks=1, k_on=k_on, k_off=steps, budget_bytes=0, dtype="f32")
    plan.run(ref, in_core=True)
    plan.close()
    d_in = torch.from_numpy(u0).cuda()
    d_out = torch.empty_like(d_in)
    stream = torch.cuda.current_stream().cuda_stream
    assert _noalloc(lib, dims, 1, so2dr.STAR, C7, steps, k_on, so2dr.F32, d_in, d_out, stream) == so2dr.OK
    torch.cuda.synchronize()
    assert torch.equal(d_out.cpu(), ref)


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    lib = so2dr.load_library()
    dims = (256, 256, 256)  # 64 MiB of FP32 > 32 MiB, in two launches
    d_in = torch.empty(dims, device="cuda")
    d_out = torch.empty(dims, device="cuda")
    rc = _noalloc(lib, dims, 1, so2dr.STAR, C7, 8, 4, so2dr.F32, d_in, d_out, 0)
    assert rc == so2dr.E_INFEASIBLE
    assert "32 MiB" in lib.so2dr_last_error().decode()
