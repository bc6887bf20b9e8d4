"""so2dr_run_device_noalloc, the entry point for callers that cannot allocate
memory (graph capture, allocation-free real-time loops, runtimes that only
hand out pre-registered buffers): called through the C ABI twice in a row, it
must reproduce the in-core so2dr_run of the same plan, within the FP32
tolerance of the parity tests (the same kernels run, so in practice bit for
bit).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_2309_08864_gb300 import inputs, so2dr

pytestmark = pytest.mark.gpu


def _noalloc(lib, dims, coeffs, steps, k_on, d_in, d_out, stream):
    d = (ctypes.c_int64 * len(dims))(*dims)
    c = (ctypes.c_double * len(coeffs))(*coeffs)
    return lib.so2dr_run_device_noalloc(len(dims), d, 1, so2dr.STAR, c, len(coeffs), steps, k_on, so2dr.F32,
                                        ctypes.c_void_p(d_in.data_ptr()), ctypes.c_void_p(d_out.data_ptr()),
                                        ctypes.c_void_p(stream))


def test_noalloc_matches_the_in_core_run_on_two_calls():
    import torch
    lib = so2dr.load_library()
    dims, coeffs, steps, k_on = (48, 80, 132), [0.4] + [0.1] * 6, 10, 4   # launch depths 4, 4, 2
    stream = torch.cuda.current_stream().cuda_stream
    for call, seed in enumerate((1, 2)):
        u0 = inputs.draw_box(seed, dims, as_f32=True)
        ref = torch.from_numpy(u0.copy()).pin_memory()
        plan = so2dr.Plan(dims, 1, "star", coeffs, steps, min_chunks=1, k_on=k_on, k_off=steps,
                          budget_bytes=0, dtype="f32")
        plan.run(ref, in_core=True)
        plan.close()
        d_in = torch.from_numpy(u0).cuda()
        d_out = torch.full_like(d_in, float("nan"))
        assert _noalloc(lib, dims, coeffs, steps, k_on, d_in, d_out, stream) == so2dr.OK, \
            lib.so2dr_last_error().decode()
        torch.cuda.synchronize()
        got = d_out.cpu().numpy()
        want = ref.numpy()
        err = float(np.max(np.abs(got - want)) / np.max(np.abs(want)))
        assert err <= 1e-5, (call, err)
        assert torch.equal(d_in.cpu(), torch.from_numpy(u0)), "d_in must not be modified"


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    lib = so2dr.load_library()
    dims = (256, 256, 256)  # 64 MiB of FP32 > 32 MiB
    d_in = torch.empty(4, device="cuda")
    d_out = torch.empty(4, device="cuda")
    rc = _noalloc(lib, dims, [0.4] + [0.1] * 6, 4, 4, d_in, d_out, 0)
    assert rc == so2dr.E_INFEASIBLE
    assert "32 MiB" in lib.so2dr_last_error().decode()
