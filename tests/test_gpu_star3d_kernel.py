"""The 3D star temporal-blocking kernel (TMA-staged register streaming)
against the generic kernel and the FP64 oracle.

Both kernels sum each cell's products in the same fixed order (axis 0 from
-R, the centre, the in-plane axes, axis 0 up to +R), so their results agree
bit for bit for every radius, fused depth and storage type; the boxes cover
ragged tiles in x and y, 16-bit boxes that start 4 columns before the tile,
and axis-0 segments."""
import numpy as np
import pytest

import oracle
from paper_2309_08864_gb300 import inputs, so2dr
from tests import gpu_util as gu
from tests.test_gpu_parity import TOL, _coeffs, check_case

pytestmark = pytest.mark.gpu

CASES = [(1, 1), (1, 2), (1, 3), (1, 4), (2, 1), (2, 2), (3, 1), (3, 2), (4, 1), (4, 2)]


@pytest.mark.parametrize("dtype", [so2dr.F32, so2dr.BF16, so2dr.F16])
@pytest.mark.parametrize("r,kon", CASES)
def test_star3d_kernel_matches_generic_kernel_bitwise(r, kon, dtype, monkeypatch):
    import torch
    dims, T = (41, 70, 264), kon + 1   # one k_on-deep launch and a depth-1 residual
    st = inputs.to_storage(inputs.draw_box(3, dims), dtype)
    c = _coeffs(3, r, "star")
    plan = so2dr.Plan(dims, r, "star", c, T, k_on=kon, k_off=T, budget_bytes=0, dtype=dtype)
    fast = gu.pinned_from_storage(st.copy(), dtype)
    plan.run(fast, in_core=True)
    monkeypatch.setenv("SO2DR_GENERIC_KERNEL", "1")
    generic = gu.pinned_from_storage(st.copy(), dtype)
    plan.run(generic, in_core=True)
    plan.close()
    assert torch.equal(fast.view(torch.uint8), generic.view(torch.uint8))
    ref = oracle.run(inputs.storage_to_f64(st, dtype), gu.compute_coeffs(c, dtype), r, 0, T)
    assert gu.rel_linf(gu.storage_of(fast, dtype), ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype,kon,koff,T", [(so2dr.BF16, 4, 8, 13), (so2dr.F16, 3, 6, 11),
                                              (so2dr.BF16, 2, 5, 7)])
def test_star3d_16bit_out_of_core(dtype, kon, koff, T):
    """16-bit storage through the out-of-core pipeline: equal to the in-core
    run byte for byte, and within the format's rounding of the oracle."""
    check_case((57, 46, 136), 1, "star", [0.4] + [0.1] * 6, T, dtype, 4, kon, koff, 0)


@pytest.mark.parametrize("split", ["grid", "rounds"])
@pytest.mark.parametrize("dims", [(41, 70, 264), (150, 96, 512)])
@pytest.mark.parametrize("r,kon", CASES)
def test_star3d_work_splits_match_generic_kernel_bitwise(r, kon, dims, split, monkeypatch):
    """Both work splits of a launch -- one tile and axis-0 segment per CTA, or
    the (tile, output plane) pairs cut into one contiguous range per CTA, whose
    pieces start and end inside tiles -- give the generic kernel's bytes."""
    import torch
    T = kon + 1
    dtype = so2dr.F32 if r != 2 else so2dr.BF16
    st = inputs.to_storage(inputs.draw_box(5, dims), dtype)
    c = _coeffs(3, r, "star")
    plan = so2dr.Plan(dims, r, "star", c, T, k_on=kon, k_off=T, budget_bytes=0, dtype=dtype)
    monkeypatch.setenv("SO2DR_WORK_SPLIT", split)
    fast = gu.pinned_from_storage(st.copy(), dtype)
    plan.run(fast, in_core=True)
    monkeypatch.setenv("SO2DR_GENERIC_KERNEL", "1")
    generic = gu.pinned_from_storage(st.copy(), dtype)
    plan.run(generic, in_core=True)
    plan.close()
    assert torch.equal(fast.view(torch.uint8), generic.view(torch.uint8))


@pytest.mark.parametrize("split", ["grid", "rounds"])
def test_star3d_work_splits_out_of_core(split, monkeypatch):
    """The out-of-core pipeline under either work split equals the in-core
    run byte for byte (trapezoid launches of every size, ragged chunks)."""
    monkeypatch.setenv("SO2DR_WORK_SPLIT", split)
    check_case((97, 70, 264), 1, "star", [0.4] + [0.1] * 6, 13, so2dr.F32, 5, 4, 8, 0)
