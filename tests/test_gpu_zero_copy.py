"""Run mode 3 of so2dr_run, zero-copy input (a GB300 option, not in the
paper): no host-to-device copy of the grid; the first launch of each chunk
reads the chunk's new planes from the pinned host grid through its device
mapping (NVLink-C2C) and writes them into the circular buffer for the next
chunk.  It must give the in-core result byte for byte, and the FP64 oracle's
within the storage type's tolerance."""
import numpy as np
import pytest

import oracle
from paper_2309_08864_gb300 import inputs, so2dr
from tests import gpu_util as gu
from tests.test_gpu_parity import TOL, _coeffs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,r,T,dmin,kon,koff,budget,dtype", [
    ((72, 70, 132), 1, 12, 5, 4, 8, 0, so2dr.F32),          # two x tiles, ragged y, residual round
    ((61, 37, 48), 1, 13, 4, 3, 5, 0, so2dr.F32),           # depths 3 and 2
    ((57, 46, 136), 1, 13, 4, 4, 8, 0, so2dr.BF16),         # 16-bit boxes start 4 columns in
    ((57, 46, 136), 1, 11, 4, 3, 6, 0, so2dr.F16),
    ((52, 45, 136), 2, 7, 3, 2, 4, 0, so2dr.F32),           # radius 2
    ((64, 70, 140), 4, 6, 3, 1, 3, 0, so2dr.F32),           # radius 4
    ((96, 64, 128), 1, 16, 8, 4, 16, 4 << 20, so2dr.F32),   # budget-bound chunking
])
def test_zero_copy_matches_in_core(dims, r, T, dmin, kon, koff, budget, dtype):
    import torch
    c = [0.4] + [0.1] * 6 if r == 1 else _coeffs(3, r, "star")
    u64 = inputs.draw_box(1, dims)
    st = inputs.to_storage(u64, dtype)
    plan = so2dr.Plan(dims, r, "star", c, T, min_chunks=dmin, k_on=kon, k_off=koff, budget_bytes=budget,
                      dtype=dtype)
    assert plan.info["zero_copy"] == 1
    zc = gu.pinned_from_storage(st.copy(), dtype)
    ic = gu.pinned_from_storage(st.copy(), dtype)
    s3 = plan.run(zc, in_core=3)
    plan.run(ic, in_core=True)
    assert s3["h2d_bytes"] == 0       # nothing went through the copy engines to the device
    assert torch.equal(zc.view(torch.uint8), ic.view(torch.uint8)), "zero-copy != in-core"
    ref = oracle.run(inputs.storage_to_f64(st, dtype), gu.compute_coeffs(c, dtype), r, 0, T)
    assert gu.rel_linf(gu.storage_of(zc, dtype), ref) <= TOL[dtype]
    # a second run on the same grid (in place), against the copy-engine pipeline
    oc = zc.clone().pin_memory()
    plan.run(zc, in_core=3)
    plan.run(oc, in_core=False)
    assert torch.equal(zc.view(torch.uint8), oc.view(torch.uint8))
    plan.close()


@pytest.mark.parametrize("split", ["grid", "rounds"])
@pytest.mark.parametrize("dims,r,kon,koff,dtype", [
    ((72, 70, 132), 1, 4, 8, so2dr.F32),
    ((57, 46, 136), 1, 3, 6, so2dr.BF16),
    ((64, 70, 140), 4, 1, 3, so2dr.F32),
])
def test_zero_copy_work_splits(dims, r, kon, koff, dtype, split, monkeypatch):
    """Zero-copy launches under either work split: in the round split a CTA's
    pieces mix planes staged from the host and planes from the circular
    buffer, and the pieces come from the launch's counter."""
    import torch
    monkeypatch.setenv("SO2DR_WORK_SPLIT", split)
    c = [0.4] + [0.1] * 6 if r == 1 else _coeffs(3, r, "star")
    st = inputs.to_storage(inputs.draw_box(2, dims), dtype)
    plan = so2dr.Plan(dims, r, "star", c, 2 * koff + kon, min_chunks=4, k_on=kon, k_off=koff, budget_bytes=0,
                      dtype=dtype)
    zc = gu.pinned_from_storage(st.copy(), dtype)
    ic = gu.pinned_from_storage(st.copy(), dtype)
    plan.run(zc, in_core=3)
    plan.run(ic, in_core=True)
    plan.close()
    assert torch.equal(zc.view(torch.uint8), ic.view(torch.uint8)), "zero-copy != in-core"
