"""The paper's box2d workloads (Table III) at their full size, 38400^2 FP32,
in the configuration bench.py times (4 GiB budget, the planner's plan):

* all 640 steps: the out-of-core run equals the in-core run byte for byte,
  the boundary ring is untouched, and every value stays within the input's
  range (the weights are positive and sum to 1, so each update is a convex
  combination: a property that holds at any size);
* the oracle, cell by cell, on sampled dependency cones after k_off + 1 steps
  with the same k_off, k_on and chunking (two rounds, the second a residual):
  a 640-step cone reaches 640r cells, too wide for the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2309_08864_gb300 import inputs, so2dr
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

DIMS, T_FULL, BUDGET = (38400, 38400), 640, 4 << 30


def _plan(r, T, **kw):
    return so2dr.Plan(DIMS, r, "box", inputs.box2d_coeffs(r), T, budget_bytes=BUDGET, dtype="f32",
                      link_gbs=(171, 171), hbm_gbs=6781, **kw)


@pytest.mark.parametrize("r", [1, 4])
def test_box2d_full_size_640_steps_out_of_core_equals_in_core(r):
    import torch
    u = inputs.draw_box(1, DIMS, as_f32=True)
    host = torch.from_numpy(u).pin_memory()
    ref = host.clone().pin_memory()
    plan = _plan(r, T_FULL)
    info = plan.info
    assert info["arena_bytes"] <= BUDGET and info["chunks"] >= 2
    plan.run(host)
    ic = so2dr.Plan(DIMS, r, "box", inputs.box2d_coeffs(r), T_FULL, k_on=info["k_on"], k_off=info["k_off"],
                    budget_bytes=0, dtype="f32")
    ic.run(ref, in_core=True)
    assert torch.equal(host.view(torch.int32), ref.view(torch.int32)), "out-of-core != in-core"
    got = host.numpy()
    assert np.array_equal(got[:r], u[:r]) and np.array_equal(got[-r:], u[-r:])
    assert np.array_equal(got[:, :r], u[:, :r]) and np.array_equal(got[:, -r:], u[:, -r:])
    assert float(got.min()) >= float(u.min()) - 1e-6 and float(got.max()) <= float(u.max()) + 1e-6
    assert not np.array_equal(got[r:-r, r:-r], u[r:-r, r:-r])
    plan.close()
    ic.close()


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_box2d_full_size_sampled_cones(r):
    import torch
    full = _plan(r, T_FULL).info
    T = full["k_off"] + 1
    # the full plan's schedule (k_off, k_on, chunks, buffer options) for T steps
    plan = so2dr.Plan(DIMS, r, "box", inputs.box2d_coeffs(r), T, budget_bytes=BUDGET, dtype="f32",
                      tune_entry=full)
    for k in ("k_off", "k_on", "chunks", "lookahead", "out_slabs"):
        assert plan.info[k] == full[k], k
    host = torch.from_numpy(inputs.draw_box(1, DIMS, as_f32=True)).pin_memory()
    plan.run(host)
    starts = plan.chunks()
    rng = np.random.default_rng(r)
    w = 6
    n0, n1 = DIMS
    los = [(0, 0), (n0 - w, n1 - w), (0, n1 - w), (n0 - w, 0)]
    los += [(int(s) - w // 2, int(rng.integers(0, n1 - w))) for s in starts[1:-1]]
    los += [(int(rng.integers(0, n0 - w)), int(rng.integers(0, n1 - w))) for _ in range(4)]
    c = gu.compute_coeffs(inputs.box2d_coeffs(r), so2dr.F32)
    got_all = host.numpy()
    for lo in los:
        hi = (lo[0] + w, lo[1] + w)
        blo, bhi = oracle.cone_box(DIMS, lo, hi, r * T)
        ub = inputs.draw_box(1, DIMS, blo, bhi, as_f32=True).astype(np.float64)
        ref = oracle.run_cone(ub, c, r, oracle.BOX, T, blo, bhi, DIMS, lo, hi)
        got = got_all[lo[0]:hi[0], lo[1]:hi[1]].astype(np.float64)
        e = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        assert e <= 1e-5, (r, lo, e)
    plan.close()
