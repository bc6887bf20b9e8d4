"""Measured autotune (so2dr_autotune) on the GPU: it measures the link and
HBM rates, times the model's best candidates and returns them sorted by
measured time; the winner's plan, built with so2dr_plan_tuned, computes the
same bytes as the in-core run and matches the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2309_08864_gb300 import inputs, so2dr
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

C7 = [0.4] + [0.1] * 6


@pytest.mark.parametrize("dims,T,budget,dtype", [((160, 96, 128), 12, 6 << 20, so2dr.F32),
                                                 ((130, 64, 96), 9, 2 << 20, so2dr.BF16)])
def test_autotune_ranks_measured_candidates_and_the_winner_is_exact(dims, T, budget, dtype):
    import torch
    scratch = torch.empty(int(np.prod(dims)) * (4 if dtype == so2dr.F32 else 2), dtype=torch.uint8).pin_memory()
    table, link = so2dr.autotune(dims, 1, "star", C7, T, budget, dtype, scratch=scratch, max_candidates=5,
                                 repeats=2)
    assert all(x > 0 for x in link), link
    timed = [e for e in table if e["measured_ms"] >= 0]
    assert len(timed) == min(5, len(table))
    assert [e["measured_ms"] for e in timed] == sorted(e["measured_ms"] for e in timed)
    assert all(e["status"] == 0 for e in timed)
    untimed = [e["predicted_ms"] for e in table[len(timed):]]
    assert untimed == sorted(untimed)
    # the five timed entries are the model's five best under the measured rates
    ranked = so2dr.candidates(dims, 1, "star", C7, T, budget_bytes=budget, dtype=dtype,
                              link_gbs=link[:2], hbm_gbs=link[2])
    key = lambda e: (e["k_off"], e["k_on"], e["chunks"], e["lookahead"], e["out_slabs"])
    assert {key(e) for e in timed} == {key(e) for e in ranked[:len(timed)]}

    u64 = inputs.draw_box(1, dims)
    st = inputs.to_storage(u64, dtype)
    plan = so2dr.Plan(dims, 1, "star", C7, T, budget_bytes=budget, dtype=dtype, tune_entry=table[0])
    assert key(plan.info) == key(table[0])
    ooc = gu.pinned_from_storage(st.copy(), dtype)
    ic = gu.pinned_from_storage(st.copy(), dtype)
    plan.run(ooc)
    plan.run(ic, in_core=True)
    assert torch.equal(ooc.view(torch.uint8), ic.view(torch.uint8))
    ref = oracle.run(inputs.storage_to_f64(st, dtype), gu.compute_coeffs(C7, dtype), 1, 0, T)
    err = gu.rel_linf(gu.storage_of(ooc, dtype), ref)
    assert err <= (1e-5 if dtype == so2dr.F32 else 2e-2), err


def test_measure_link_reports_every_rate():
    r = so2dr.measure_link(64 << 20, sm_ctas=64, repeats=2)
    assert set(r) == set(so2dr.LINK_KEYS)
    for k, v in r.items():
        assert v > 1.0, (k, v)   # GB/s; pinned buffers from torch are mapped on this platform
    assert r["hbm"] > r["ce_h2d"]

