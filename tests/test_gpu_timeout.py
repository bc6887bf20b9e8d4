"""Failure detection without a GPU fault: every wait of the executor polls
completion events against a deadline (SO2DR_TIMEOUT_S) and returns
SO2DR_E_TIMEOUT instead of blocking.  Here the deadline is made to run out
on purpose (1 ns) while the work is certainly still running; the call reports
the timeout, the work already queued still completes, and the context stays
usable: the next run, with the normal deadline, succeeds and the two runs
together equal one in-core run of twice the steps."""
import pytest

from paper_2309_08864_gb300 import inputs, so2dr
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def test_deadline_reports_a_timeout_and_the_context_stays_usable(monkeypatch):
    import torch
    dims, T = (384, 384, 384), 32
    st = inputs.to_storage(inputs.draw_box(1, dims), so2dr.F32)
    plan = so2dr.Plan(dims, 1, "star", [0.4] + [0.1] * 6, T, k_on=4, k_off=8, budget_bytes=64 << 20, dtype="f32")
    plan.bind()
    host = gu.pinned_from_storage(st.copy(), so2dr.F32)
    monkeypatch.setenv("SO2DR_TIMEOUT_S", "1e-9")
    with pytest.raises(so2dr.So2drError) as ex:
        plan.run(host)
    assert ex.value.code == so2dr.E_TIMEOUT
    monkeypatch.delenv("SO2DR_TIMEOUT_S")
    torch.cuda.synchronize()          # the queued run completes on its own
    plan.run(host)                    # the context is usable: a second run succeeds
    ref = gu.pinned_from_storage(st.copy(), so2dr.F32)
    ic = so2dr.Plan(dims, 1, "star", [0.4] + [0.1] * 6, 2 * T, k_on=4, k_off=8, budget_bytes=0, dtype="f32")
    ic.run(ref, in_core=True)
    assert torch.equal(host, ref)
