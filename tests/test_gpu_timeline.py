"""Tracing (so2dr_run_timeline) on the GPU: the per-op timeline of a run
shows the declared schedule was the one executed -- ops of one stream never
overlap, and every op starts only after each op it waits for has completed
(CUDA events; 2 us allowance for event resolution)."""
import pytest

from paper_2309_08864_gb300 import inputs, so2dr
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

EPS = 2e-3  # ms


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_timeline_follows_the_declared_waits(mode):
    dims = (160, 96, 128)
    plan = so2dr.Plan(dims, 1, "star", [0.4] + [0.1] * 6, 12, min_chunks=5, k_on=3, k_off=6,
                      budget_bytes=6 << 20, dtype="f32")
    if mode == 2:
        assert plan.info["result_reuse_chunks"] >= 2
    host = gu.pinned_from_storage(inputs.to_storage(inputs.draw_box(1, dims), so2dr.F32), so2dr.F32)
    st = plan.run(host, in_core=mode)
    tl = plan.timeline(in_core=mode)
    assert len(tl) == st["ops"] and len(tl) > 0
    last_end = {}
    for j, o in enumerate(tl):
        assert o["end_ms"] >= o["start_ms"] - EPS, (j, o)
        if o["stream"] in last_end:
            assert o["start_ms"] >= last_end[o["stream"]] - EPS, (j, o)   # one stream, one op at a time
        last_end[o["stream"]] = o["end_ms"]
        for w in o["wait_op"]:
            if w >= 0:
                assert o["start_ms"] >= tl[w]["end_ms"] - EPS, (j, w)
    assert max(o["end_ms"] for o in tl) <= st["total_ms"] + EPS
