"""Property test of the planner's schedules (host only): for random problems
-- dimension, radius, stencil, steps, k_off, k_on, chunk floor, budget and
the two buffer options -- the out-of-core op list, replayed on the CPU in a
random order that respects only its declared waits, equals the FP64 oracle
bit for bit; so does the result-reuse list where the plan has one."""
import os

import numpy as np
import pytest

import oracle
from paper_2309_08864_gb300 import inputs, so2dr
from tests.emulator import replay
from tests.test_oracle_pins import my_offsets

hyp = pytest.importorskip("hypothesis")
from hypothesis import HealthCheck, event, given, settings, strategies as st  # noqa: E402


@settings(max_examples=200, deadline=None, suppress_health_check=[HealthCheck.too_slow])
@given(data=st.data())
def test_random_plans_replay_exactly(data):
    nd = data.draw(st.sampled_from([2, 3]), label="ndim")
    r = data.draw(st.integers(1, 3), label="r")
    kind = data.draw(st.sampled_from(["star", "box"]) if nd == 2 else st.just("star"), label="kind")
    n0 = data.draw(st.integers(2 * r + 1, 40), label="n0")
    inplane = (data.draw(st.integers(2 * r + 1, 24)),) if nd == 2 else \
        (data.draw(st.integers(2 * r + 1, 9)), data.draw(st.integers(2 * r + 1, 9)))
    dims = (n0,) + inplane
    T = data.draw(st.integers(0, 12), label="T")
    k_off = data.draw(st.integers(1, 9), label="k_off")
    k_on = data.draw(st.integers(1, 5), label="k_on")
    dmin = data.draw(st.integers(1, max(1, n0 - 2 * r)), label="min_chunks")
    la = data.draw(st.sampled_from(["0", "1"]), label="lookahead")
    no = data.draw(st.sampled_from(["1", "2"]), label="out_slabs")
    plane = int(np.prod(inplane)) * 8
    budget = data.draw(st.sampled_from([0, plane * (2 * r * k_off + 12) * 4, plane * (2 * r * k_off + 4) * 3]),
                       label="budget")
    n = len(my_offsets(nd, r, 0 if kind == "star" else 1))
    c = inputs.draw_box(5, (n,), a=0.5, b=1.5)
    c = c / c.sum()
    old = {k: os.environ.get(k) for k in ("SO2DR_LOOKAHEAD", "SO2DR_NOUT")}
    os.environ["SO2DR_LOOKAHEAD"], os.environ["SO2DR_NOUT"] = la, no
    try:
        try:
            p = so2dr.Plan(dims, r, kind, c, T, min_chunks=dmin, k_on=k_on, k_off=k_off, budget_bytes=budget,
                           dtype="f64")
        except so2dr.So2drError as e:
            # a budget too small for any chunking, or a fused depth beyond the
            # deepest kernel for this stencil (both documented statuses)
            assert (e.code == so2dr.E_INFEASIBLE and budget > 0) or \
                (e.code == so2dr.E_UNSUPPORTED and "deepest fused kernel" in str(e)), str(e)
            event("no plan: %s" % ("budget" if e.code == so2dr.E_INFEASIBLE else "depth"))
            return
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    info = p.info
    if budget:
        assert info["arena_bytes"] <= budget
    u0 = inputs.draw_box(1, dims)
    ref = oracle.run(u0, c, r, 0 if kind == "star" else 1, T)
    seed = data.draw(st.integers(0, 1 << 16), label="seed")
    assert np.array_equal(replay(p, u0, None, seed=seed), ref)
    event("replayed: %d chunks, %d rounds" % (min(info["chunks"], 3), min(info["rounds"], 3)))
    if info["result_reuse_chunks"]:
        assert np.array_equal(replay(p, u0, None, in_core=2, seed=seed), ref)
        event("result-reuse list replayed")
