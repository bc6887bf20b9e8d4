"""Run-time parameter search (host only, no GPU): the cost model's candidate
list (so2dr_plan_candidates) and plans built from one of its rows
(so2dr_plan_tuned).  The measured autotune itself is in test_gpu_tune.py."""
import random

import pytest

from paper_2309_08864_gb300 import so2dr

C7 = [0.4] + [0.1] * 6
PROBLEMS = [
    dict(dims=(256, 128, 128), radius=1, kind="star", coeffs=C7, time_steps=32, budget_bytes=16 << 20,
         dtype="f32"),
    dict(dims=(300, 64, 96), radius=1, kind="star", coeffs=C7, time_steps=20, budget_bytes=4 << 20,
         dtype="bf16"),
    dict(dims=(2000, 512), radius=1, kind="star", coeffs=[0.2] * 5, time_steps=24, budget_bytes=1 << 20,
         dtype="f64"),
]
KEYS = ("k_off", "k_on", "chunks", "lookahead", "out_slabs")


def _plan_key(p):
    i = p.info
    return (i["k_off"], i["k_on"], i["chunks"], i["lookahead"], i["out_slabs"])


@pytest.mark.parametrize("prob", PROBLEMS)
def test_candidates_are_ranked_and_the_automatic_plan_follows_the_band_rule(prob):
    t = so2dr.candidates(**prob, link_gbs=(200.0, 190.0), hbm_gbs=6800.0)
    assert len(t) > 1
    preds = [e["predicted_ms"] for e in t]
    assert preds == sorted(preds) and preds[0] > 0
    assert len({tuple(e[k] for k in KEYS) for e in t}) == len(t)  # no duplicates
    for e in t:
        assert e["status"] == 0 and e["measured_ms"] == -1.0
        assert 1 <= e["k_on"] <= e["k_off"] and e["chunks"] >= 1
    # the automatic plan: among candidates predicted within 2% of the best,
    # those with the fewest rounds (least host-link traffic); among these,
    # within 1% of their lowest prediction, the smallest k_off, then the
    # lowest prediction
    auto = so2dr.Plan(**prob, link_gbs=(200.0, 190.0), hbm_gbs=6800.0)
    rounds = lambda e: -(-prob["time_steps"] // e["k_off"])
    band = [e for e in t if e["predicted_ms"] <= 1.02 * preds[0]]
    fewest = [e for e in band if rounds(e) == min(rounds(x) for x in band)]
    low = min(e["predicted_ms"] for e in fewest)
    pick = min([e for e in fewest if e["predicted_ms"] <= 1.01 * low], key=lambda e: (e["k_off"], e["predicted_ms"]))
    assert _plan_key(auto) == tuple(pick[k] for k in KEYS)


@pytest.mark.parametrize("prob", PROBLEMS)
def test_tuned_plan_reproduces_its_entry_within_budget(prob):
    t = so2dr.candidates(**prob)
    rng = random.Random(5)
    for e in [t[0], t[-1]] + rng.sample(t, min(6, len(t))):
        p = so2dr.Plan(**prob, tune_entry=e)
        assert _plan_key(p) == tuple(e[k] for k in KEYS)
        assert p.info["arena_bytes"] <= prob["budget_bytes"]


def test_pinned_parameters_restrict_the_candidates():
    prob = PROBLEMS[0]
    t = so2dr.candidates(**prob, k_off=8, k_on=4)
    assert {(e["k_off"], e["k_on"]) for e in t} == {(8, 4)}
    assert {(e["lookahead"], e["out_slabs"]) for e in t} <= {(0, 1), (0, 2), (1, 1), (1, 2)}


def test_bad_entries_are_rejected():
    prob = PROBLEMS[0]
    e = dict(so2dr.candidates(**prob)[0])
    with pytest.raises(so2dr.So2drError) as ex:
        so2dr.Plan(**prob, tune_entry=dict(e, out_slabs=3))
    assert ex.value.code == so2dr.E_INVAL
    # one chunk cannot hold this grid under the budget: the planner would raise d
    with pytest.raises(so2dr.So2drError) as ex:
        so2dr.Plan(**prob, tune_entry=dict(e, chunks=1))
    assert ex.value.code == so2dr.E_INFEASIBLE
    with pytest.raises(so2dr.So2drError) as ex:
        so2dr.candidates(**dict(prob, budget_bytes=4096))
    assert ex.value.code == so2dr.E_INFEASIBLE


def test_measure_link_rejects_bad_arguments_before_any_device_work():
    lib = so2dr.load_library()
    import ctypes
    out = (ctypes.c_double * 9)()
    buf = ctypes.create_string_buffer(16)
    assert lib.so2dr_measure_link(None, None, None, 1 << 20, 64, 1, out) == so2dr.E_INVAL
    assert lib.so2dr_measure_link(buf, buf, buf, 1000, 64, 1, out) == so2dr.E_INVAL   # < 1 MiB
    assert lib.so2dr_measure_link(buf, buf, buf, (1 << 20) + 8, 64, 1, out) == so2dr.E_INVAL  # not 16-byte multiple
    assert lib.so2dr_measure_link(buf, buf, buf, 1 << 20, 0, 1, out) == so2dr.E_INVAL


def test_timeline_is_empty_before_any_timed_run():
    import ctypes
    lib = so2dr.load_library()
    p = so2dr.Plan((40, 36, 44), 1, "star", C7, 4, min_chunks=3, budget_bytes=0)
    n = ctypes.c_int64(-1)
    assert lib.so2dr_run_timeline(p._h, None, None, 0, ctypes.byref(n)) == so2dr.OK
    assert n.value == 0
    assert lib.so2dr_run_timeline(None, None, None, 0, ctypes.byref(n)) == so2dr.E_INVAL

