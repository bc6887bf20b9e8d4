"""Planner properties (host only, no GPU): chunking, Algorithm 1's rounds and
launch depths, transfer coverage, budget fitting and argument errors."""
import os

import numpy as np
import pytest

from paper_2309_08864_gb300 import so2dr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _depths_from_golden(s):
    if s == "-":
        return None
    out = []
    for part in s.split(","):
        d, n = part.split("x")
        out += [int(d)] * int(n)
    return out


def _rounds(ops):
    return sorted({o["round"] for o in ops})


@pytest.mark.parametrize("row", [l.split() for l in open(os.path.join(GOLDEN, "alg1_schedule.txt"))
                                 if l.strip() and not l.startswith("#")])
def test_algorithm1_rounds_and_launch_depths(row):
    n, k_off, k_on, nt, last, full, lastd = row
    n, k_off, k_on, nt, last = int(n), int(k_off), int(k_on), int(nt), int(last)
    p = so2dr.Plan((40, 24), 1, "star", [0.2] * 5, n, min_chunks=3, k_on=k_on, k_off=k_off,
                   budget_bytes=0, dtype="f32")
    info = p.info
    assert info["rounds"] == nt
    ops = p.ops()
    d = info["chunks"]
    for t in range(nt):
        for c in range(d):
            depths = [o["depth"] for o in ops if o["kind"] == 1 and o["round"] == t and o["chunk"] == c]
            want = _depths_from_golden(lastd if t == nt - 1 else full)
            assert depths == want, (t, c, depths, want)
            assert sum(depths) == (last if t == nt - 1 else k_off)


CASES = [
    dict(dims=(512, 512), r=1, kind="star", T=16, min_chunks=4, k_on=4, k_off=8, budget=1 << 20, dtype="f64"),
    dict(dims=(64, 20, 18), r=1, kind="star", T=13, min_chunks=5, k_on=3, k_off=5, budget=0, dtype="f32"),
    dict(dims=(70, 30, 30), r=4, kind="star", T=9, min_chunks=3, k_on=2, k_off=4, budget=0, dtype="f32"),
    dict(dims=(100, 37), r=2, kind="box", T=11, min_chunks=7, k_on=4, k_off=7, budget=0, dtype="f32"),
    dict(dims=(33, 9, 11), r=1, kind="varcoef", T=7, min_chunks=4, k_on=2, k_off=3, budget=0, dtype="f32"),
]


def _coeffs(c):
    from tests.test_oracle_pins import my_offsets
    if c["kind"] == "varcoef":
        return None
    n = len(my_offsets(len(c["dims"]), c["r"], 0 if c["kind"] == "star" else 1))
    return np.full(n, 1.0 / n)


@pytest.mark.parametrize("c", CASES)
def test_transfers_cover_every_plane_once_per_round(c):
    p = so2dr.Plan(c["dims"], c["r"], c["kind"], _coeffs(c), c["T"], min_chunks=c["min_chunks"],
                   k_on=c["k_on"], k_off=c["k_off"], budget_bytes=c["budget"], dtype=c["dtype"])
    info = p.info
    n0, r = c["dims"][0], c["r"]
    ops = p.ops()
    starts = p.chunks()
    assert starts[0] == 0 and starts[-1] == n0 and np.all(np.diff(starts) > 0)
    assert info["chunks"] >= c["min_chunks"]
    for t in range(info["rounds"]):
        h2d = np.zeros(n0, int)
        d2h = np.zeros(n0, int)
        for o in ops:
            if o["round"] != t:
                continue
            if o["kind"] == 0 and o["dst_buf"] == 0:
                h2d[o["src_lo"]:o["src_hi"]] += 1
            if o["kind"] == 2:
                d2h[o["dst_lo"]:o["dst_hi"]] += 1
        assert np.all(h2d == 1), "every plane is sent exactly once per round (region sharing)"
        assert np.all(d2h[r:n0 - r] == 1) and np.all(d2h[:r] == 0) and np.all(d2h[n0 - r:] == 0)
    # d * N_t host-to-device and device-to-host transfers of the grid (Sec. IV-A)
    n_h2d = sum(1 for o in ops if o["kind"] == 0 and o["dst_buf"] == 0)
    n_d2h = sum(1 for o in ops if o["kind"] == 2)
    assert n_h2d == n_d2h == info["chunks"] * info["rounds"]
    if c["budget"]:
        assert info["arena_bytes"] <= c["budget"]


def test_budget_raises_chunk_count_and_infeasible_budget_fails():
    a = so2dr.Plan((256, 64, 64), 1, "star", [0.4] + [0.1] * 6, 16, min_chunks=2, k_on=4, k_off=8,
                   budget_bytes=0, dtype="f32")
    b = so2dr.Plan((256, 64, 64), 1, "star", [0.4] + [0.1] * 6, 16, min_chunks=2, k_on=4, k_off=8,
                   budget_bytes=8 << 20, dtype="f32")
    assert a.info["chunks"] == 2
    assert b.info["chunks"] > 2 and b.info["arena_bytes"] <= 8 << 20
    with pytest.raises(so2dr.So2drError) as e:
        so2dr.Plan((256, 64, 64), 1, "star", [0.4] + [0.1] * 6, 16, min_chunks=2, k_on=4, k_off=8,
                   budget_bytes=64 << 10, dtype="f32")
    assert e.value.code == so2dr.E_INFEASIBLE


@pytest.mark.parametrize("kw,code", [
    (dict(dims=(8, 8, 8, 8)), so2dr.E_INVAL),
    (dict(radius=0), so2dr.E_INVAL),
    (dict(radius=5), so2dr.E_INVAL),
    (dict(coeffs=[0.2] * 4), so2dr.E_INVAL),
    (dict(time_steps=-1), so2dr.E_INVAL),
    (dict(min_chunks=0), so2dr.E_INVAL),
    (dict(k_on=17), so2dr.E_INVAL),
    (dict(dtype=7), so2dr.E_INVAL),
    (dict(coeffs=[0.2, 0.2, float("nan"), 0.2, 0.2]), so2dr.E_INVAL),
])
def test_invalid_arguments_are_rejected(kw, code):
    args = dict(dims=(32, 32), radius=1, kind="star", coeffs=[0.2] * 5, time_steps=4, min_chunks=2,
                k_on=2, k_off=4, budget_bytes=0, dtype="f32")
    args.update(kw)
    with pytest.raises(so2dr.So2drError) as e:
        so2dr.Plan(**args)
    assert e.value.code == code


def test_auto_parameters_fit_the_budget():
    p = so2dr.Plan((1024, 1024, 1024), 1, "star", [0.4] + [0.1] * 6, 64, min_chunks=8,
                   budget_bytes=1 << 30, dtype="f32", link_gbs=(171, 171), hbm_gbs=6781)
    info = p.info
    assert info["arena_bytes"] <= 1 << 30
    assert info["chunks"] >= 8
    assert 1 <= info["k_on"] <= info["k_off"] <= 64


def test_varcoef_plan_rejects_budgets_the_adjoint_cannot_fit():
    with pytest.raises(so2dr.So2drError) as e:
        so2dr.Plan((16, 12, 16), 1, "varcoef", None, 5, min_chunks=1, k_on=2, k_off=1, budget_bytes=40 << 10,
                   dtype="f32")
    assert e.value.code == so2dr.E_INFEASIBLE and "adjoint" in str(e.value)


def test_beyond_hbm_grid_plans_within_the_budget():
    """The optional beyond-HBM run of the radius-4 workload, 4096 x 4096 x 3200
    FP32 (214.7 GB, more than one GB300's HBM), plans under a 4 GiB budget:
    every plane crosses the link once per round, and the arena fits."""
    dims, T, budget = (3200, 4096, 4096), 32, 4 << 30
    c = np.full(25, 1.0 / 25)
    p = so2dr.Plan(dims, 4, "star", c, T, min_chunks=1, budget_bytes=budget, dtype="f32",
                   link_gbs=(171.35, 171.35), hbm_gbs=6781.4)
    info = p.info
    assert info["arena_bytes"] <= budget and info["chunks"] >= 2
    assert info["plane_bytes"] == 4096 * 4096 * 4
    ops = p.ops()
    n0 = dims[0]
    for t in range(info["rounds"]):
        h2d = np.zeros(n0, int)
        for o in ops:
            if o["round"] == t and o["kind"] == 0:
                h2d[o["src_lo"]:o["src_hi"]] += 1
        assert np.all(h2d == 1)
    assert info["h2d_bytes_per_run"] == info["rounds"] * n0 * info["plane_bytes"]


@pytest.mark.parametrize("dims,r,kind,T,dmin,kon,koff,budget", [
    ((48, 40), 1, "star", 16, 4, 4, 8, 0),
    ((70, 12, 14), 1, "star", 11, 7, 4, 8, 0),
    ((64, 14, 15), 4, "star", 5, 3, 2, 5, 0),
    ((90, 40), 2, "box", 9, 3, 3, 4, 0),
    ((512, 512), 1, "star", 16, 4, 4, 8, 1 << 20),
    ((256, 128, 128), 1, "star", 32, 1, 0, 0, 16 << 20),
    ((40, 16), 1, "star", 10, 38, 4, 10, 0),
])
def test_arena_buffers_are_aligned_disjoint_and_inside_the_arena(dims, r, kind, T, dmin, kon, koff, budget):
    """Every buffer of every run mode lies inside that mode's arena, starts on
    a 256-byte boundary and overlaps no other buffer (guard against layout
    bugs that would let one stage overwrite another's planes)."""
    n = 1 + 2 * r * len(dims) if kind == "star" else (2 * r + 1) ** 2
    p = so2dr.Plan(dims, r, kind, np.full(n, 1.0 / n), T, min_chunks=dmin, k_on=kon, k_off=koff,
                   budget_bytes=budget, dtype="f32")
    info = p.info
    arenas = {0: info["arena_bytes"], 1: info["arena_bytes_in_core"], 2: info["arena_bytes_result_reuse"]}
    for mode, arena in arenas.items():
        if mode == 2 and not info["result_reuse_chunks"]:
            continue
        spans = []
        for off, cap in p.buffers(mode):
            assert off % 256 == 0 and cap >= 0
            if cap:
                spans.append((off, off + cap * info["plane_bytes"]))
        spans.sort()
        assert spans and spans[-1][1] <= arena, (mode, spans[-1], arena)
        for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
            assert a1 <= b0, (mode, (a0, a1), (b0, b1))
        if budget and mode == 0:
            assert arena <= budget
