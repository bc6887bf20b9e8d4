"""Replays plans' op lists on the CPU (tests/emulator.py) in random stream
interleavings allowed by the planner's waits: the out-of-core result must be
bit-identical to the in-core FP64 oracle (Sec. IV-B: redundant computation and
region sharing recompute and reuse the same values)."""
import numpy as np
import pytest

import oracle
from paper_2309_08864_gb300 import inputs, so2dr
from tests.emulator import replay
from tests.test_oracle_pins import my_offsets

CASES = [
    # dims, r, kind, T, min_chunks, k_on, k_off, budget
    ((48, 40), 1, "star", 16, 4, 4, 8, 0),
    ((48, 40), 1, "star", 13, 5, 3, 5, 0),
    ((60, 33), 2, "star", 9, 6, 2, 4, 0),
    ((70, 12, 14), 1, "star", 11, 7, 4, 8, 0),
    ((71, 13, 12), 1, "star", 19, 3, 5, 19, 0),
    ((64, 14, 15), 4, "star", 5, 3, 2, 5, 0),
    ((50, 30), 3, "box", 7, 4, 2, 3, 0),
    ((40, 16), 1, "star", 10, 1, 4, 4, 0),      # a single chunk
    ((40, 16), 1, "star", 10, 38, 4, 10, 0),    # one plane per chunk, P << 2rk
    ((33, 9, 11), 1, "varcoef", 7, 4, 2, 3, 0),
    ((512, 512), 1, "star", 16, 4, 4, 8, 1 << 20),  # the 2D Jacobi workload at full size
    ((90, 40), 2, "box", 9, 3, 3, 4, 0),        # box stencil with chunks thick enough for result reuse
]


def _setup(dims, r, kind):
    nd = len(dims)
    if kind == "varcoef":
        faces = np.stack([inputs.draw_box(100 + f, dims, a=0.05, b=0.15) for f in range(6)])
        return None, faces
    k = 0 if kind == "star" else 1
    n = len(my_offsets(nd, r, k))
    c = inputs.draw_box(5, (n,), a=0.5, b=1.5)
    return c / c.sum(), None


@pytest.mark.parametrize("case", CASES)
def test_out_of_core_replay_is_bit_identical_to_in_core_oracle(case):
    dims, r, kind, T, dmin, kon, koff, budget = case
    c, faces = _setup(dims, r, kind)
    p = so2dr.Plan(dims, r, kind, c, T, min_chunks=dmin, k_on=kon, k_off=koff, budget_bytes=budget,
                   dtype="f64")
    u0 = inputs.draw_box(1, dims)
    if kind == "varcoef":
        ref = oracle.run_varcoef(u0, faces, T)
    else:
        ref = oracle.run(u0, c, r, 0 if kind == "star" else 1, T)
    seeds = [0, 1, 2] if np.prod(dims) < 100000 else [0]
    for sd in seeds:
        got = replay(p, u0, faces, in_core=False, seed=sd)
        assert np.array_equal(got, ref), "seed %d" % sd
    for pol in ("h2d_first", "d2h_first"):
        got = replay(p, u0, faces, in_core=False, policy=pol)
        assert np.array_equal(got, ref), pol
    got = replay(p, u0, faces, in_core=True)
    assert np.array_equal(got, ref)


def test_emulator_detects_a_missing_wait():
    """Sanity check of the emulator itself: dropping the wait that orders a
    chunk's first kernel after its host-to-device copy must break the result
    in some interleaving."""
    dims, r, T = (48, 40), 1, 8
    c = np.full(5, 0.2)
    p = so2dr.Plan(dims, r, "star", c, T, min_chunks=4, k_on=4, k_off=8, budget_bytes=0, dtype="f64")
    ops = p.ops()
    broken = [dict(o) for o in ops]
    for o in broken:
        if o["kind"] == 1:
            w = list(o["wait_op"])
            w[0] = -1
            o["wait_op"] = tuple(w)
    assert any(o["kind"] == 1 and o["wait_op"][0] >= 0 for o in ops)
    p.ops = lambda in_core=False: broken if not in_core else ops
    u0 = inputs.draw_box(1, dims)
    ref = oracle.run(u0, c, r, 0, T)
    bad = 0
    for pol in ("d2h_first", "random"):
        for sd in range(3):
            got = replay(p, u0, None, seed=sd, policy=pol)
            bad += not np.array_equal(got, ref)
    assert bad > 0


@pytest.mark.parametrize("lookahead,nout", [(0, 1), (0, 2), (1, 1)])
@pytest.mark.parametrize("case", [CASES[0], CASES[3], CASES[4], CASES[8], CASES[9]])
def test_buffer_options_stay_race_free(case, lookahead, nout, monkeypatch):
    """Without the one-chunk look-ahead and/or with a single output slab the
    planner's waits must still order every reuse (random interleavings)."""
    monkeypatch.setenv("SO2DR_LOOKAHEAD", str(lookahead))
    monkeypatch.setenv("SO2DR_NOUT", str(nout))
    dims, r, kind, T, dmin, kon, koff, budget = case
    c, faces = _setup(dims, r, kind)
    p = so2dr.Plan(dims, r, kind, c, T, min_chunks=dmin, k_on=kon, k_off=koff, budget_bytes=budget,
                   dtype="f64")
    assert p.info["lookahead"] == lookahead and p.info["out_slabs"] == nout
    u0 = inputs.draw_box(1, dims)
    ref = oracle.run_varcoef(u0, faces, T) if kind == "varcoef" else oracle.run(u0, c, r, 0 if kind == "star" else 1, T)
    for sd in (0, 1):
        assert np.array_equal(replay(p, u0, faces, seed=sd), ref)
    for pol in ("h2d_first", "d2h_first"):
        assert np.array_equal(replay(p, u0, faces, policy=pol), ref)


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[2], CASES[3], CASES[5], CASES[6], CASES[8], CASES[10],
                                  CASES[11]])
def test_result_reuse_code_is_exact(case):
    """The redundancy-free comparison code (single-step launches, region
    sharing of intermediate results before every step) computes the same
    values as the in-core oracle, in any interleaving the waits allow."""
    dims, r, kind, T, dmin, kon, koff, budget = case
    c, faces = _setup(dims, r, kind)
    p = so2dr.Plan(dims, r, kind, c, T, min_chunks=dmin, k_on=kon, k_off=koff, budget_bytes=budget, dtype="f64")
    info = p.info
    starts = p.chunks()
    if info["result_reuse_chunks"] == 0:
        # unavailable exactly when some chunk cannot hold the parallelogram's shift
        assert np.min(np.diff(starts)) < (koff + 2) * r or info["rounds"] == 0
        return
    if budget:
        assert info["arena_bytes_result_reuse"] <= budget
    ops = p.ops(2)
    assert all(o["depth"] == 1 for o in ops if o["kind"] == 1)   # single-step kernels only
    u0 = inputs.draw_box(1, dims)
    ref = oracle.run(u0, c, r, 0 if kind == "star" else 1, T)
    for sd in (0, 1):
        assert np.array_equal(replay(p, u0, None, in_core=2, seed=sd), ref)
    assert np.array_equal(replay(p, u0, None, in_core=2, policy="h2d_first"), ref)


ZC_CASES = [
    # dims, r, T, min_chunks, k_on, k_off, dtype
    ((70, 12, 16), 1, 11, 7, 4, 8, "f32"),     # residual round, ragged chunks
    ((71, 13, 16), 1, 19, 3, 4, 19, "f32"),    # one round
    ((64, 14, 16), 2, 9, 5, 2, 4, "bf16"),     # radius 2, 16-bit storage
    ((40, 8, 8), 1, 10, 38, 2, 10, "f32"),     # one plane per chunk, P << 2rk
    ((60, 10, 16), 4, 5, 3, 1, 3, "f32"),      # radius 4
]


@pytest.mark.parametrize("case", ZC_CASES)
def test_zero_copy_replay_is_bit_identical_to_in_core_oracle(case):
    """Run mode 3 (zero-copy input): no host-to-device copy of the grid; the
    first launch of each chunk reads its new planes from the host grid and
    writes them into the circular buffer for the next chunk.  Any interleaving
    the waits allow gives the in-core result, and the in-place host grid is
    read only after the previous round wrote it back."""
    dims, r, T, dmin, kon, koff, dtype = case
    c, _ = _setup(dims, r, "star")
    p = so2dr.Plan(dims, r, "star", c, T, min_chunks=dmin, k_on=kon, k_off=koff, budget_bytes=0, dtype=dtype)
    assert p.info["zero_copy"] == 1
    ops = p.ops(3)
    assert not any(o["kind"] == 0 for o in ops)   # no host-to-device copy at all
    u0 = inputs.draw_box(1, dims)
    ref = oracle.run(u0, c, r, 0, T)
    for sd in (0, 1, 2):
        assert np.array_equal(replay(p, u0, None, in_core=3, seed=sd), ref), sd
    for pol in ("h2d_first", "d2h_first"):
        assert np.array_equal(replay(p, u0, None, in_core=3, policy=pol), ref), pol


def test_zero_copy_needs_the_3d_star_kernel():
    p = so2dr.Plan((48, 40), 1, "star", [0.2] * 5, 8, min_chunks=3, k_on=2, k_off=4, dtype="f32")
    assert p.info["zero_copy"] == 0   # 2D: the generic kernel
    p = so2dr.Plan((40, 12, 16), 1, "star", C7_STAR, 8, min_chunks=3, k_on=2, k_off=4, dtype="f64")
    assert p.info["zero_copy"] == 0   # FP64 storage: the generic kernel
    p = so2dr.Plan((40, 12, 18), 1, "star", C7_STAR, 8, min_chunks=3, k_on=2, k_off=4, dtype="f32")
    assert p.info["zero_copy"] == 0   # rows of 18 FP32 values are not a whole number of 16 bytes


C7_STAR = [0.4] + [0.1] * 6
