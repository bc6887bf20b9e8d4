"""Degenerate and edge cases through the C ABI on the GPU, against the FP64
oracle and the in-core run: no time steps, grids with no interior cell (the
fixed ring covers everything), one plane per chunk, a single round, k_on above
k_off, and a last round shorter than one launch."""
import numpy as np
import pytest

import oracle
from paper_2309_08864_gb300 import inputs, so2dr
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

C7 = [0.4] + [0.1] * 6


def _run(dims, r, kind, c, T, dtype=so2dr.F32, **kw):
    import torch
    u64 = inputs.draw_box(4, dims)
    st = inputs.to_storage(u64, dtype)
    plan = so2dr.Plan(dims, r, kind, c, T, dtype=dtype, **kw)
    ooc = gu.pinned_from_storage(st.copy(), dtype)
    ic = gu.pinned_from_storage(st.copy(), dtype)
    plan.run(ooc)
    plan.run(ic, in_core=True)
    assert torch.equal(ooc.view(torch.uint8), ic.view(torch.uint8))
    ref = oracle.run(inputs.storage_to_f64(st, dtype), gu.compute_coeffs(c, dtype), r,
                     0 if kind == "star" else 1, T)
    return gu.storage_of(ooc, dtype), ref, inputs.storage_to_f64(st, dtype), plan.info


def test_zero_steps_leave_the_grid_unchanged():
    got, ref, u0, info = _run((40, 36, 44), 1, "star", C7, 0, min_chunks=3, budget_bytes=0)
    assert info["rounds"] == 0
    assert np.array_equal(got, u0) and np.array_equal(ref, u0)


@pytest.mark.parametrize("dims,r", [((2, 40, 40), 1), ((8, 8, 8), 4), ((30, 2, 64), 1), ((30, 64, 8), 4)])
def test_grids_without_interior_cells_are_unchanged(dims, r):
    c = C7 if r == 1 else inputs.radius4_star_coeffs()
    got, ref, u0, _ = _run(dims, r, "star", c, 5, min_chunks=1, budget_bytes=0)
    assert np.array_equal(got, u0) and np.array_equal(ref, u0)


def test_one_plane_per_chunk():
    dims, T = (34, 40, 64), 7
    got, ref, _, info = _run(dims, 1, "star", C7, T, min_chunks=32, k_on=3, k_off=5, budget_bytes=0)
    assert info["chunks"] == 32 and info["max_chunk_planes"] <= 2
    assert gu.rel_linf(got, ref) <= 1e-5


@pytest.mark.parametrize("T,kon,koff", [(6, 4, 64),   # one round: k_off beyond T
                                        (9, 8, 3),    # k_on above k_off: launches of k_off steps
                                        (13, 4, 6)])  # last round (1 step) shorter than a launch
def test_round_and_launch_edges(T, kon, koff):
    dims = (60, 48, 132)
    got, ref, _, info = _run(dims, 1, "star", C7, T, min_chunks=4, k_on=kon, k_off=koff, budget_bytes=0)
    assert info["k_on"] <= info["k_off"] or info["rounds"] == 1
    assert gu.rel_linf(got, ref) <= 1e-5


def test_box2d_single_row_chunks_and_residual():
    dims, r = (41, 1040), 2
    c = inputs.box2d_coeffs(r)
    got, ref, _, info = _run(dims, r, "box", c, 11, min_chunks=37, k_on=4, k_off=5, budget_bytes=0)
    assert info["chunks"] == 37
    assert gu.rel_linf(got, ref) <= 1e-5
