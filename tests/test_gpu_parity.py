"""GPU vs FP64 oracle, element by element, through the C ABI; out-of-core vs
in-core, byte for byte (Sec. IV-B: the reorganisation recomputes identical
values).  Tolerances: relative L-infinity 1e-12 for FP64 storage and 1e-5 for
FP32 storage after the configured steps; BF16/FP16 storage report their error
against the FP64 oracle started from the same rounded input, bounded here by
a few units of the format's rounding per kernel store."""
import numpy as np
import pytest

import oracle
from paper_2309_08864_gb300 import inputs, so2dr
from tests import gpu_util as gu
from tests.test_oracle_pins import my_offsets

pytestmark = pytest.mark.gpu

TOL = {so2dr.F64: 1e-12, so2dr.F32: 1e-5, so2dr.BF16: 2e-2, so2dr.F16: 4e-3}


def _coeffs(nd, r, kind, seed=5):
    n = len(my_offsets(nd, r, 0 if kind == "star" else 1))
    c = inputs.draw_box(seed, (n,), a=0.5, b=1.5)
    return c / c.sum()


def check_case(dims, r, kind, coeffs, T, dtype, min_chunks, k_on, k_off, budget, zero_ring=False,
               faces=None):
    u64 = inputs.draw_box(1, dims)
    if zero_ring:
        inputs.zero_ring(u64, r)
    st = inputs.to_storage(u64, dtype)
    u_ref0 = inputs.storage_to_f64(st, dtype)
    plan = so2dr.Plan(dims, r, kind, coeffs, T, min_chunks=min_chunks, k_on=k_on, k_off=k_off,
                      budget_bytes=budget, dtype=dtype)
    ooc = gu.pinned_from_storage(st.copy(), dtype)
    ic = gu.pinned_from_storage(st.copy(), dtype)
    cf = None
    if faces is not None:
        import torch
        cdt = np.float64 if dtype == so2dr.F64 else np.float32
        faces_c = faces.astype(cdt)
        cf = torch.from_numpy(faces_c).pin_memory()
        ref = oracle.run_varcoef(u_ref0, faces_c.astype(np.float64), T)
    else:
        ref = oracle.run(u_ref0, gu.compute_coeffs(coeffs, dtype), r, 0 if kind == "star" else 1, T)
    s1 = plan.run(ooc, cf, in_core=False)
    s2 = plan.run(ic, cf, in_core=True)
    got = gu.storage_of(ooc, dtype)
    err = gu.rel_linf(got, ref)
    assert err <= TOL[dtype], (err, plan.info)
    import torch
    assert torch.equal(ooc.view(torch.uint8), ic.view(torch.uint8)), "out-of-core differs from in-core"
    # boundary planes of axis 0 untouched, byte for byte
    assert np.array_equal(gu.storage_of(ooc, dtype)[:r], u_ref0[:r])
    assert np.array_equal(gu.storage_of(ooc, dtype)[-r:], u_ref0[-r:])
    info = plan.info
    plan.close()
    return err, info, s1, s2


def test_jacobi_2d_fp64_full_size():
    """2D 5-point Jacobi, 512 x 512 FP64, zero ring, 16 steps, 1 MiB budget,
    k_on = 4 (the 2D Jacobi workload at its stated size)."""
    err, info, s1, _ = check_case((512, 512), 1, "star", [0.2] * 5, 16, so2dr.F64, 4, 4, 8, 1 << 20,
                                  zero_ring=True)
    assert info["arena_bytes"] <= 1 << 20 and info["chunks"] >= 4


@pytest.mark.parametrize("dims,T,dmin,kon,koff", [
    ((72, 70, 132), 12, 5, 4, 8),   # register-streaming kernel, depth 4, two x tiles, ragged y
    ((61, 37, 44), 13, 4, 3, 5),    # depths 3 and 2 (residual), ragged everything
    ((40, 33, 260), 9, 3, 2, 9),    # depths 2 and 1, three x tiles
    ((45, 50, 16), 7, 2, 1, 7),     # depth 1, a single narrow x tile
    ((72, 70, 66), 12, 5, 4, 8),    # nx % 4 != 0: the generic kernel
    ((30, 24, 24), 5, 1, 5, 5),     # depth 5: the generic kernel
])
def test_star3d_r1_fp32(dims, T, dmin, kon, koff):
    check_case(dims, 1, "star", [0.4] + [0.1] * 6, T, so2dr.F32, dmin, kon, koff, 0)


def test_star3d_r1_fp64():
    check_case((50, 44, 41), 1, "star", [0.4] + [0.1] * 6, 10, so2dr.F64, 4, 4, 8, 0)


@pytest.mark.parametrize("dims,T,kon,koff", [((60, 72, 68), 7, 2, 4), ((50, 41, 53), 6, 3, 6),
                                             ((64, 70, 140), 6, 1, 3)])
def test_star3d_r4_fp32(dims, T, kon, koff):
    check_case(dims, 4, "star", inputs.radius4_star_coeffs(), T, so2dr.F32, 3, kon, koff, 0)


@pytest.mark.parametrize("r,kon,koff", [(2, 2, 4), (2, 1, 3), (3, 1, 2)])
def test_star3d_r2_r3_fp32(r, kon, koff):
    check_case((52, 45, 136), r, "star", _coeffs(3, r, "star"), 7, so2dr.F32, 3, kon, koff, 0)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_star2d_fp32(r):
    check_case((90, 300), r, "star", _coeffs(2, r, "star"), 11, so2dr.F32, 5, 4, 6, 0)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_box2d_fp32(r):
    check_case((80, 301), r, "box", _coeffs(2, r, "box"), 9, so2dr.F32, 4, 4, 5, 0)


@pytest.mark.parametrize("r,kon,koff,T,dtype", [
    (1, 8, 16, 21, so2dr.F32),    # deepest launch, then a 5-step residual
    (1, 4, 6, 13, so2dr.F32),
    (2, 4, 8, 11, so2dr.F32),
    (3, 3, 5, 11, so2dr.F32),
    (4, 2, 4, 9, so2dr.F32),
    (4, 1, 3, 5, so2dr.F32),
    (1, 4, 8, 16, so2dr.BF16),
    (2, 3, 6, 13, so2dr.F16),
])
def test_box2d_fast_kernel(r, kon, koff, T, dtype):
    """Register-streaming 2D box kernel (the paper's box2d workloads, Table
    III): three x tiles with a ragged last one, chunked rows, residual
    launches, 16-bit storage."""
    check_case((170, 2312), r, "box", _coeffs(2, r, "box"), T, dtype, 3, kon, koff, 0)


@pytest.mark.parametrize("r,kon", [(1, 8), (2, 4), (3, 3), (4, 2), (1, 4), (2, 2), (3, 1), (4, 1)])
def test_box2d_fast_kernel_matches_generic_kernel_bitwise(r, kon, monkeypatch):
    """Both kernels sum each cell's products in the same order (row by row
    from offset (-R, -R), a multiply first), so their FP32 results agree bit
    for bit."""
    import torch
    dims, T = (96, 1104), kon + 1
    st = inputs.to_storage(inputs.draw_box(3, dims), so2dr.F32)
    plan = so2dr.Plan(dims, r, "box", _coeffs(2, r, "box"), T, k_on=kon, k_off=T, budget_bytes=0, dtype="f32")
    fast = gu.pinned_from_storage(st.copy(), so2dr.F32)
    plan.run(fast, in_core=True)
    monkeypatch.setenv("SO2DR_GENERIC_KERNEL", "1")
    generic = gu.pinned_from_storage(st.copy(), so2dr.F32)
    plan.run(generic, in_core=True)
    assert torch.equal(fast, generic)
    assert not torch.equal(fast, gu.pinned_from_storage(st.copy(), so2dr.F32))


@pytest.mark.parametrize("dtype", [so2dr.BF16, so2dr.F16])
def test_star3d_16bit_storage(dtype):
    err, info, _, _ = check_case((64, 48, 52), 1, "star", [0.4] + [0.1] * 6, 16, dtype, 4, 4, 8, 0)
    assert err > 0  # rounding at kernel stores is visible


@pytest.mark.parametrize("dtype", [so2dr.F32, so2dr.F64])
def test_varcoef_forward(dtype):
    dims = (40, 36, 34)
    faces = np.stack([inputs.draw_box(100 + f, dims, a=0.05, b=0.15) for f in range(6)])
    check_case(dims, 1, "varcoef", None, 9, dtype, 4, 3, 5, 0, faces=faces)


@pytest.mark.parametrize("dims,r,T,koff,kon,budget", [((96, 80, 132), 1, 12, 6, 3, 8 << 20),
                                                      ((120, 64, 128), 2, 8, 4, 2, 16 << 20),
                                                      ((160, 40, 256), 1, 10, 10, 4, 8 << 20)])
def test_result_reuse_code_matches_in_core(dims, r, T, koff, kon, budget):
    """Mode 2 (the redundancy-free comparison code: single-step launches,
    region sharing of intermediate results) computes the same cells as the
    in-core run: FP32 storage keeps every level in FP32 either way."""
    import torch
    c = [0.4] + [0.1] * 6 if r == 1 else _coeffs(3, r, "star")
    u = inputs.draw_box(1, dims, as_f32=True)
    p = so2dr.Plan(dims, r, "star", c, T, min_chunks=4, k_on=kon, k_off=koff, budget_bytes=budget, dtype="f32")
    assert p.info["result_reuse_chunks"] >= 2
    rr = torch.from_numpy(u.copy()).pin_memory()
    ic = torch.from_numpy(u.copy()).pin_memory()
    oc = torch.from_numpy(u.copy()).pin_memory()
    p.run(rr, in_core=2)
    p.run(ic, in_core=1)
    p.run(oc, in_core=0)
    assert torch.equal(rr, ic) and torch.equal(oc, ic)
    ref = oracle.run(u.astype(np.float64), gu.compute_coeffs(c, so2dr.F32), r, 0, T)
    assert gu.rel_linf(rr.numpy().astype(np.float64), ref) <= 1e-5
    p.close()
