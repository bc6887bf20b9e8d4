"""Parity at the full workload sizes, in the launch configuration the benchmark
times: the out-of-core GPU run is compared, element by element, with the FP64
oracle on sampled sub-boxes computed from their dependency cones (a cell after
T steps of a radius-r stencil depends only on cells within r*T of it, the
fixed ring clipping the cone), and byte for byte with the in-core GPU run."""
import numpy as np
import pytest

import oracle
from paper_2309_08864_gb300 import inputs, so2dr
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

C2 = dict(dims=(1024, 1024, 1024), r=1, coeffs=[0.4] + [0.1] * 6, T=64, budget=1 << 30, min_chunks=8)


def sample_boxes(dims, chunk_starts, rng, n_random=3, w=4, every_boundary=False):
    """Corners, chunk boundaries (every one, on both sides, or a quarter of
    them) and random spots."""
    boxes = [((0, 0, 0)), tuple(d - w for d in dims)]
    inner = chunk_starts[1:-1]
    if every_boundary:
        for s in inner:
            for z in (max(0, s - w), min(dims[0] - w, s)):
                boxes.append((z, int(rng.integers(0, dims[1] - w)), int(rng.integers(0, dims[2] - w))))
    else:
        for s in inner[:: max(1, len(chunk_starts) // 4)]:
            boxes.append((max(0, s - w // 2), int(rng.integers(0, dims[1] - w)), dims[2] - w))
    for _ in range(n_random):
        boxes.append(tuple(int(rng.integers(0, d - w)) for d in dims))
    return [(lo, tuple(l + w for l in lo)) for lo in boxes]


def cone_check(dims, r, coeffs, T, dtype, host_after, starts, tol, seed=1, n_random=3, every_boundary=False):
    rng = np.random.default_rng(0)
    errs = []
    c_ref = gu.compute_coeffs(coeffs, dtype)
    for lo, hi in sample_boxes(dims, starts, rng, n_random, every_boundary=every_boundary):
        blo, bhi = oracle.cone_box(dims, lo, hi, r * T)
        ub = inputs.to_storage(inputs.draw_box(seed, dims, blo, bhi), dtype)
        ref = oracle.run_cone(inputs.storage_to_f64(ub, dtype), c_ref, r, oracle.STAR, T, blo, bhi, dims, lo, hi)
        got = host_after[tuple(slice(l, h) for l, h in zip(lo, hi))]
        got = gu.storage_of(got.contiguous(), dtype)
        e = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        errs.append(e)
        assert e <= tol, (lo, e)
    return max(errs), len(errs)


def _full_run(dims, r, coeffs, T, dtype, budget, min_chunks, k_on=0, k_off=0, in_core_check=True, seed=1,
              plan=None):
    import torch
    u = inputs.draw_box(seed, dims, as_f32=True)
    st = inputs.to_storage(u, dtype) if dtype != so2dr.F32 else u
    host = gu.pinned_from_storage(st, dtype)
    ref_copy = host.clone().pin_memory() if in_core_check else None
    if plan is None:
        plan = so2dr.Plan(dims, r, "star", coeffs, T, min_chunks=min_chunks, k_on=k_on, k_off=k_off,
                          budget_bytes=budget, dtype=dtype)
    info = plan.info
    assert info["arena_bytes"] <= budget
    plan.run(host)
    starts = plan.chunks()
    if in_core_check:
        ic = so2dr.Plan(dims, r, "star", coeffs, T, min_chunks=1, k_on=info["k_on"], k_off=info["k_off"],
                        budget_bytes=0, dtype=dtype)
        ic.run(ref_copy, in_core=True)
        assert torch.equal(host.view(torch.uint8), ref_copy.view(torch.uint8)), "out-of-core != in-core"
        ic.close()
    plan.close()
    return host, starts, info


def bench_plan(name):
    """The plan bench.py times for one of its configs (same constructor)."""
    import bench
    cfg = dict(bench.CONFIGS[name])
    return cfg, bench.coeffs_of(cfg["coeffs"], inputs), bench.make_plan(cfg, bench.coeffs_of(cfg["coeffs"], inputs),
                                                                        so2dr)


def test_c2_7pt_1024cubed_fp32_full_size():
    """The benchmarked plan of the 1024^3 7-point FP32 workload (64 steps,
    1 GiB): out-of-core byte-identical to in-core, and the FP64 oracle on
    dependency cones on both sides of every chunk boundary plus random spots."""
    cfg, c, plan = bench_plan("c2")
    dims = cfg["dims"]
    host, starts, info = _full_run(dims, cfg["r"], c, cfg["T"], so2dr.F32, cfg["budget"], cfg["min_chunks"],
                                   plan=plan)
    assert info["chunks"] >= 8
    err, n = cone_check(dims, cfg["r"], c, cfg["T"], so2dr.F32, host, starts, 1e-5, n_random=8, every_boundary=True)
    assert n == 2 + 2 * (len(starts) - 2) + 8
    print("C2_PLAN k_off=%d k_on=%d chunks=%d cones=%d max_rel_err=%.3e" % (info["k_off"], info["k_on"],
                                                                        info["chunks"], n, err))


def test_c3_25pt_r4_1536cubed_fp32_full_size():
    cfg, c, plan = bench_plan("c3")
    host, starts, info = _full_run(cfg["dims"], cfg["r"], c, cfg["T"], so2dr.F32, cfg["budget"], cfg["min_chunks"],
                                   plan=plan)
    err, n = cone_check(cfg["dims"], cfg["r"], c, cfg["T"], so2dr.F32, host, starts, 1e-5, n_random=2,
                        every_boundary=True)
    print("C3_PLAN k_off=%d k_on=%d chunks=%d cones=%d max_rel_err=%.3e" % (info["k_off"], info["k_on"],
                                                                        info["chunks"], n, err))


def test_c4_precision_forms_1024cubed_128_steps():
    """Storage in FP32 / BF16 / FP16 with FP32 arithmetic, 1 GiB budget, the
    benchmarked plans: the error against the FP64 oracle (same rounded input)
    on sampled cones, and out-of-core byte-identical to in-core for every
    storage type."""
    import json
    import torch
    dims, r, T = (1024, 1024, 1024), 1, 128
    coeffs = [0.4] + [0.1] * 6
    report = {}
    for dtype, tol, name in ((so2dr.F32, 1e-5, "c4-f32"), (so2dr.BF16, 3e-2, "c4-bf16"), (so2dr.F16, 5e-3, "c4-f16")):
        _, _, plan = bench_plan(name)
        host, starts, info = _full_run(dims, r, coeffs, T, dtype, 1 << 30, 8, plan=plan)
        rng = np.random.default_rng(0)
        errs, l2n, l2d, errs_u, l2n_u, l2d_u = [], 0.0, 0.0, [], 0.0, 0.0
        for lo, hi in sample_boxes(dims, starts, rng, n_random=0, w=2)[:3]:
            blo, bhi = oracle.cone_box(dims, lo, hi, r * T)
            u32 = inputs.draw_box(1, dims, blo, bhi, as_f32=True)
            ub = inputs.storage_to_f64(inputs.to_storage(u32.astype(np.float64), dtype), dtype)
            ref = oracle.run_cone(ub, gu.compute_coeffs(coeffs, dtype), r, oracle.STAR, T, blo, bhi, dims, lo, hi)
            # also: the FP64 oracle from the unrounded draw with the exact weights
            ref_u = oracle.run_cone(inputs.draw_box(1, dims, blo, bhi), coeffs, r, oracle.STAR, T, blo, bhi,
                                    dims, lo, hi)
            got = gu.storage_of(host[tuple(slice(l, h) for l, h in zip(lo, hi))].contiguous(), dtype)
            errs.append(float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))))
            l2n += float(np.sum((got - ref) ** 2))
            l2d += float(np.sum(ref ** 2))
            errs_u.append(float(np.max(np.abs(got - ref_u)) / np.max(np.abs(ref_u))))
            l2n_u += float(np.sum((got - ref_u) ** 2))
            l2d_u += float(np.sum(ref_u ** 2))
        report[{so2dr.F32: "f32", so2dr.BF16: "bf16", so2dr.F16: "f16"}[dtype]] = {
            "rel_linf": max(errs), "rel_l2": (l2n / l2d) ** 0.5,
            "rel_linf_vs_unrounded_draw": max(errs_u), "rel_l2_vs_unrounded_draw": (l2n_u / l2d_u) ** 0.5,
            "k_off": info["k_off"], "chunks": info["chunks"]}
        assert max(errs) <= tol, (dtype, errs)
        del host
    print("PRECISION_REPORT " + json.dumps(report))


def test_c5_adjoint_512cubed_finite_differences():
    """Differentiation form at full size: 512^3 FP32, 64 steps, checkpoints
    every 8 steps, 256 MiB budget; 16 central-difference directions (8 in u0,
    8 in the face fields) of the FP64 loss against the adjoint gradient."""
    from tests.test_gpu_adjoint import fd_check
    err = fd_check((512, 512, 512), 64, 8, 256 << 20, 8, 8, 1e-4)
    print("C5_FD_MAX_REL_ERR %.3e" % err)
