"""Benchmark of the SO2DR out-of-core stencil path on GB300.

Metric: Gcell-updates/s out-of-core on one GB300 (interior cells x time steps
per second) and its fraction of the roofline max(host-link bytes / measured
link bandwidth, HBM bytes / measured HBM bandwidth).

Default workload (the 3D 7-point star, FP32, 1024^3 grid of 4 GiB held in
pinned host memory, 64 time steps, device budget 1 GiB): one benchmark step is
one so2dr_run over the whole grid -- every round of Algorithm 1: host-to-device
transfers, the on-chip temporal-blocking kernels over the circular
region-sharing buffer, device-to-host transfers.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl so2dr|reference]
                  [--config c2|c1|c3|c4-bf16|c4-f16|c4-f32|c5|box2d{1..4}r|box2d{1..4}r-ic]
                  [--mode so2dr|incore|resreu] [--k-off k] [--k-on k]
                  [--tune N] [--timeline FILE] [--no-cpu-baseline]
  python bench.py --sweep 4,8,16,32 [--k-on 4]    # run-time tuning trade-off (Sec. V-B)
  python bench.py --link                          # host link: copy engines vs SM copies
  python bench.py --kernel-case 512 --k-on 4 [--kind box --radius R]
                                                  # in-core kernel run (profiling)

--mode resreu runs the redundancy-free comparison code (single-step launches,
region sharing of intermediate results); --mode incore the in-core code (whole
grid on the device, transfers outside the timed region).  --tune N times the
cost model's N best plans (so2dr_autotune) and benchmarks the fastest.

k_off / k_on of 0 let the planner choose them (and its buffer options) from its
cost model calibrated to the measured kernel rates.

--impl reference times the FP64 CPU oracle (the only reference this method has:
the paper ships no code) on the host cores, on bounded samples of the same
workload.  Under torchrun (N > 1) every rank runs its own replica (the path
does not shard across GPUs); rank 0 prints the line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
KERNEL_SRC = {"star": os.path.join(ROOT, "paper_2309_08864_gb300", "csrc", "star3d_tb.cuh"),
              "box": os.path.join(ROOT, "paper_2309_08864_gb300", "csrc", "box2d_fast.cuh")}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per k_on-deep launch
# of the benchmarked plan, from one ncu capture of the benchmark command (the
# summaries under profiles/ give the commands), keyed by the first 16 hex
# digits of the SHA-256 of the kernel source they were taken with: a capture
# of an older kernel is not reported.
# Captured launches are one run's middle chunks; the figure is their DRAM
# bytes per input+output plane times the mean input+output planes of all of
# the plan's k_on-deep launches (edge chunks clip their trapezoids).
DRAM_TRAFFIC = {
    # config: (k_off, k_on, chunks of the captured plan, bytes per launch, of which read, written)
    "38a01a2b0291d24d": {"c2": (22, 4, 29, 441.9e6, 260.9e6, 180.9e6), "c3": (8, 1, 23, 1815.3e6, 977.8e6, 837.6e6)},
}
# host-link bandwidths measured earlier on the GB300 machines with pinned
# buffers (cudaMemcpyAsync, 4 GiB): host-to-device 211, device-to-host 193,
# both directions at once 343 GB/s in total; reported beside the rates the
# benchmark measures in its own process
LINK_H2D_GBS, LINK_D2H_GBS, LINK_BIDIR_GBS = 211.3, 193.4, 342.7
# FP32 rate of the SM units (no tensor cores: a stencil is not a dense
# contraction): 152 SMs x 128 FMA lanes x 2 FLOP x 2.07 GHz (maximum SM clock)
ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12

CONFIGS = {
    # name: dims, radius, coefficients, steps, dtype, budget, min_chunks
    "c1": dict(workload="2D 5-point Jacobi FP64 512x512, zero ring, 16 steps, 1 MiB budget",
               dims=(512, 512), r=1, coeffs="jacobi2d", T=16, dtype="f64", budget=1 << 20,
               min_chunks=4, k_on=4, k_off=8, zero_ring=True),
    "c2": dict(workload="3D 7-point star FP32 1024^3 (4 GiB), 64 steps, 1 GiB budget",
               dims=(1024, 1024, 1024), r=1, coeffs="star7", T=64, dtype="f32", budget=1 << 30,
               min_chunks=8, k_on=0, k_off=0),
    "c3": dict(workload="3D 25-point star r=4 FP32 1536^3 (14.5 GB), 32 steps, 4 GiB budget",
               dims=(1536, 1536, 1536), r=4, coeffs="r4", T=32, dtype="f32", budget=4 << 30,
               min_chunks=1, k_on=0, k_off=0),
    "c4-bf16": dict(workload="3D 7-point star BF16 storage 1024^3, 128 steps, 1 GiB budget",
                    dims=(1024, 1024, 1024), r=1, coeffs="star7", T=128, dtype="bf16",
                    budget=1 << 30, min_chunks=8, k_on=0, k_off=0),
    "c4-f16": dict(workload="3D 7-point star FP16 storage 1024^3, 128 steps, 1 GiB budget",
                   dims=(1024, 1024, 1024), r=1, coeffs="star7", T=128, dtype="f16",
                   budget=1 << 30, min_chunks=8, k_on=0, k_off=0),
    "c4-f32": dict(workload="3D 7-point star FP32 storage 1024^3, 128 steps, 1 GiB budget",
                   dims=(1024, 1024, 1024), r=1, coeffs="star7", T=128, dtype="f32",
                   budget=1 << 30, min_chunks=8, k_on=0, k_off=0),
    "box2d1r": dict(workload="2D 9-point box (radius 1) FP32 38400^2 (5.9 GB), 640 steps, 4 GiB budget "
                             "(the paper's box2d1r workload, seeded weights)",
                    dims=(38400, 38400), r=1, kind="box", coeffs="box1", T=640, dtype="f32", budget=4 << 30,
                    min_chunks=1, k_on=0, k_off=0),
    "box2d2r": dict(workload="2D 25-point box (radius 2) FP32 38400^2 (5.9 GB), 640 steps, 4 GiB budget "
                             "(the paper's box2d2r workload, seeded weights)",
                    dims=(38400, 38400), r=2, kind="box", coeffs="box2", T=640, dtype="f32", budget=4 << 30,
                    min_chunks=1, k_on=0, k_off=0),
    "box2d3r": dict(workload="2D 49-point box (radius 3) FP32 38400^2 (5.9 GB), 640 steps, 4 GiB budget "
                             "(the paper's box2d3r workload, seeded weights)",
                    dims=(38400, 38400), r=3, kind="box", coeffs="box3", T=640, dtype="f32", budget=4 << 30,
                    min_chunks=1, k_on=0, k_off=0),
    "box2d4r": dict(workload="2D 81-point box (radius 4) FP32 38400^2 (5.9 GB), 640 steps, 4 GiB budget "
                             "(the paper's box2d4r workload, seeded weights)",
                    dims=(38400, 38400), r=4, kind="box", coeffs="box4", T=640, dtype="f32", budget=4 << 30,
                    min_chunks=1, k_on=0, k_off=0),
    "box2d1r-ic": dict(workload="2D 9-point box (radius 1) FP32 12800^2 (the paper's in-core dataset), 640 "
                                "steps, at least 4 chunks under a 1 GiB budget",
                       dims=(12800, 12800), r=1, kind="box", coeffs="box1", T=640, dtype="f32", budget=1 << 30,
                       min_chunks=4, k_on=0, k_off=0),
    "box2d2r-ic": dict(workload="2D 25-point box (radius 2) FP32 12800^2 (the paper's in-core dataset), 640 "
                                "steps, at least 4 chunks under a 1 GiB budget",
                       dims=(12800, 12800), r=2, kind="box", coeffs="box2", T=640, dtype="f32", budget=1 << 30,
                       min_chunks=4, k_on=0, k_off=0),
    "box2d3r-ic": dict(workload="2D 49-point box (radius 3) FP32 12800^2 (the paper's in-core dataset), 640 "
                                "steps, at least 4 chunks under a 1 GiB budget",
                       dims=(12800, 12800), r=3, kind="box", coeffs="box3", T=640, dtype="f32", budget=1 << 30,
                       min_chunks=4, k_on=0, k_off=0),
    "box2d4r-ic": dict(workload="2D 81-point box (radius 4) FP32 12800^2 (the paper's in-core dataset), 640 "
                                "steps, at least 4 chunks under a 1 GiB budget",
                       dims=(12800, 12800), r=4, kind="box", coeffs="box4", T=640, dtype="f32", budget=1 << 30,
                       min_chunks=4, k_on=0, k_off=0),
    "c5": dict(workload="3D variable-coefficient 7-point FP32 512^3, 64 steps, adjoint with checkpoints "
                        "every 8 steps, 256 MiB budget",
               dims=(512, 512, 512), r=1, coeffs=None, T=64, dtype="f32", budget=256 << 20,
               min_chunks=1, k_on=4, k_off=8, adjoint=True),
}


def source_digest(path):
    import hashlib
    try:
        with open(path, "rb") as f:
            return hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None


def path_roofline(grid_bytes, rounds, launches, link, hbm_gbs):
    """Roofline time of a plan: every cell crosses the host link once each way
    per round (the two directions at the rates measured while both run), and
    HBM sees the landing write and the read for the transfers plus one read
    and one write per fused launch."""
    t_link = max(grid_bytes * rounds / (link["ce_both_h2d"] * 1e9), grid_bytes * rounds / (link["ce_both_d2h"] * 1e9))
    hbm_bytes = grid_bytes * rounds * (2.0 + 2.0 * launches)
    t_hbm = hbm_bytes / (hbm_gbs * 1e9)
    return {"t_roof_s": max(t_link, t_hbm), "t_link_s": t_link, "t_hbm_s": t_hbm, "hbm_bytes": hbm_bytes,
            "bound": "host-link" if t_link >= t_hbm else "hbm"}


def make_plan(cfg, coeffs, so2dr):
    """The benchmarked plan: k_off / k_on as the config gives them, else the
    planner's own choice under its default rates (so that the plan does not
    depend on the box; the parity tests build it through this function)."""
    return so2dr.Plan(cfg["dims"], cfg["r"], cfg.get("kind", "star"), coeffs, cfg["T"], min_chunks=cfg["min_chunks"],
                      k_on=cfg["k_on"], k_off=cfg["k_off"], budget_bytes=cfg["budget"], dtype=cfg["dtype"])


def coeffs_of(name, inputs):
    if name.startswith("box"):
        return list(inputs.box2d_coeffs(int(name[3:])))
    if name == "jacobi2d":
        return [0.2] * 5
    if name == "star7":
        return [0.4] + [0.1] * 6
    return list(inputs.radius4_star_coeffs())


def measured_peaks():
    try:
        with open(MEASURED) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ CPU oracle

DTYPE_CODE = {"f64": 0, "f32": 1, "bf16": 2, "f16": 3}


def oracle_sample(cfg, inputs, steps=None, planes=None, rounded=True, keep=False):
    """Times the FP64 oracle on a bounded slab of the workload: `planes`
    planes of axis 0 (full extent on the other axes) for `steps` time steps.
    rounded: the slab as the GPU stores it (storage-rounded values, weights
    rounded to the compute type); else the unrounded draw and exact weights.
    Returns (cell_updates_per_s, cores, sample description, seconds, output
    or None)."""
    import numpy as np
    import oracle
    dims = cfg["dims"]
    nd = len(dims)
    T = cfg["T"] if steps is None else steps
    n0 = dims[0] if planes is None else min(planes, dims[0])
    sub = (n0,) + tuple(dims[1:])
    u = inputs.draw_box(1, dims, lo=(0,) * nd, hi=sub)
    if cfg.get("zero_ring"):
        inputs.zero_ring(u, cfg["r"])
    c = np.asarray(coeffs_of(cfg["coeffs"], inputs), dtype=np.float64)
    if rounded and cfg["dtype"] != "f64":
        code = DTYPE_CODE[cfg["dtype"]]
        u = inputs.storage_to_f64(inputs.to_storage(u, code), code)
        c = c.astype(np.float32).astype(np.float64)
    kind = 1 if cfg.get("kind") == "box" else 0
    t0 = time.perf_counter()
    out = oracle.run(u, c, cfg["r"], kind, T)
    dt = time.perf_counter() - t0
    inner = 1
    for e in sub:
        inner *= max(0, e - 2 * cfg["r"])
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    desc = "FP64 oracle on a %s slab of the workload (first %d planes), %d steps" % (
        "x".join(map(str, sub)), n0, T)
    return inner * T / dt, cores, desc, dt, (out if keep else None)


def slab_errors(cfg, gpu_out, ref, planes):
    """Relative L-infinity and L2 error of the GPU result on the part of an
    oracle slab that the cut does not reach: planes below planes - r(T+1)
    (a cell depends only on cells within r*T of it; the slab's top r planes
    act as a fixed ring in the oracle run)."""
    import numpy as np
    hi = planes - cfg["r"] * (cfg["T"] + 1)
    if hi <= cfg["r"]:
        return None
    got = gpu_out[:hi]
    want = ref[:hi]
    d = got - want
    return {"rel_linf": float(np.max(np.abs(d)) / np.max(np.abs(want))),
            "rel_l2": float(np.linalg.norm(d.ravel()) / np.linalg.norm(want.ravel())), "planes": [0, int(hi)]}


def oracle_sample_planes(cfg, budget_s, inputs):
    """Slab thickness giving roughly budget_s seconds of oracle work (probe)."""
    dims = cfg["dims"]
    probe_planes = min(dims[0], 2 * cfg["r"] + 8)
    rate, _, _, _, _ = oracle_sample(cfg, inputs, steps=2, planes=probe_planes)
    plane_cells = 1
    for e in dims[1:]:
        plane_cells *= e
    want = rate * budget_s / (plane_cells * cfg["T"])
    return int(max(2 * cfg["r"] + 2, min(dims[0], want)))


def cpu_baseline_leg(cfg, plan, mode, torch, inputs, so2dr):
    """The FP64 oracle timed on the host cores on a bounded slab of the
    workload (about 15 s), and the error of this plan's GPU result against
    it: one more run of the plan, outside the timed region, from the seeded
    input, compared on the slab's exact part -- with the oracle started from
    the same storage-rounded input, and from the unrounded draw with exact
    weights (for FP64 storage the two coincide)."""
    import numpy as np
    import oracle
    oracle.build.build()
    planes = oracle_sample_planes(cfg, 15.0, inputs)
    rate, cores, desc, dt, ref = oracle_sample(cfg, inputs, planes=planes, keep=True)
    if dt < 10.0 and planes < cfg["dims"][0]:
        # the small probe overstates the per-plane cost: rescale once
        planes = int(min(cfg["dims"][0], planes * 15.0 / max(dt, 0.05)))
        rate, cores, desc, dt, ref = oracle_sample(cfg, inputs, planes=planes, keep=True)
    base = {"value": rate / 1e9, "unit": "Gcell/s", "cores": cores, "kind": "oracle",
            "sample": desc + " (%.1f s)" % dt}
    host = make_input(cfg, inputs, so2dr, torch)
    plan.run(host, in_core=mode)
    code = DTYPE_CODE[cfg["dtype"]]
    if cfg["dtype"] == "bf16":
        gpu = inputs.bf16_bits_to_f64(host[:planes].contiguous().view(torch.int16).numpy().view(np.uint16))
    else:
        gpu = host[:planes].numpy().astype(np.float64)
    err = {"reference": "FP64 oracle from the storage-rounded input and weights rounded to the compute type",
           "slab": desc}
    err.update(slab_errors(cfg, gpu, ref, planes) or {})
    if code != 0:
        _, _, _, _, ref_u = oracle_sample(cfg, inputs, planes=planes, rounded=False, keep=True)
        eu = slab_errors(cfg, gpu, ref_u, planes) or {}
        err["rel_linf_vs_unrounded_draw"] = eu.get("rel_linf")
        err["rel_l2_vs_unrounded_draw"] = eu.get("rel_l2")
    return base, err


def run_reference(args, cfg, world, rank):
    from paper_2309_08864_gb300 import inputs
    import oracle
    oracle.build.build()
    inputs.build()
    if rank != 0:
        return 0
    budget_each = float(os.environ.get("SO2DR_REF_STEP_SECONDS", "8"))
    planes = oracle_sample_planes(cfg, budget_each, inputs)
    rates = []
    for i in range(args.warmup + args.steps):
        rate, cores, desc, dt, _ = oracle_sample(cfg, inputs, planes=planes)
        if i == 0 and dt < 0.6 * budget_each and planes < cfg["dims"][0]:
            # the small probe overstates the per-plane cost: rescale once
            planes = int(min(cfg["dims"][0], planes * budget_each / max(dt, 0.05)))
        if i >= args.warmup:
            rates.append(rate)
    value = statistics.mean(rates) / 1e9
    line = {"impl": "reference", "metric": "Gcell-updates/s out-of-core on 1 GB300; % of max(host-link, HBM) roofline",
            "value": value, "unit": "Gcell/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (SplitMix64-seeded)",
            "config": {"workload": cfg["workload"], "sample": desc},
            "cpu_baseline": {"value": value, "unit": "Gcell/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "Gcell/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU path

def make_input(cfg, inputs, so2dr, torch):
    import numpy as np
    dims = cfg["dims"]
    dt = cfg["dtype"]
    if dt in ("f32", "bf16", "f16"):
        u = inputs.draw_box(1, dims, as_f32=True)
        if dt == "bf16":
            t = torch.from_numpy(u).to(torch.bfloat16)
        elif dt == "f16":
            t = torch.from_numpy(u).to(torch.float16)
        else:
            t = torch.from_numpy(u)
    else:
        u = inputs.draw_box(1, dims)
        if cfg.get("zero_ring"):
            inputs.zero_ring(u, cfg["r"])
        t = torch.from_numpy(u)
    if cfg.get("zero_ring") and dt != "f64":
        inputs.zero_ring(t.numpy(), cfg["r"])
    return t.pin_memory()


def run_kernel_case(args):
    """In-core run of the temporal-blocking kernel on an n^3 FP32 grid (the
    shape the ncu captures use)."""
    import torch
    from paper_2309_08864_gb300 import inputs, so2dr
    n = args.kernel_case
    r = args.radius
    kon = args.k_on or 4
    T = kon * max(1, args.launches)
    if args.kind == "box":
        dims, kind, coeffs = (n, n), "box", list(inputs.box2d_coeffs(r))
    else:
        dims, kind = (n, n, n), "star"
        if r == 1:
            coeffs = [0.4] + [0.1] * 6
        elif r == 4:
            coeffs = list(inputs.radius4_star_coeffs())
        else:  # 6r + 1 seeded weights summing to 1, as for radius 4
            c = inputs.draw_box(7, (6 * r + 1,), dist="uniform", a=0.5, b=1.5)
            coeffs = list(c / c.sum())
    cells = 1
    for e in dims:
        cells *= e
    u = torch.from_numpy(inputs.draw_box(1, dims, as_f32=True)).pin_memory()
    plan = so2dr.Plan(dims, r, kind, coeffs, T, min_chunks=1, k_on=kon, k_off=T, budget_bytes=0, dtype="f32")
    for _ in range(max(1, args.warmup) + args.steps):
        st = plan.run(u, in_core=True)
    ms = st["kernel_ms"] / st["launches"]
    print(json.dumps({"kernel_case": n, "kind": kind, "radius": r, "k_on": kon, "launches": st["launches"],
                      "kernel_ms_per_launch": ms, "alg_GBs": 2 * 4 * cells / (ms * 1e-3) / 1e9,
                      "gcell_steps_per_s": cells * kon / (ms * 1e-3) / 1e9}))
    return 0


def run_adjoint(args, cfg, world, rank, local):
    """Differentiation form: one step = one so2dr_adjoint (checkpointed forward,
    loss, recomputation and the transposed stencil backward) over the grid."""
    import numpy as np
    import torch
    from paper_2309_08864_gb300 import inputs, so2dr
    dims, T, C = cfg["dims"], cfg["T"], cfg["k_off"]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    u0 = pin(inputs.draw_box(1, dims, as_f32=True))
    faces = np.empty((6,) + dims, dtype=np.float32)
    for f in range(6):
        inputs.draw_box(100 + f, dims, a=0.05, b=0.15, as_f32=True, out=faces[f])
    faces = pin(faces)
    tgt = pin(inputs.draw_box(2, dims, as_f32=True))
    plan = so2dr.Plan(dims, 1, "varcoef", None, T, min_chunks=cfg["min_chunks"], k_on=cfg["k_on"], k_off=C,
                      budget_bytes=cfg["budget"], dtype="f32")
    gu_ = torch.empty_like(u0).pin_memory()
    gc_ = torch.empty_like(faces).pin_memory()
    ws = plan.workspace(C)
    for _ in range(args.warmup):
        plan.adjoint(u0, faces, tgt, gu_, gc_, ws, C)
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    stats = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        loss, st = plan.adjoint(u0, faces, tgt, gu_, gc_, ws, C)
        stats.append(st)
    wall = allreduce_max(time.perf_counter() - t0, world)
    clk = clocks.stop()
    inner = 1
    for e in dims:
        inner *= e - 2
    cells = 2.0 * inner * T   # forward + adjoint cell updates
    ms = allreduce_max(sum(s["total_ms"] for s in stats), world)
    value = world * cells * args.steps / (ms * 1e-3) / 1e9
    h2d = stats[-1]["h2d_bytes"]
    d2h = stats[-1]["d2h_bytes"]
    line = {"metric": "Gcell-updates/s out-of-core on 1 GB300 (forward + adjoint updates)", "value": value,
            "unit": "Gcell/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (SplitMix64-seeded)",
            "config": {"workload": cfg["workload"], "chunks": plan.info["chunks"], "loss": loss},
            "e2e": {"value": world * cells * args.steps / wall / 1e9, "unit": "Gcell/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(sum(s["launches"] for s in stats)), "clocks": clk,
            "stage_ms_per_step": {"kernel": sum(s["kernel_ms"] for s in stats) / args.steps,
                                  "h2d": sum(s["h2d_ms"] for s in stats) / args.steps,
                                  "d2h": sum(s["d2h_ms"] for s in stats) / args.steps}}
    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_sweep(args, cfg, coeffs, host, hbm_peak, rank):
    """Run-time tuning trade-off (Sec. V-B, Fig. 5): one plan per k_off (k_on and
    the buffer options as the planner picks them for that k_off, or --k-on),
    each run warmup + steps times; least measured time beside the model's
    prediction, the chunk count and redundancy the budget forces, and the
    stage times."""
    from paper_2309_08864_gb300 import so2dr
    link = (LINK_BIDIR_GBS / 2, LINK_BIDIR_GBS / 2)
    rows = []
    for ko in [int(x) for x in args.sweep.split(",") if x]:
        kon = args.k_on or 0
        try:
            plan = so2dr.Plan(cfg["dims"], cfg["r"], cfg.get("kind", "star"), coeffs, cfg["T"], min_chunks=cfg["min_chunks"],
                              k_on=kon, k_off=ko, budget_bytes=cfg["budget"], dtype=cfg["dtype"], link_gbs=link,
                              hbm_gbs=hbm_peak)
        except so2dr.So2drError as e:
            rows.append({"k_off": ko, "status": str(e)})
            continue
        info = plan.info
        pred = so2dr.candidates(cfg["dims"], cfg["r"], cfg.get("kind", "star"), coeffs, cfg["T"], min_chunks=cfg["min_chunks"],
                                k_on=info["k_on"], k_off=ko, budget_bytes=cfg["budget"], dtype=cfg["dtype"],
                                link_gbs=link, hbm_gbs=hbm_peak)
        pred_ms = [e["predicted_ms"] for e in pred if e["lookahead"] == info["lookahead"] and
                   e["out_slabs"] == info["out_slabs"]][0]
        plan.bind()
        best = None
        for i in range(args.warmup + args.steps):
            st = plan.run(host)
            if i >= args.warmup and (best is None or st["total_ms"] < best["total_ms"]):
                best = st
        rows.append({"k_off": ko, "k_on": info["k_on"], "chunks": info["chunks"], "rounds": info["rounds"],
                     "lookahead": info["lookahead"], "out_slabs": info["out_slabs"],
                     "redundancy": round(info["redundancy"], 4), "predicted_ms": round(pred_ms, 2),
                     "measured_ms": round(best["total_ms"], 2),
                     "gcells_per_s": round(info["cell_updates_per_run"] / (best["total_ms"] * 1e-3) / 1e9, 1),
                     "kernel_ms": round(best["kernel_ms"], 2), "h2d_ms": round(best["h2d_ms"], 2),
                     "d2h_ms": round(best["d2h_ms"], 2)})
        plan.close()
    if rank == 0:
        print(json.dumps({"sweep": rows, "workload": cfg["workload"], "steps": args.steps,
                          "warmup": args.warmup}), flush=True)
    return 0


def bench_config(args, cfg, name, world, rank, local, torch, inputs, so2dr, link=None):
    """Times one configuration (warm-up runs, then args.steps timed runs of
    so2dr_run) and returns its JSON line."""
    hbm_peak, peak_kind = measured_peaks()
    coeffs = coeffs_of(cfg["coeffs"], inputs)
    host = make_input(cfg, inputs, so2dr, torch)
    # the host link of this machine, measured in this process before the timed
    # region: copy engines, 1 GiB per direction, each alone and both at once
    if link is None:
        link = so2dr.measure_link(1 << 30, sm_ctas=64, repeats=3)
        torch.cuda.synchronize()
    tuned = None
    if args.tune > 0:
        # the timings do not depend on the values: the benchmark grid is the scratch
        table, tl = so2dr.autotune(cfg["dims"], cfg["r"], cfg.get("kind", "star"), coeffs, cfg["T"], cfg["budget"],
                                   cfg["dtype"], scratch=host, max_candidates=args.tune, repeats=2,
                                   min_chunks=cfg["min_chunks"], k_on=cfg["k_on"] if args.k_on else 0,
                                   k_off=cfg["k_off"] if args.k_off else 0)
        tuned = {"candidates_timed": args.tune, "link_gbs": {"h2d": tl[0], "d2h": tl[1], "hbm": tl[2]},
                 "table": [[e["k_off"], e["k_on"], e["chunks"], e["lookahead"], e["out_slabs"],
                            round(e["predicted_ms"], 2), round(e["measured_ms"], 2)] for e in table[:args.tune]],
                 "columns": ["k_off", "k_on", "chunks", "lookahead", "out_slabs", "predicted_ms", "measured_ms"]}
        plan = so2dr.Plan(cfg["dims"], cfg["r"], cfg.get("kind", "star"), coeffs, cfg["T"], budget_bytes=cfg["budget"],
                          dtype=cfg["dtype"], tune_entry=table[0])
    else:
        plan = make_plan(cfg, coeffs, so2dr)
    info = plan.info
    mode = {"so2dr": 0, "incore": 1, "resreu": 2, "zerocopy": 3}[args.mode]
    plan.bind(in_core=mode)
    for _ in range(args.warmup):
        plan.run(host, in_core=mode)
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    stats = []
    walls = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        stats.append(plan.run(host, in_core=mode))   # synchronous: joins every stream before returning
        walls.append(time.perf_counter() - t0)
    torch.cuda.synchronize()
    t_all = time.perf_counter() - t_all
    barrier(world)
    clk = clocks.stop()

    if mode == 1:
        # in-core comparison code: transfers are excluded (Sec. V-D), time the kernels
        for s_ in stats:
            s_["total_ms"] = s_["kernel_ms"]
    dev_ms = sum(s["total_ms"] for s in stats)
    dev_ms_max = allreduce_max(dev_ms, world)
    wall_max = allreduce_max(sum(walls), world)
    cells = info["cell_updates_per_run"]
    value = world * cells * args.steps / (dev_ms_max * 1e-3) / 1e9
    e2e = world * cells * args.steps / wall_max / 1e9
    # roofline of the dominant kernel (the k_on-deep launches)
    mk_ms = sum(s["main_kernel_ms"] for s in stats)
    mk_n = sum(s["main_kernel_launches"] for s in stats)
    mk_cells = sum(s["main_kernel_cells"] for s in stats)
    b = {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}[cfg["dtype"]]
    alg_bytes_per_launch = 2 * b * mk_cells / max(1, mk_n)
    avg_launch_s = mk_ms / max(1, mk_n) * 1e-3
    achieved = alg_bytes_per_launch / avg_launch_s / 1e9 if mk_n else 0.0
    # FP32 work of the same launches: 2n - 1 FLOP per cell-step of an n-point
    # stencil (Table III's count), against the FP32 rate of the SM units
    npts = (2 * cfg["r"] + 1) ** 2 if cfg.get("kind") == "box" else 1 + 2 * cfg["r"] * len(cfg["dims"])
    depth = info["k_on"] if mode != 2 else 1
    alg_flops_per_launch = (2 * npts - 1) * depth * mk_cells / max(1, mk_n)
    achieved_tf = alg_flops_per_launch / avg_launch_s / 1e12 if mk_n else 0.0
    alu_bound = alg_flops_per_launch / (ALU_PEAK_TFLOPS * 1e12) > alg_bytes_per_launch / (hbm_peak * 1e9)
    kind = cfg.get("kind", "star")
    cap = DRAM_TRAFFIC.get(source_digest(KERNEL_SRC[kind]), {}).get(name) if mode == 0 else None
    if cap and (cap[0], cap[1], cap[2]) != (info["k_off"], info["k_on"], info["chunks"]):
        cap = None
    traffic = cap[3] if cap else None
    # whole-path roofline: max(host-link time, HBM time) of the algorithmic
    # bytes (every cell sent and received once per round; two HBM passes for
    # the transfers and two per fused launch), against the link measured above
    t_meas = dev_ms / args.steps * 1e-3
    Nb = b
    for e in cfg["dims"]:
        Nb *= e
    pr = path_roofline(Nb, info["rounds"], -(-info["k_off"] // info["k_on"]), link, hbm_peak)
    if mode == 1:
        # in-core: no host traffic inside the run; one read and one write of
        # the grid per k_on-deep launch
        hb = 2.0 * Nb * -(-cfg["T"] // info["k_on"])
        pr = {"t_roof_s": hb / (hbm_peak * 1e9), "t_link_s": 0.0, "t_hbm_s": hb / (hbm_peak * 1e9),
              "hbm_bytes": hb, "bound": "hbm"}
    # the same against the fewest rounds the budget admits (largest feasible
    # k_off), so that plans with different round counts read on one scale
    cand = so2dr.candidates(cfg["dims"], cfg["r"], kind, coeffs, cfg["T"], min_chunks=cfg["min_chunks"],
                            budget_bytes=cfg["budget"], dtype=cfg["dtype"])
    kmax = max(c["k_off"] for c in cand)
    konmax = max(c["k_on"] for c in cand if c["k_off"] == kmax)
    rmin = -(-cfg["T"] // kmax)
    prm = path_roofline(Nb, rmin, -(-kmax // konmax), link, hbm_peak)
    t_pool = max(2.0 * Nb * info["rounds"] / (LINK_BIDIR_GBS * 1e9), pr["t_hbm_s"])
    h2d = stats[-1]["h2d_bytes"]
    d2h = stats[-1]["d2h_bytes"]
    if mode == 3:
        # zero-copy input: the first launches read the new planes over the link
        h2d = info["h2d_bytes_per_run"]
    line = {
        "metric": "Gcell-updates/s out-of-core on 1 GB300; % of max(host-link, HBM) roofline",
        "value": value, "unit": "Gcell/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dev_ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": cfg["dtype"], "data": "synthetic (SplitMix64-seeded)",
        "config": {"workload": cfg["workload"], "mode": args.mode, "dims": list(cfg["dims"]), "radius": cfg["r"],
                   "time_steps": cfg["T"], "device_budget_bytes": cfg["budget"], "k_off": info["k_off"],
                   "k_on": info["k_on"] if mode != 2 else 1,
                   "chunks": info["chunks"] if mode != 2 else info["result_reuse_chunks"], "rounds": info["rounds"],
                   "ring_planes": info["ring_planes"], "arena_bytes": info["arena_bytes"],
                   "lookahead": info["lookahead"], "out_slabs": info["out_slabs"],
                   "redundancy": info["redundancy"], "plan": "given k_off/k_on" if (cfg["k_off"] or cfg["k_on"])
                   else "the planner's automatic choice",
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "l2": "inputs larger than L2 (grid of %.1f GiB vs 126 MB L2)" % (Nb / 2 ** 30)},
        "path_roofline": {"bound": pr["bound"], "t_roof_ms": pr["t_roof_s"] * 1e3, "t_measured_ms": t_meas * 1e3,
                          "frac": pr["t_roof_s"] / t_meas, "frac_vs_measured_link": pr["t_roof_s"] / t_meas,
                          "link_measured_gbs": {k: link[k] for k in ("ce_h2d", "ce_d2h", "ce_both_h2d",
                                                                     "ce_both_d2h")},
                          "frac_min_rounds": prm["t_roof_s"] / t_meas if mode != 1 else None,
                          "min_rounds": rmin, "k_off_max": kmax,
                          "frac_vs_pool_link": t_pool / t_meas if mode != 1 else None,
                          "link_pool_bidir_gbs": LINK_BIDIR_GBS,
                          "host_bytes": 2.0 * Nb * info["rounds"] if mode != 1 else 0.0, "hbm_bytes": pr["hbm_bytes"], "hbm_gbs": hbm_peak,
                          "stream_gbs_during_run": {"h2d": (stats[-1]["h2d_bytes"] / (stats[-1]["h2d_ms"] * 1e-3) / 1e9
                                                            if stats[-1]["h2d_ms"] > 0 else None),
                                                    "d2h": (d2h / (stats[-1]["d2h_ms"] * 1e-3) / 1e9
                                                            if stats[-1]["d2h_ms"] > 0 else None)}},
        "roofline": {"bound": "alu" if alu_bound else "hbm",
                     "achieved": achieved_tf if alu_bound else achieved,
                     "peak": ALU_PEAK_TFLOPS if alu_bound else hbm_peak,
                     "unit": "TFLOP/s" if alu_bound else "GB/s",
                     "frac": achieved_tf / ALU_PEAK_TFLOPS if alu_bound else achieved / hbm_peak,
                     "hbm": {"achieved_gbs": achieved, "peak_gbs": hbm_peak, "frac": achieved / hbm_peak},
                     "alu": {"achieved_tflops": achieved_tf, "peak_tflops": ALU_PEAK_TFLOPS,
                             "frac": achieved_tf / ALU_PEAK_TFLOPS, "flop_per_cell_step": 2 * npts - 1},
                     "traffic": traffic,
                     # above 1 by the redundant trapezoid planes a launch also computes
                     "traffic_vs_alg": traffic / alg_bytes_per_launch if traffic and alg_bytes_per_launch else None,
                     "traffic_read_vs_alg": cap[4] / (alg_bytes_per_launch / 2) if traffic and alg_bytes_per_launch else None,
                     "traffic_write_vs_alg": cap[5] / (alg_bytes_per_launch / 2) if traffic and alg_bytes_per_launch else None,
                     "kernel": ("box2d_fast_kernel" if kind == "box" else "star3d_tb_kernel")
                               + " (k_on-step TB launch)", "peak_kind": ("derived from unit counts and the maximum SM clock" if alu_bound
                                   else peak_kind + " (burst)"),
                     "alg_bytes_per_launch": alg_bytes_per_launch,
                     "avg_launch_ms": avg_launch_s * 1e3, "launches": mk_n},
        "e2e": {"value": e2e, "unit": "Gcell/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(sum(s["launches"] for s in stats)),
        "clocks": clk,
        "stage_ms_per_step": {"kernel": sum(s["kernel_ms"] for s in stats) / args.steps,
                              "h2d": sum(s["h2d_ms"] for s in stats) / args.steps,
                              "d2h": sum(s["d2h_ms"] for s in stats) / args.steps},
    }
    if tuned:
        line["autotune"] = tuned
    if args.timeline:
        with open(args.timeline, "w") as f:
            json.dump(plan.timeline(in_core=mode), f)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], line["error_vs_oracle"] = cpu_baseline_leg(cfg, plan, mode, torch, inputs, so2dr)
    plan.close()
    del host
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="so2dr", choices=["so2dr", "reference"])
    ap.add_argument("--config", default="c2", choices=sorted(CONFIGS) + ["c4"])
    ap.add_argument("--k-off", type=int, default=None)
    ap.add_argument("--k-on", type=int, default=None)
    ap.add_argument("--kernel-case", type=int, default=0)
    ap.add_argument("--radius", type=int, default=1)
    ap.add_argument("--kind", default="star", choices=["star", "box"], help="--kernel-case stencil (box: 2D n x n)")
    ap.add_argument("--launches", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="so2dr", choices=["so2dr", "incore", "resreu", "zerocopy"],
                    help="so2dr: the out-of-core SO2DR pipeline (default); incore: the whole grid on the "
                         "device, same launch depths, transfers outside the timed region; resreu: the "
                         "redundancy-free out-of-core comparison code (single-step launches, region "
                         "sharing of intermediate results); zerocopy: the SO2DR pipeline whose first "
                         "launches read the new planes from the mapped host grid (no host-to-device copy)")
    ap.add_argument("--tune", type=int, default=0,
                    help="measured autotune before timing: time the model's N best plans (so2dr_autotune) "
                         "and benchmark the fastest")
    ap.add_argument("--sweep", default="",
                    help="comma-separated k_off values: measured and predicted time of one run per k_off "
                         "(the run-time tuning trade-off of Sec. V-B); prints one JSON line")
    ap.add_argument("--timeline", default="",
                    help="write the per-op timeline (so2dr_run_timeline) of the last timed run to this JSON file")
    ap.add_argument("--link", action="store_true",
                    help="measure the host link (copy engines vs SM-driven copies over the mapped pinned "
                         "buffers, each direction and both at once) and HBM; prints one JSON line")
    args = ap.parse_args()
    cfg = dict(CONFIGS[args.config if args.config != "c4" else "c4-f32"])
    if args.k_off is not None:
        cfg["k_off"] = args.k_off
    if args.k_on is not None:
        cfg["k_on"] = args.k_on
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, cfg, world, rank)

    import torch
    from paper_2309_08864_gb300 import inputs, so2dr
    torch.cuda.set_device(local)
    if args.kernel_case:
        return run_kernel_case(args)
    if args.link:
        rows = {}
        for ctas in (32, 64, 152):
            rows[ctas] = so2dr.measure_link(1 << 30, sm_ctas=ctas, repeats=3)
        print(json.dumps({"link_gbs": rows, "bytes": 1 << 30, "note": "keys by SM-copy CTA count; ce_* are "
                          "cudaMemcpyAsync, sm_* a copy kernel over the mapped pinned buffer"}), flush=True)
        return 0
    if cfg.get("adjoint"):
        return run_adjoint(args, cfg, world, rank, local)

    if args.sweep:
        hbm_peak, _ = measured_peaks()
        return run_sweep(args, cfg, coeffs_of(cfg["coeffs"], inputs), make_input(cfg, inputs, so2dr, torch),
                         hbm_peak, rank)
    if args.config == "c4":
        # the precision forms back to back on one box: FP32, BF16 and FP16
        # storage (FP32 arithmetic), each with its error against the oracle
        link = so2dr.measure_link(1 << 30, sm_ctas=64, repeats=3)
        forms = {}
        for dt in ("f32", "bf16", "f16"):
            c = dict(CONFIGS["c4-" + dt])
            forms[dt] = bench_config(args, c, "c4-" + dt, world, rank, local, torch, inputs, so2dr, link=link)
        line = dict(forms["bf16"])
        line["config"] = dict(line["config"], workload="3D 7-point star 1024^3, 128 steps, 1 GiB budget: FP32 vs "
                                                       "BF16 vs FP16 storage (FP32 arithmetic); value: BF16")
        line["precision_forms"] = {dt: {"value": f["value"], "unit": f["unit"], "ms_per_step": f["ms_per_step"],
                                        "plan": {k: f["config"][k] for k in ("k_off", "k_on", "chunks", "rounds")},
                                        "error_vs_oracle": f.get("error_vs_oracle"),
                                        "path_roofline_frac": f["path_roofline"]["frac"]}
                                   for dt, f in forms.items()}
        line["precision_forms"]["bf16_over_f32"] = forms["bf16"]["value"] / forms["f32"]["value"]
        line["precision_forms"]["f16_over_f32"] = forms["f16"]["value"] / forms["f32"]["value"]
    else:
        line = bench_config(args, cfg, args.config, world, rank, local, torch, inputs, so2dr)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
