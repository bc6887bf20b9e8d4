"""Thin Python binding of the SO2DR C ABI (include/so2dr.h).

Argument marshalling only: every step of the stencil path runs in libso2dr.so
(CUDA kernels for sm_103a plus the C++ planner and executor).  PyTorch supplies
the device arena, the three streams and pinned host tensors.  There is no CPU
fallback: if the library is missing or fails to load, every call raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

F64, F32, BF16, F16 = 0, 1, 2, 3
STAR, BOX, VARCOEF_STAR = 0, 1, 2
DTYPES = {"f64": F64, "f32": F32, "bf16": BF16, "f16": F16}
KINDS = {"star": STAR, "box": BOX, "varcoef": VARCOEF_STAR}

OK, E_INVAL, E_INFEASIBLE, E_NOT_BOUND, E_CUDA, E_TIMEOUT, E_DEVICE_CHECK, E_NOMEM, \
    E_NOT_PINNED, E_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9

SYMBOLS = ["so2dr_plan", "so2dr_plan_ex", "so2dr_plan_info", "so2dr_plan_chunks", "so2dr_plan_ops",
           "so2dr_plan_buffers", "so2dr_bind", "so2dr_run", "so2dr_adjoint", "so2dr_loss", "so2dr_dot",
           "so2dr_destroy", "so2dr_strerror", "so2dr_last_error", "so2dr_abi_version",
           "so2dr_run_device_noalloc", "so2dr_plan_candidates", "so2dr_plan_tuned", "so2dr_autotune",
           "so2dr_measure_link", "so2dr_run_timeline"]


class So2drError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_strerror(code), code, msg))
        self.code = code


class PlanInfo(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("dims", ctypes.c_int64 * 3), ("radius", ctypes.c_int),
                ("kind", ctypes.c_int), ("dtype", ctypes.c_int), ("time_steps", ctypes.c_int64),
                ("k_off", ctypes.c_int), ("k_on", ctypes.c_int), ("rounds", ctypes.c_int),
                ("chunks", ctypes.c_int), ("n_streams", ctypes.c_int),
                ("max_chunk_planes", ctypes.c_int64), ("ring_planes", ctypes.c_int64),
                ("plane_bytes", ctypes.c_int64), ("arena_bytes", ctypes.c_size_t),
                ("arena_bytes_in_core", ctypes.c_size_t), ("host_workspace_bytes", ctypes.c_size_t),
                ("ops_per_run", ctypes.c_int64), ("launches_per_run", ctypes.c_int64),
                ("h2d_bytes_per_run", ctypes.c_double), ("d2h_bytes_per_run", ctypes.c_double),
                ("cell_updates_per_run", ctypes.c_double), ("redundancy", ctypes.c_double),
                ("lookahead", ctypes.c_int), ("out_slabs", ctypes.c_int),
                ("arena_bytes_result_reuse", ctypes.c_size_t), ("result_reuse_chunks", ctypes.c_int),
                ("zero_copy", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("total_ms", ctypes.c_double), ("kernel_ms", ctypes.c_double),
                ("h2d_ms", ctypes.c_double), ("d2h_ms", ctypes.c_double),
                ("h2d_bytes", ctypes.c_double), ("d2h_bytes", ctypes.c_double),
                ("launches", ctypes.c_int64), ("ops", ctypes.c_int64),
                ("gcells_per_s", ctypes.c_double), ("main_kernel_ms", ctypes.c_double),
                ("main_kernel_launches", ctypes.c_int64), ("main_kernel_cells", ctypes.c_double)]


class OpRec(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("stream", ctypes.c_int), ("round", ctypes.c_int),
                ("chunk", ctypes.c_int), ("depth", ctypes.c_int), ("edge_lo", ctypes.c_int),
                ("edge_hi", ctypes.c_int), ("src_buf", ctypes.c_int), ("dst_buf", ctypes.c_int),
                ("src_lo", ctypes.c_int64), ("src_hi", ctypes.c_int64), ("src_slot0", ctypes.c_int64),
                ("dst_lo", ctypes.c_int64), ("dst_hi", ctypes.c_int64), ("dst_slot0", ctypes.c_int64),
                ("wait_op", ctypes.c_int64 * 4)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("k_off", ctypes.c_int), ("k_on", ctypes.c_int), ("chunks", ctypes.c_int),
                ("lookahead", ctypes.c_int), ("out_slabs", ctypes.c_int), ("status", ctypes.c_int),
                ("predicted_ms", ctypes.c_double), ("measured_ms", ctypes.c_double)]


class BufRec(ctypes.Structure):
    _fields_ = [("offset_bytes", ctypes.c_int64), ("capacity_planes", ctypes.c_int64)]


_lib = None


def load_library(path=None):
    """Loads (building if needed) libso2dr.so.  Raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libso2dr.so is not built; run __graft_entry__.build() "
                               "(the CUDA extension is required, there is no fallback)")
    lib = ctypes.CDLL(path)
    vp, i64, i64p, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), \
        ctypes.POINTER(ctypes.c_double)
    c_int, c_size = ctypes.c_int, ctypes.c_size_t
    planp = ctypes.POINTER(ctypes.c_void_p)
    lib.so2dr_plan_ex.argtypes = [planp, c_int, i64p, c_int, c_int, dp, c_int, i64, c_int, c_int,
                                  c_int, c_size, c_int, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double]
    lib.so2dr_plan.argtypes = [planp, c_int, i64p, c_int, c_int, dp, c_int, i64, c_int, c_int, c_int,
                               c_size, c_int]
    lib.so2dr_plan_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
    lib.so2dr_plan_chunks.argtypes = [vp, i64p, c_int]
    lib.so2dr_plan_ops.argtypes = [vp, c_int, ctypes.POINTER(OpRec), i64, i64p]
    lib.so2dr_plan_buffers.argtypes = [vp, c_int, ctypes.POINTER(BufRec), c_int, ctypes.POINTER(c_int)]
    lib.so2dr_bind.argtypes = [vp, vp, c_size, ctypes.POINTER(vp), c_int]
    lib.so2dr_run.argtypes = [vp, vp, vp, c_int, ctypes.POINTER(Stats)]
    lib.so2dr_adjoint.argtypes = [vp, vp, vp, vp, vp, vp, vp, c_size, c_int, dp, ctypes.POINTER(Stats)]
    lib.so2dr_loss.argtypes = [vp, vp, vp, vp, vp, c_size, dp]
    lib.so2dr_dot.argtypes = [vp, vp, vp, i64, c_int, dp]
    lib.so2dr_run_device_noalloc.argtypes = [c_int, i64p, c_int, c_int, dp, c_int, i64, c_int, c_int, vp, vp, vp]
    tep = ctypes.POINTER(TuneEntry)
    lib.so2dr_plan_candidates.argtypes = [c_int, i64p, c_int, c_int, dp, c_int, i64, c_int, c_int, c_int,
                                          c_size, c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          tep, c_int, ctypes.POINTER(c_int)]
    lib.so2dr_plan_tuned.argtypes = [planp, c_int, i64p, c_int, c_int, dp, c_int, i64, tep, c_size, c_int]
    lib.so2dr_autotune.argtypes = [c_int, i64p, c_int, c_int, dp, c_int, i64, c_int, c_int, c_int, c_size,
                                   c_int, vp, ctypes.POINTER(vp), c_int, vp, c_int, c_int, tep, c_int,
                                   ctypes.POINTER(c_int), dp]
    lib.so2dr_measure_link.argtypes = [vp, vp, vp, c_size, c_int, c_int, dp]
    lib.so2dr_run_timeline.argtypes = [vp, dp, dp, i64, i64p]
    lib.so2dr_destroy.argtypes = [vp]
    lib.so2dr_destroy.restype = None
    lib.so2dr_strerror.argtypes = [c_int]
    lib.so2dr_strerror.restype = ctypes.c_char_p
    lib.so2dr_last_error.argtypes = []
    lib.so2dr_last_error.restype = ctypes.c_char_p
    lib.so2dr_abi_version.restype = c_int
    _lib = lib
    return lib


def _strerror(code):
    return load_library().so2dr_strerror(code).decode()


def _check(rc):
    if rc != OK:
        raise So2drError(rc, load_library().so2dr_last_error().decode())


def _ptr(t):
    """Data pointer of a torch tensor or numpy array."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t.ctypes.data)


def _stats_dict(s):
    return {k: getattr(s, k) for k, _ in Stats._fields_}


class Plan:
    """A planned SO2DR sweep (so2dr_plan).  Host-only until bind()."""

    def __init__(self, dims, radius=1, kind="star", coeffs=None, time_steps=1, min_chunks=1,
                 k_on=0, k_off=0, budget_bytes=1 << 30, dtype="f32", link_gbs=(0.0, 0.0),
                 hbm_gbs=0.0, tune_entry=None):
        """tune_entry: a row of candidates()/autotune() (so2dr_plan_tuned);
        it replaces min_chunks, k_on, k_off and the link rates."""
        lib = load_library()
        self.kind = KINDS[kind] if isinstance(kind, str) else int(kind)
        self.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        self.dims = tuple(int(x) for x in dims)
        c = None if coeffs is None else np.ascontiguousarray(coeffs, dtype=np.float64)
        self._coeffs = c
        h = ctypes.c_void_p()
        d = (ctypes.c_int64 * len(self.dims))(*self.dims)
        cp = None if c is None else c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        nc = 0 if c is None else int(c.size)
        if tune_entry is not None:
            e = _entry_struct(tune_entry)
            rc = lib.so2dr_plan_tuned(ctypes.byref(h), len(self.dims), d, int(radius), self.kind, cp, nc,
                                      int(time_steps), ctypes.byref(e), int(budget_bytes), self.dtype)
        else:
            rc = lib.so2dr_plan_ex(ctypes.byref(h), len(self.dims), d, int(radius), self.kind, cp, nc,
                                   int(time_steps), int(min_chunks), int(k_on), int(k_off),
                                   int(budget_bytes), self.dtype, float(link_gbs[0]), float(link_gbs[1]),
                                   float(hbm_gbs))
        _check(rc)
        self._h = h
        self._budget = int(budget_bytes)
        self._arena = None
        self._streams = None
        self._bound_in_core = None

    # ------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_h", None):
            load_library().so2dr_destroy(self._h)
            self._h = None
        self._arena = None
        self._streams = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------ introspection
    @property
    def info(self):
        i = PlanInfo()
        _check(load_library().so2dr_plan_info(self._h, ctypes.byref(i)))
        out = {k: getattr(i, k) for k, _ in PlanInfo._fields_}
        out["dims"] = tuple(i.dims)
        return out

    def chunks(self):
        n = self.info["chunks"]
        buf = (ctypes.c_int64 * (n + 1))()
        _check(load_library().so2dr_plan_chunks(self._h, buf, n + 1))
        return np.array(buf, dtype=np.int64)

    def ops(self, in_core=False):
        lib = load_library()
        n = ctypes.c_int64()
        _check(lib.so2dr_plan_ops(self._h, int(in_core), None, 0, ctypes.byref(n)))
        arr = (OpRec * n.value)()
        _check(lib.so2dr_plan_ops(self._h, int(in_core), arr, n.value, ctypes.byref(n)))
        return [{k: (tuple(getattr(o, k)) if k == "wait_op" else getattr(o, k)) for k, _ in OpRec._fields_}
                for o in arr]

    def buffers(self, in_core=False):
        lib = load_library()
        n = ctypes.c_int()
        _check(lib.so2dr_plan_buffers(self._h, int(in_core), None, 0, ctypes.byref(n)))
        arr = (BufRec * n.value)()
        _check(lib.so2dr_plan_buffers(self._h, int(in_core), arr, n.value, ctypes.byref(n)))
        return [(b.offset_bytes, b.capacity_planes) for b in arr]

    # ------------------------------------------------------------ execution
    def bind(self, in_core=False, arena=None, streams=None):
        """Lends a torch device arena and four torch streams to the plan
        (in_core: 0 out-of-core, 1 in-core, 2 the result-reuse code)."""
        import torch
        info = self.info
        mode = int(in_core)
        need = (info["arena_bytes_in_core"] if mode == 1 else
                info["arena_bytes_result_reuse"] if mode == 2 else info["arena_bytes"])
        if self.kind == VARCOEF_STAR and not in_core and self._budget:
            # the adjoint's pipelines fit their own chunkings into the bound arena
            need = max(need, self._budget)
        if arena is None:
            arena = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
        if streams is None:
            streams = [torch.cuda.Stream() for _ in range(4)]
        hs = (ctypes.c_void_p * len(streams))(*[ctypes.c_void_p(s.cuda_stream) for s in streams])
        _check(load_library().so2dr_bind(self._h, ctypes.c_void_p(arena.data_ptr()),
                                         arena.numel() * arena.element_size(), hs, len(streams)))
        self._arena = arena
        self._streams = streams
        self._bound_in_core = mode
        return self

    def run(self, host_grid, coeff_fields=None, in_core=False, stats=True):
        """Advances host_grid (pinned CPU tensor of the plan's dtype) in place."""
        if self._arena is None or int(in_core) != self._bound_in_core:
            self.bind(in_core=in_core)
        st = Stats()
        _check(load_library().so2dr_run(self._h, _ptr(host_grid), _ptr(coeff_fields), int(in_core),
                                         ctypes.byref(st) if stats else None))
        return _stats_dict(st) if stats else None

    def timeline(self, in_core=False):
        """Per-op (start_ms, end_ms) of the last run made with stats, joined
        with the op records of that mode (so2dr_run_timeline)."""
        lib = load_library()
        n = ctypes.c_int64()
        _check(lib.so2dr_run_timeline(self._h, None, None, 0, ctypes.byref(n)))
        a = (ctypes.c_double * max(1, n.value))()
        b = (ctypes.c_double * max(1, n.value))()
        _check(lib.so2dr_run_timeline(self._h, a, b, n.value, ctypes.byref(n)))
        ops = self.ops(in_core)
        if len(ops) != n.value:
            raise So2drError(E_INVAL, "the last timed run replayed another op list")
        return [dict(o, start_ms=a[j], end_ms=b[j]) for j, o in enumerate(ops)]

    def adjoint(self, u0, coeff_fields, target, grad_u0, grad_coeffs, workspace, checkpoint_every=8,
                stats=True):
        if self._arena is None or self._bound_in_core != 0:
            self.bind()
        loss = ctypes.c_double()
        st = Stats()
        nbytes = workspace.numel() * workspace.element_size()
        _check(load_library().so2dr_adjoint(self._h, _ptr(u0), _ptr(coeff_fields), _ptr(target),
                                            _ptr(grad_u0), _ptr(grad_coeffs), _ptr(workspace), nbytes,
                                            int(checkpoint_every), ctypes.byref(loss),
                                            ctypes.byref(st) if stats else None))
        return loss.value, (_stats_dict(st) if stats else None)

    def loss(self, u0, coeff_fields, target, workspace):
        if self._arena is None:
            self.bind()
        loss = ctypes.c_double()
        nbytes = workspace.numel() * workspace.element_size()
        _check(load_library().so2dr_loss(self._h, _ptr(u0), _ptr(coeff_fields), _ptr(target),
                                         _ptr(workspace), nbytes, ctypes.byref(loss)))
        return loss.value

    def workspace(self, checkpoint_every=8):
        """Pinned host workspace so2dr_adjoint needs: (segments + C - 1) grids."""
        import torch
        info = self.info
        T, C = info["time_steps"], int(checkpoint_every)
        S = max(1, -(-T // C))
        grid = info["dims"][0] * info["dims"][1] * max(1, info["dims"][2]) * (8 if self.dtype == F64 else 4)
        return torch.empty((S + C - 1) * grid, dtype=torch.uint8).pin_memory()

    def dot(self, a, b):
        if self._arena is None:
            self.bind()
        out = ctypes.c_double()
        dt = F64 if str(a.dtype).endswith("float64") else F32
        _check(load_library().so2dr_dot(self._h, _ptr(a), _ptr(b), int(a.numel()), dt, ctypes.byref(out)))
        return out.value


def _entry_struct(e):
    t = TuneEntry()
    for k, _ in TuneEntry._fields_:
        setattr(t, k, e.get(k, -1.0 if k == "measured_ms" else 0))
    return t


def _problem(dims, kind, coeffs):
    dims = tuple(int(x) for x in dims)
    c = None if coeffs is None else np.ascontiguousarray(coeffs, dtype=np.float64)
    cp = None if c is None else c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return (dims, (ctypes.c_int64 * len(dims))(*dims), KINDS[kind] if isinstance(kind, str) else int(kind),
            c, cp, 0 if c is None else int(c.size))


def candidates(dims, radius=1, kind="star", coeffs=None, time_steps=1, min_chunks=1, k_on=0, k_off=0,
               budget_bytes=1 << 30, dtype="f32", link_gbs=(0.0, 0.0), hbm_gbs=0.0):
    """Every feasible point of the planner's search, cheapest predicted first
    (so2dr_plan_candidates; host only)."""
    lib = load_library()
    dims, d, kd, c, cp, nc = _problem(dims, kind, coeffs)
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    n = ctypes.c_int()
    args = [len(dims), d, int(radius), kd, cp, nc, int(time_steps), int(min_chunks), int(k_on), int(k_off),
            int(budget_bytes), dt, float(link_gbs[0]), float(link_gbs[1]), float(hbm_gbs)]
    _check(lib.so2dr_plan_candidates(*args, None, 0, ctypes.byref(n)))
    arr = (TuneEntry * max(1, n.value))()
    _check(lib.so2dr_plan_candidates(*args, arr, n.value, ctypes.byref(n)))
    return [{k: getattr(e, k) for k, _ in TuneEntry._fields_} for e in arr[:n.value]]


def autotune(dims, radius=1, kind="star", coeffs=None, time_steps=1, budget_bytes=1 << 30, dtype="f32",
             scratch=None, arena=None, streams=None, max_candidates=8, repeats=2, min_chunks=1, k_on=0,
             k_off=0):
    """Measured autotune (so2dr_autotune): returns (table sorted by measured
    time, (h2d, d2h, hbm) GB/s).  scratch is a pinned host grid of the
    problem's shape and dtype; its contents are overwritten."""
    import torch
    lib = load_library()
    dims, d, kd, c, cp, nc = _problem(dims, kind, coeffs)
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    if arena is None:
        arena = torch.empty(int(budget_bytes), dtype=torch.uint8, device="cuda")
    if streams is None:
        streams = [torch.cuda.Stream() for _ in range(4)]
    hs = (ctypes.c_void_p * len(streams))(*[ctypes.c_void_p(s.cuda_stream) for s in streams])
    cap = 4096
    arr = (TuneEntry * cap)()
    n = ctypes.c_int()
    link = (ctypes.c_double * 3)()
    _check(lib.so2dr_autotune(len(dims), d, int(radius), kd, cp, nc, int(time_steps), int(min_chunks), int(k_on),
                              int(k_off), int(budget_bytes), dt, ctypes.c_void_p(arena.data_ptr()), hs,
                              len(streams), _ptr(scratch), int(max_candidates), int(repeats), arr, cap,
                              ctypes.byref(n), link))
    return [{k: getattr(e, k) for k, _ in TuneEntry._fields_} for e in arr[:min(cap, n.value)]], tuple(link)


LINK_KEYS = ("ce_h2d", "ce_d2h", "ce_both_h2d", "ce_both_d2h", "sm_h2d", "sm_d2h", "sm_both_h2d", "sm_both_d2h",
             "hbm")


def measure_link(bytes_=1 << 30, sm_ctas=64, repeats=3):
    """Host-link and HBM rates in GB/s (so2dr_measure_link): copy engines and
    SM-driven copies over the mapped pinned buffers, each direction alone and
    both at once, and an on-device copy."""
    import torch
    lib = load_library()
    a = torch.empty(int(bytes_), dtype=torch.uint8).pin_memory()
    b = torch.empty(int(bytes_), dtype=torch.uint8).pin_memory()
    arena = torch.empty(2 * int(bytes_), dtype=torch.uint8, device="cuda")
    out = (ctypes.c_double * 9)()
    _check(lib.so2dr_measure_link(_ptr(a), _ptr(b), ctypes.c_void_p(arena.data_ptr()), int(bytes_), int(sm_ctas),
                                  int(repeats), out))
    return dict(zip(LINK_KEYS, list(out)))


def _varcoef_loss_fn():
    import torch

    class VarcoefLoss(torch.autograd.Function):
        """L = 1/2 ||u_T - u*||^2 of the variable-coefficient sweep, with
        gradients w.r.t. the initial field and the six face fields from the
        out-of-core adjoint (so2dr_adjoint)."""

        @staticmethod
        def forward(ctx, u0, faces, target, plan, checkpoint_every):
            pin = lambda t: t.detach().contiguous() if t.is_pinned() else t.detach().contiguous().pin_memory()
            u0p, fp, tp = pin(u0), pin(faces), pin(target)
            gu = torch.empty_like(u0p).pin_memory()
            gc = torch.empty_like(fp).pin_memory()
            ws = plan.workspace(checkpoint_every)
            loss, _ = plan.adjoint(u0p, fp, tp, gu, gc, ws, checkpoint_every, stats=False)
            ctx.save_for_backward(gu, gc)
            return torch.tensor(loss, dtype=torch.float64)

        @staticmethod
        def backward(ctx, g):
            gu, gc = ctx.saved_tensors
            return (g * gu).to(gu.dtype), (g * gc).to(gc.dtype), None, None, None

    return VarcoefLoss


_VL = None


def varcoef_loss(u0, faces, target, plan, checkpoint_every=8):
    """Differentiable loss through the out-of-core pipeline (torch.autograd)."""
    global _VL
    if _VL is None:
        _VL = _varcoef_loss_fn()
    return _VL.apply(u0, faces, target, plan, checkpoint_every)
