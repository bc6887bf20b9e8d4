"""Differentiation form: the out-of-core adjoint (transposed stencil run
backward through the chunked pipeline with host checkpoints) against the FP64
oracle's adjoint, and against central finite differences of the loss."""
import numpy as np
import pytest

import oracle
from paper_2309_08864_gb300 import inputs, so2dr
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def _problem(dims, dtype, seed_u=1, seed_t=2):
    import torch
    cdt = np.float64 if dtype == so2dr.F64 else np.float32
    u0 = inputs.draw_box(seed_u, dims).astype(cdt)
    faces = np.stack([inputs.draw_box(100 + f, dims, a=0.05, b=0.15) for f in range(6)]).astype(cdt)
    tgt = inputs.draw_box(seed_t, dims).astype(cdt)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    return u0, faces, tgt, pin(u0), pin(faces), pin(tgt)


@pytest.mark.parametrize("dtype,dims,T,C,budget,K", [
    (so2dr.F64, (20, 18, 24), 11, 4, 384 << 10, 0),   # 9 chunks, segments 4, 4, 3
    (so2dr.F64, (20, 18, 24), 11, 4, 384 << 10, 3),   # rounds of 3 steps: 3 + 1 per segment of 4
    (so2dr.F32, (24, 20, 28), 11, 4, 256 << 10, 0),   # 11 chunks
    (so2dr.F32, (24, 20, 28), 11, 4, 256 << 10, 2),   # rounds of 2 steps
    (so2dr.F32, (30, 17, 20), 8, 8, 0, 0),            # one segment, 3 chunks
    (so2dr.F32, (30, 17, 20), 8, 8, 0, 8),            # one segment in one adjoint round
    (so2dr.F32, (16, 12, 16), 5, 1, 64 << 10, 0),     # a checkpoint every step, 5 forward chunks
])
def test_adjoint_matches_oracle(dtype, dims, T, C, budget, K, monkeypatch):
    """K > 0 pins the steps per adjoint round (SO2DR_ADJOINT_STEPS): the
    gradient is accumulated over K steps on the device before it goes back."""
    import torch
    if K:
        monkeypatch.setenv("SO2DR_ADJOINT_STEPS", str(K))
    u0, faces, tgt, tu0, tf, tt = _problem(dims, dtype)
    plan = so2dr.Plan(dims, 1, "varcoef", None, T, min_chunks=3, k_on=2, k_off=C, budget_bytes=budget,
                      dtype=dtype)
    gu_ = torch.empty_like(tu0).pin_memory()
    gc_ = torch.empty_like(tf).pin_memory()
    ws = plan.workspace(C)
    loss, st = plan.adjoint(tu0, tf, tt, gu_, gc_, ws, C)
    L, gref_u, gref_c = oracle.adjoint_varcoef(u0.astype(np.float64), faces.astype(np.float64),
                                               tgt.astype(np.float64), T, ckpt_every=C)
    tol = 1e-12 if dtype == so2dr.F64 else 2e-5
    assert abs(loss - L) <= tol * abs(L) * 10
    assert gu.rel_linf(gu_.numpy().astype(np.float64), gref_u) <= tol
    assert gu.rel_linf(gc_.numpy().astype(np.float64), gref_c) <= tol
    # the loss pass alone
    ws1 = torch.empty(u0.nbytes, dtype=torch.uint8).pin_memory()
    assert abs(plan.loss(tu0, tf, tt, ws1) - L) <= tol * abs(L) * 10
    plan.close()


def test_dot_is_fp64_exact_enough():
    import torch
    n = 3_000_001
    a = inputs.draw_box(11, (n,), dist="normal").astype(np.float32)
    b = inputs.draw_box(12, (n,), dist="normal").astype(np.float32)
    plan = so2dr.Plan((20, 18, 24), 1, "varcoef", None, 2, min_chunks=1, k_on=1, k_off=2,
                      budget_bytes=1 << 22, dtype=so2dr.F32)
    got = plan.dot(torch.from_numpy(a).pin_memory(), torch.from_numpy(b).pin_memory())
    ref = float(np.dot(a.astype(np.float64), b.astype(np.float64)))
    assert abs(got - ref) <= 1e-12 * np.sum(np.abs(a.astype(np.float64) * b))
    plan.close()


def fd_check(dims, T, C, budget, n_dirs_u, n_dirs_c, tol, eps_c_rel=1e-3):
    """Central differences of the FP64 loss vs <grad, v> of the FP32 adjoint
    (directions: N(0,1) on interior cells, seeds 1000+k)."""
    import torch
    u0, faces, tgt, tu0, tf, tt = _problem(dims, so2dr.F32)
    p32 = so2dr.Plan(dims, 1, "varcoef", None, T, min_chunks=1, k_on=4, k_off=C, budget_bytes=budget,
                     dtype=so2dr.F32)
    gu_ = torch.empty_like(tu0).pin_memory()
    gc_ = torch.empty_like(tf).pin_memory()
    loss, st = p32.adjoint(tu0, tf, tt, gu_, gc_, p32.workspace(C), C)
    print("ADJOINT %s T=%d: %.1f ms, %.2f Gcell/s (forward + adjoint updates), chunks %d" % (
        dims, T, st["total_ms"], st["gcells_per_s"], p32.info["chunks"]))
    # FP64 copies of the same inputs (FP32 values are exact in FP64)
    p64 = so2dr.Plan(dims, 1, "varcoef", None, T, min_chunks=1, k_on=4, k_off=C, budget_bytes=4 * budget,
                     dtype=so2dr.F64)
    u64, f64, t64 = u0.astype(np.float64), faces.astype(np.float64), tgt.astype(np.float64)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    ws = torch.empty(u64.nbytes, dtype=torch.uint8).pin_memory()
    inner = np.zeros(dims, dtype=bool)
    inner[1:-1, 1:-1, 1:-1] = True
    errs = []
    for k in range(n_dirs_u + n_dirs_c):
        on_u = k < n_dirs_u
        if on_u:
            v = inputs.draw_box(1000 + k, dims, dist="normal") * inner
        else:
            v = inputs.draw_box(1000 + k, (6 * dims[0],) + dims[1:], dist="normal").reshape((6,) + dims)
            v = v * inner[None]
        if on_u:
            eps = 1.0   # L is quadratic in u0: central differences are exact up to rounding
            lp = p64.loss(pin(u64 + eps * v), pin(f64), pin(t64), ws)
            lm = p64.loss(pin(u64 - eps * v), pin(f64), pin(t64), ws)
            gv = p32.dot(gu_.view(-1).to(torch.float64).contiguous().pin_memory(), pin(v.ravel()))
        else:
            eps = eps_c_rel * float(f64.max())
            lp = p64.loss(pin(u64), pin(f64 + eps * v), pin(t64), ws)
            lm = p64.loss(pin(u64), pin(f64 - eps * v), pin(t64), ws)
            gv = p32.dot(gc_.view(-1).to(torch.float64).contiguous().pin_memory(), pin(v.ravel()))
        fd = (lp - lm) / (2 * eps)
        err = abs(fd - gv) / max(abs(fd), abs(gv))
        errs.append(err)
        assert err <= tol, (k, fd, gv, err)
    p32.close()
    p64.close()
    return max(errs)


def test_adjoint_finite_differences_small():
    fd_check((40, 36, 44), 16, 8, 2 << 20, 2, 2, 1e-4)


def test_autograd_function():
    import torch
    dims, T, C = (18, 16, 20), 6, 3
    u0, faces, tgt, tu0, tf, tt = _problem(dims, so2dr.F32)
    plan = so2dr.Plan(dims, 1, "varcoef", None, T, min_chunks=2, k_on=2, k_off=C, budget_bytes=1 << 20,
                      dtype=so2dr.F32)
    x = torch.from_numpy(u0.copy()).requires_grad_(True)
    c = torch.from_numpy(faces.copy()).requires_grad_(True)
    L = so2dr.varcoef_loss(x, c, torch.from_numpy(tgt), plan, C)
    L.backward()
    Lr, gr_u, gr_c = oracle.adjoint_varcoef(u0.astype(np.float64), faces.astype(np.float64),
                                            tgt.astype(np.float64), T, ckpt_every=C)
    assert abs(L.item() - Lr) <= 1e-5 * Lr
    assert gu.rel_linf(x.grad.numpy().astype(np.float64), gr_u) <= 2e-5
    assert gu.rel_linf(c.grad.numpy().astype(np.float64), gr_c) <= 2e-5
    plan.close()
