"""Pins for the FP64 oracle against things other than itself: closed forms
(sin-mode eigenvalues), a library routine (scipy.ndimage.correlate), invariants
(constant fields, linearity, first moments, the adjoint identity), brute-force
matrices on tiny grids, FP64 finite differences and the paper's Table III."""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2309_08864_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ helpers

def my_offsets(ndim, r, kind):
    """Independent reading of the documented coefficient-table order."""
    if kind == oracle.STAR:
        offs = [(0,) * ndim]
        for a in range(ndim):
            for j in range(1, r + 1):
                for s in (-j, +j):
                    o = [0] * ndim
                    o[a] = s
                    offs.append(tuple(o))
        return offs
    if kind == oracle.BOX:
        return list(itertools.product(range(-r, r + 1), repeat=ndim))
    raise ValueError


def interior_mask(shape, r):
    m = np.zeros(shape, dtype=bool)
    m[tuple(slice(r, n - r) for n in shape)] = True
    return m


def dense_matrix(shape, r, offs, coeffs):
    """A as an explicit N x N matrix, row p = stencil weights for interior p,
    identity row otherwise."""
    N = int(np.prod(shape))
    A = np.zeros((N, N))
    idx = np.arange(N).reshape(shape)
    mask = interior_mask(shape, r)
    for p in itertools.product(*[range(n) for n in shape]):
        i = idx[p]
        if not mask[p]:
            A[i, i] = 1.0
            continue
        for o, c in zip(offs, coeffs):
            q = tuple(pa + oa for pa, oa in zip(p, o))
            A[i, idx[q]] += c
    return A


def dense_varcoef(shape, faces):
    N = int(np.prod(shape))
    nd = len(shape)
    A = np.zeros((N, N))
    idx = np.arange(N).reshape(shape)
    mask = interior_mask(shape, 1)
    for p in itertools.product(*[range(n) for n in shape]):
        i = idx[p]
        if not mask[p]:
            A[i, i] = 1.0
            continue
        csum = 0.0
        for a in range(nd):
            for s, f in ((-1, 2 * a), (+1, 2 * a + 1)):
                q = list(p)
                q[a] += s
                A[i, idx[tuple(q)]] += faces[f][p]
                csum += faces[f][p]
        A[i, i] += 1.0 - csum
    return A


def rel_linf(x, ref):
    return np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300)


# ------------------------------------------------------------ offset tables

@pytest.mark.parametrize("ndim,r,kind", [(2, 1, 0), (3, 1, 0), (3, 4, 0), (2, 3, 0),
                                         (2, 1, 1), (2, 4, 1), (3, 1, 1)])
def test_offset_order_matches_documented_order(ndim, r, kind):
    got = [tuple(o) for o in oracle.offsets(ndim, r, kind)]
    assert got == my_offsets(ndim, r, kind)


def test_table3_box_point_and_flop_counts():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table3_box_stencils.txt"))
            if l.strip() and not l.startswith("#")]
    for x, pts, flops in ((int(a), int(b), int(c)) for a, b, c in rows):
        n = len(oracle.offsets(2, x, oracle.BOX))
        assert n == pts
        assert 2 * n - 1 == flops  # n multiplies + (n - 1) adds per element


# --------------------------------------------------------- sin-mode pins

@pytest.mark.parametrize("ks", [(1, 1), (2, 3), (5, 1), (7, 8)])
def test_sin_mode_eigenvalue_2d_5pt(ks):
    m = (13, 9)
    shape = tuple(x + 2 for x in m)
    i = np.arange(shape[0])[:, None]
    j = np.arange(shape[1])[None, :]
    th = [ks[0] * np.pi / (m[0] + 1), ks[1] * np.pi / (m[1] + 1)]
    u0 = np.sin(th[0] * i) * np.sin(th[1] * j)
    lam = 0.2 * (1 + 2 * np.cos(th[0]) + 2 * np.cos(th[1]))
    T = 6  # keeps |lam|^T far above the rounding floor for every mode tested
    uT = oracle.run(u0, [0.2] * 5, 1, oracle.STAR, T)
    ref = lam ** T * u0
    assert abs(lam) ** T > 1e-6
    assert np.max(np.abs(uT - ref)) <= 1e-14 * T


@pytest.mark.parametrize("ks", [(1, 1, 1), (2, 1, 3), (4, 4, 1)])
def test_sin_mode_eigenvalue_3d_7pt(ks):
    m = (9, 7, 6)
    shape = tuple(x + 2 for x in m)
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    th = [k * np.pi / (mm + 1) for k, mm in zip(ks, m)]
    u0 = np.ones(shape)
    for g, t in zip(grids, th):
        u0 = u0 * np.sin(t * g)
    lam = 0.4 + 0.2 * sum(np.cos(t) for t in th)
    T = 12
    uT = oracle.run(u0, [0.4] + [0.1] * 6, 1, oracle.STAR, T)
    assert abs(lam) ** T > 1e-3
    assert np.max(np.abs(uT - lam ** T * u0)) <= 1e-14 * T


def test_varcoef_constant_faces_is_the_7pt_eigenproblem():
    m = (6, 5, 7)
    shape = tuple(x + 2 for x in m)
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    ks = (1, 2, 1)
    th = [k * np.pi / (mm + 1) for k, mm in zip(ks, m)]
    u0 = np.ones(shape)
    for g, t in zip(grids, th):
        u0 = u0 * np.sin(t * g)
    faces = np.full((6,) + shape, 0.1)
    lam = 0.4 + 0.2 * sum(np.cos(t) for t in th)
    uT = oracle.run_varcoef(u0, faces, 10)
    assert np.max(np.abs(uT - lam ** 10 * u0)) <= 1e-13


# ------------------------------------------------------- library routine

@pytest.mark.parametrize("shape,r,kind", [((17, 19), 1, 0), ((23, 21), 4, 0), ((12, 13, 11), 1, 0),
                                          ((15, 14, 13), 4, 0), ((16, 18), 2, 1), ((19, 17), 4, 1),
                                          ((9, 10, 8), 1, 1), ((14, 12), 3, 0)])
def test_steps_match_scipy_correlate(shape, r, kind):
    ndi = pytest.importorskip("scipy.ndimage")
    nd = len(shape)
    offs = my_offsets(nd, r, kind)
    rng = np.random.default_rng(3)
    coeffs = rng.uniform(-1, 1, len(offs))  # asymmetric on purpose
    coeffs /= np.abs(coeffs).sum()
    u = rng.uniform(size=shape)
    W = np.zeros((2 * r + 1,) * nd)
    for o, c in zip(offs, coeffs):
        W[tuple(oa + r for oa in o)] += c
    mask = interior_mask(shape, r)
    ref = u.copy()
    T = 5
    for _ in range(T):
        v = ndi.correlate(ref, W, mode="constant", cval=0.0)
        ref = np.where(mask, v, ref)
    got = oracle.run(u, coeffs, r, kind, T)
    assert rel_linf(got, ref) <= 1e-13


# ------------------------------------------------------------- invariants

@pytest.mark.parametrize("shape,r,kind", [((20, 24), 1, 0), ((11, 12, 13), 1, 0), ((19, 18, 17), 4, 0),
                                          ((20, 22), 2, 1)])
def test_constant_field_preserved(shape, r, kind):
    n = len(my_offsets(len(shape), r, kind))
    c = np.random.default_rng(5).uniform(0.5, 1.5, n)
    c /= c.sum()
    u = np.full(shape, 0.7)
    T = 8
    got = oracle.run(u, c, r, kind, T)
    assert np.max(np.abs(got - 0.7)) <= 1e-14 * T


def test_linearity():
    shape = (14, 15, 16)
    rng = np.random.default_rng(9)
    c = rng.uniform(-1, 1, 25)
    u, v = rng.uniform(size=shape), rng.uniform(size=shape)
    al, be = 0.37, -1.9
    lhs = oracle.run(al * u + be * v, c, 4, oracle.STAR, 3)
    rhs = al * oracle.run(u, c, 4, oracle.STAR, 3) + be * oracle.run(v, c, 4, oracle.STAR, 3)
    assert rel_linf(lhs, rhs) <= 1e-12


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_first_moment_drift_radius4(axis):
    """For weights summing to 1 with first moment m, a linear field g.p is
    shifted by g.m per step away from the fixed ring (an affine invariant that
    fails for a swapped offset sign or a wrong axis)."""
    r, T = 4, 3
    shape = (40, 38, 36)
    offs = my_offsets(3, r, oracle.STAR)
    rng = np.random.default_rng(11)
    c = rng.uniform(0.5, 1.5, len(offs))
    c /= c.sum()
    m = np.sum([ci * np.array(o) for ci, o in zip(c, offs)], axis=0)
    g = np.zeros(3)
    g[axis] = 1.0
    grids = np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij")
    u0 = grids[axis].copy()
    got = oracle.run(u0, c, r, oracle.STAR, T)
    inner = tuple(slice(r * (T + 1), n - r * (T + 1)) for n in shape)
    expect = u0 + T * float(g @ m)
    assert np.max(np.abs(got[inner] - expect[inner])) <= 1e-12


# ------------------------------------------------- brute-force matrix powers

@pytest.mark.parametrize("shape,r,kind", [((8, 8), 1, 0), ((4, 4, 4), 1, 0), ((6, 7), 1, 1),
                                          ((10, 10, 10), 4, 0), ((8, 9), 2, 0), ((9, 9), 3, 1)])
def test_matrix_power_bruteforce(shape, r, kind):
    offs = my_offsets(len(shape), r, kind)
    rng = np.random.default_rng(13)
    c = rng.uniform(-0.5, 1.0, len(offs))
    u0 = rng.uniform(size=shape)
    T = 6
    A = dense_matrix(shape, r, offs, c)
    ref = (np.linalg.matrix_power(A, T) @ u0.ravel()).reshape(shape)
    assert rel_linf(oracle.run(u0, c, r, kind, T), ref) <= 1e-13


@pytest.mark.parametrize("shape", [(4, 4, 5), (6, 7), (5, 4, 4)])
def test_varcoef_matrix_power_and_transpose(shape):
    nd = len(shape)
    rng = np.random.default_rng(17)
    faces = rng.uniform(0.05, 0.15, (2 * nd,) + shape)
    u0 = rng.uniform(size=shape)
    A = dense_varcoef(shape, faces)
    T = 5
    ref = (np.linalg.matrix_power(A, T) @ u0.ravel()).reshape(shape)
    assert rel_linf(oracle.run_varcoef(u0, faces, T), ref) <= 1e-13
    lam = rng.normal(size=shape)
    refT = (A.T @ lam.ravel()).reshape(shape)
    assert rel_linf(oracle.apply_varcoef_transpose(lam, faces), refT) <= 1e-13


def test_adjoint_dot_product_identity():
    shape = (9, 8, 10)
    rng = np.random.default_rng(19)
    faces = rng.uniform(0.05, 0.15, (6,) + shape)
    u, lam = rng.normal(size=shape), rng.normal(size=shape)
    lhs = np.vdot(oracle.apply_varcoef_transpose(lam, faces), u)
    rhs = np.vdot(lam, oracle.apply_varcoef(u, faces))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)


# ------------------------------------------------------------------ adjoint

def test_adjoint_gradient_u0_bruteforce():
    shape = (5, 4, 6)
    rng = np.random.default_rng(23)
    faces = rng.uniform(0.05, 0.15, (6,) + shape)
    u0, tgt = rng.uniform(size=shape), rng.uniform(size=shape)
    T = 7
    AT = np.linalg.matrix_power(dense_varcoef(shape, faces), T)
    res = AT @ u0.ravel() - tgt.ravel()
    L, gu, gf = oracle.adjoint_varcoef(u0, faces, tgt, T, ckpt_every=3)
    assert abs(L - 0.5 * res @ res) <= 1e-13 * L
    assert rel_linf(gu, (AT.T @ res).reshape(shape)) <= 1e-12
    # boundary cells carry no coefficient gradient
    ring = ~interior_mask(shape, 1)
    assert np.all(gf[:, ring] == 0)


def test_adjoint_gradient_faces_central_differences():
    shape = (6, 7, 5)
    rng = np.random.default_rng(29)
    faces = rng.uniform(0.05, 0.15, (6,) + shape)
    u0, tgt = rng.uniform(size=shape), rng.uniform(size=shape)
    T = 6
    _, _, gf = oracle.adjoint_varcoef(u0, faces, tgt, T)
    mask = interior_mask(shape, 1)
    for k in range(3):
        v = rng.normal(size=faces.shape) * mask
        eps = 1e-5
        lp = oracle.loss(oracle.run_varcoef(u0, faces + eps * v, T), tgt)
        lm = oracle.loss(oracle.run_varcoef(u0, faces - eps * v, T), tgt)
        fd = (lp - lm) / (2 * eps)
        gv = np.vdot(gf, v)
        assert abs(fd - gv) <= 1e-7 * max(abs(fd), abs(gv))


def test_adjoint_checkpoint_interval_does_not_change_result():
    shape = (7, 6, 6)
    rng = np.random.default_rng(31)
    faces = rng.uniform(0.05, 0.15, (6,) + shape)
    u0, tgt = rng.uniform(size=shape), rng.uniform(size=shape)
    ref = oracle.adjoint_varcoef(u0, faces, tgt, 11, ckpt_every=11)
    for c in (1, 3, 8):
        got = oracle.adjoint_varcoef(u0, faces, tgt, 11, ckpt_every=c)
        assert got[0] == ref[0]
        assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])


# --------------------------------------------------------- dependency cone

def test_dependency_cone_matches_full_run():
    shape = (40, 36, 38)
    r, T = 4, 3
    c = inputs.radius4_star_coeffs()
    u0 = inputs.draw_box(1, shape)
    full = oracle.run(u0, c, r, oracle.STAR, T)
    for lo, hi in (((0, 0, 0), (5, 6, 7)), ((17, 12, 20), (21, 15, 22)), ((35, 30, 33), (40, 36, 38))):
        blo, bhi = oracle.cone_box(shape, lo, hi, r * T)
        ub = inputs.draw_box(1, shape, blo, bhi)
        got = oracle.run_cone(ub, c, r, oracle.STAR, T, blo, bhi, shape, lo, hi)
        assert np.array_equal(got, full[tuple(slice(l, h) for l, h in zip(lo, hi))])
