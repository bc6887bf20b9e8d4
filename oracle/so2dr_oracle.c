/*
 * so2dr_oracle.c -- plain, slow, FP64 reference implementation of what the
 * SO2DR hot path computes.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path
 * (the CUDA library and its Python binding) never calls, links or imports it,
 * and it shares no code, header, table or constant with that path.
 *
 * What it computes (paper Sec. I and Sec. II-A, Fig. 1a): a stencil sweep updates
 * every element of an array from the values of its neighbours with a fixed
 * template.  SO2DR (Sec. IV, Algorithm 1, Sec. IV-B) only reorganises that
 * sweep -- chunking, region sharing and redundant trapezoid computation all
 * recompute the same values -- so the oracle is the plain definition,
 * time-stepped over the whole grid held in memory:
 *
 *   interior I = { p : r <= p_a < n_a - r for every axis a }
 *   u^{t+1}[p] = sum_{o in O} c_o * u^t[p+o]   for p in I
 *   u^{t+1}[p] = u^t[p]                        otherwise (fixed Dirichlet ring)
 *
 * Offsets O and the order of the coefficient table:
 *   STAR (kind 0): index 0 is the centre; then for axis a = 0..D-1 and
 *                  j = 1..r: -j*e_a, then +j*e_a.              (1 + 2rD points)
 *   BOX  (kind 1): every o with max_a |o_a| <= r, lexicographic with axis 0
 *                  the slowest and each component running -r..r. ((2r+1)^D)
 *   VARCOEF_STAR (kind 2, r = 1): per-cell face weights c_f[p] for the faces
 *                  f = 2a (-e_a) and f = 2a+1 (+e_a); centre 1 - sum_f c_f[p].
 *
 * Arrays are row-major with axis 0 the slowest; D is 2 or 3.
 * Everything is FP64 and out-of-place (two buffers per step).
 *
 * Adjoint of the variable-coefficient sweep (u_{t+1} = A u_t,
 * L = 1/2 ||u_T - u*||^2):
 *   lambda_T = u_T - u*,  lambda_t = A^T lambda_{t+1},  dL/du_0 = lambda_0
 *   (A^T l)[q] = [q not in I] l[q] + [q in I] c_c[q] l[q]
 *                + sum_f [q - e_f in I] c_f[q - e_f] l[q - e_f]
 *   dL/dc_f[p] = sum_t lambda_{t+1}[p] (u_t[p + e_f] - u_t[p]),  p in I
 * States are recomputed from checkpoints stored every `ckpt_every` steps.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_STAR 0
#define OR_BOX 1
#define OR_VARCOEF_STAR 2

/* -------------------------------------------------------------- geometry */

typedef struct {
    int nd;          /* 2 or 3 */
    int64_t n[3];    /* extents; unused trailing axes are 1 */
    int64_t st[3];   /* row-major strides in elements */
    int64_t cells;
} grid_t;

static int make_grid(grid_t* g, int ndim, const int64_t* dims) {
    if (ndim != 2 && ndim != 3) return -1;
    g->nd = ndim;
    g->n[0] = g->n[1] = g->n[2] = 1;
    for (int a = 0; a < ndim; ++a) {
        if (dims[a] <= 0) return -1;
        g->n[a] = dims[a];
    }
    g->st[2] = 1;
    g->st[1] = (ndim == 3) ? g->n[2] : 1;
    g->st[0] = (ndim == 3) ? g->n[1] * g->n[2] : g->n[1];
    if (ndim == 2) { g->st[1] = 1; g->st[2] = 0; }
    g->cells = g->n[0] * g->n[1] * g->n[2];
    return 0;
}

/* p in I for the cell with coordinates c[0..nd-1] */
static int is_interior(const grid_t* g, const int64_t* c, int r) {
    for (int a = 0; a < g->nd; ++a)
        if (c[a] < r || c[a] >= g->n[a] - r) return 0;
    return 1;
}

/* coordinates of flat index idx */
static void coords(const grid_t* g, int64_t idx, int64_t* c) {
    if (g->nd == 3) {
        c[0] = idx / (g->n[1] * g->n[2]);
        int64_t rem = idx % (g->n[1] * g->n[2]);
        c[1] = rem / g->n[2];
        c[2] = rem % g->n[2];
    } else {
        c[0] = idx / g->n[1];
        c[1] = idx % g->n[1];
        c[2] = 0;
    }
}

/* ------------------------------------------------------------- offsets */

int oracle_num_offsets(int ndim, int radius, int kind) {
    if ((ndim != 2 && ndim != 3) || radius < 1) return -1;
    if (kind == OR_STAR) return 1 + 2 * radius * ndim;
    if (kind == OR_BOX) {
        int w = 2 * radius + 1, n = 1;
        for (int a = 0; a < ndim; ++a) n *= w;
        return n;
    }
    if (kind == OR_VARCOEF_STAR) return radius == 1 ? 2 * ndim : -1;
    return -1;
}

/* Writes the offsets as out[3*k + a] (a = 0..2, unused axes 0). */
int oracle_offsets(int ndim, int radius, int kind, int* out) {
    int n = oracle_num_offsets(ndim, radius, kind);
    if (n < 0) return -1;
    memset(out, 0, sizeof(int) * 3 * (size_t)n);
    if (kind == OR_STAR) {
        int k = 1; /* k = 0 is the centre, all zeros */
        for (int a = 0; a < ndim; ++a)
            for (int j = 1; j <= radius; ++j) {
                out[3 * k + a] = -j; ++k;
                out[3 * k + a] = +j; ++k;
            }
    } else if (kind == OR_BOX) {
        int w = 2 * radius + 1;
        for (int k = 0; k < n; ++k) {
            int rem = k;
            for (int a = ndim - 1; a >= 0; --a) { /* last axis fastest */
                out[3 * k + a] = rem % w - radius;
                rem /= w;
            }
        }
    } else { /* faces: f = 2a -> -e_a, f = 2a+1 -> +e_a */
        for (int a = 0; a < ndim; ++a) {
            out[3 * (2 * a) + a] = -1;
            out[3 * (2 * a + 1) + a] = +1;
        }
    }
    return n;
}

static int64_t offset_stride(const grid_t* g, const int* o) {
    int64_t s = 0;
    for (int a = 0; a < g->nd; ++a) s += (int64_t)o[a] * g->st[a];
    return s;
}

/* ------------------------------------------------- constant coefficients */

static void step_const(const grid_t* g, int r, int npts, const int64_t* ost,
                       const double* c, const double* u, double* v) {
    int64_t plane = g->st[0];
#pragma omp parallel for schedule(static)
    for (int64_t i0 = 0; i0 < g->n[0]; ++i0) {
        for (int64_t rem = 0; rem < plane; ++rem) {
            int64_t idx = i0 * plane + rem;
            int64_t cc[3];
            coords(g, idx, cc);
            if (!is_interior(g, cc, r)) { v[idx] = u[idx]; continue; }
            double acc = 0.0;
            for (int k = 0; k < npts; ++k) acc += c[k] * u[idx + ost[k]];
            v[idx] = acc;
        }
    }
}

/* u (in/out): steps applications of the constant-coefficient stencil. */
int oracle_run_const(int ndim, const int64_t* dims, int radius, int kind,
                     const double* coeffs, double* u, int64_t steps) {
    grid_t g;
    if (make_grid(&g, ndim, dims) || (kind != OR_STAR && kind != OR_BOX) || steps < 0) return -1;
    int npts = oracle_num_offsets(ndim, radius, kind);
    if (npts <= 0) return -1;
    int* offs = (int*)malloc(sizeof(int) * 3 * (size_t)npts);
    int64_t* ost = (int64_t*)malloc(sizeof(int64_t) * (size_t)npts);
    double* tmp = (double*)malloc(sizeof(double) * (size_t)g.cells);
    if (!offs || !ost || !tmp) { free(offs); free(ost); free(tmp); return -2; }
    oracle_offsets(ndim, radius, kind, offs);
    for (int k = 0; k < npts; ++k) ost[k] = offset_stride(&g, offs + 3 * k);
    double* a = u; double* b = tmp;
    for (int64_t t = 0; t < steps; ++t) {
        step_const(&g, radius, npts, ost, coeffs, a, b);
        double* s = a; a = b; b = s;
    }
    if (a != u) memcpy(u, a, sizeof(double) * (size_t)g.cells);
    free(offs); free(ost); free(tmp);
    return 0;
}

/* ------------------------------------------------- variable coefficients */

static void face_strides(const grid_t* g, int64_t* fst) {
    for (int a = 0; a < g->nd; ++a) {
        fst[2 * a] = -g->st[a];
        fst[2 * a + 1] = +g->st[a];
    }
}

static void step_varcoef(const grid_t* g, const double* cf, const double* u, double* v) {
    int nf = 2 * g->nd;
    int64_t fst[6];
    face_strides(g, fst);
    int64_t plane = g->st[0], N = g->cells;
#pragma omp parallel for schedule(static)
    for (int64_t i0 = 0; i0 < g->n[0]; ++i0) {
        for (int64_t rem = 0; rem < plane; ++rem) {
            int64_t idx = i0 * plane + rem;
            int64_t cc[3];
            coords(g, idx, cc);
            if (!is_interior(g, cc, 1)) { v[idx] = u[idx]; continue; }
            double csum = 0.0, acc = 0.0;
            for (int f = 0; f < nf; ++f) {
                double w = cf[(int64_t)f * N + idx];
                csum += w;
                acc += w * u[idx + fst[f]];
            }
            v[idx] = (1.0 - csum) * u[idx] + acc;
        }
    }
}

/* A^T applied to lam, gather form (see the header). */
static void step_varcoef_T(const grid_t* g, const double* cf, const double* lam, double* out) {
    int nf = 2 * g->nd;
    int64_t fst[6];
    face_strides(g, fst);
    int64_t plane = g->st[0], N = g->cells;
#pragma omp parallel for schedule(static)
    for (int64_t i0 = 0; i0 < g->n[0]; ++i0) {
        for (int64_t rem = 0; rem < plane; ++rem) {
            int64_t q = i0 * plane + rem;
            int64_t cq[3];
            coords(g, q, cq);
            double acc;
            if (is_interior(g, cq, 1)) {
                double csum = 0.0;
                for (int f = 0; f < nf; ++f) csum += cf[(int64_t)f * N + q];
                acc = (1.0 - csum) * lam[q];
            } else {
                acc = lam[q];
            }
            for (int f = 0; f < nf; ++f) {
                /* neighbour p = q - e_f; it uses weight c_f[p] on u[p + e_f] = u[q] */
                int a = f / 2, s = (f % 2) ? +1 : -1;
                int64_t cp[3] = {cq[0], cq[1], cq[2]};
                cp[a] -= s;
                if (cp[a] < 0 || cp[a] >= g->n[a]) continue;
                if (!is_interior(g, cp, 1)) continue;
                int64_t p = q - fst[f];
                acc += cf[(int64_t)f * N + p] * lam[p];
            }
            out[q] = acc;
        }
    }
}

int oracle_run_varcoef(int ndim, const int64_t* dims, const double* faces,
                       double* u, int64_t steps) {
    grid_t g;
    if (make_grid(&g, ndim, dims) || steps < 0) return -1;
    double* tmp = (double*)malloc(sizeof(double) * (size_t)g.cells);
    if (!tmp) return -2;
    double* a = u; double* b = tmp;
    for (int64_t t = 0; t < steps; ++t) {
        step_varcoef(&g, faces, a, b);
        double* s = a; a = b; b = s;
    }
    if (a != u) memcpy(u, a, sizeof(double) * (size_t)g.cells);
    free(tmp);
    return 0;
}

int oracle_apply_varcoef(int ndim, const int64_t* dims, const double* faces,
                         const double* u, double* out) {
    grid_t g;
    if (make_grid(&g, ndim, dims)) return -1;
    step_varcoef(&g, faces, u, out);
    return 0;
}

int oracle_apply_varcoef_transpose(int ndim, const int64_t* dims, const double* faces,
                                   const double* lam, double* out) {
    grid_t g;
    if (make_grid(&g, ndim, dims)) return -1;
    step_varcoef_T(&g, faces, lam, out);
    return 0;
}

/* Loss, dL/du_0 (all cells) and dL/dc_f (all cells; zero off the interior). */
int oracle_adjoint_varcoef(int ndim, const int64_t* dims, const double* faces,
                           const double* u0, const double* target, int64_t steps,
                           int64_t ckpt_every, double* grad_u0, double* grad_faces,
                           double* loss) {
    grid_t g;
    if (make_grid(&g, ndim, dims) || steps < 0 || ckpt_every < 1) return -1;
    int64_t N = g.cells;
    int nd = g.nd, nf = 2 * nd;
    int64_t nseg = (steps + ckpt_every - 1) / ckpt_every;
    if (nseg == 0) nseg = 1;
    double* ckpt = (double*)malloc(sizeof(double) * (size_t)(N * nseg));
    double* seg = (double*)malloc(sizeof(double) * (size_t)(N * ckpt_every));
    double* cur = (double*)malloc(sizeof(double) * (size_t)N);
    double* nxt = (double*)malloc(sizeof(double) * (size_t)N);
    if (!ckpt || !seg || !cur || !nxt) { free(ckpt); free(seg); free(cur); free(nxt); return -2; }

    /* forward sweep, keeping u_{j*ckpt_every} */
    memcpy(cur, u0, sizeof(double) * (size_t)N);
    for (int64_t t = 0; t < steps; ++t) {
        if (t % ckpt_every == 0) memcpy(ckpt + (t / ckpt_every) * N, cur, sizeof(double) * (size_t)N);
        step_varcoef(&g, faces, cur, nxt);
        double* s = cur; cur = nxt; nxt = s;
    }
    if (steps == 0) memcpy(ckpt, cur, sizeof(double) * (size_t)N);

    /* lambda_T = u_T - u*,  L = 1/2 sum lambda_T^2 */
    double L = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double d = cur[i] - target[i];
        grad_u0[i] = d;  /* grad_u0 holds lambda from here on */
        L += d * d;
    }
    *loss = 0.5 * L;
    memset(grad_faces, 0, sizeof(double) * (size_t)(N * nf));

    int64_t fst[6];
    face_strides(&g, fst);
    int64_t plane = g.st[0];
    for (int64_t j = nseg - 1; j >= 0 && steps > 0; --j) {
        int64_t t0 = j * ckpt_every;
        int64_t len = steps - t0 < ckpt_every ? steps - t0 : ckpt_every;
        /* recompute u_{t0} .. u_{t0+len-1} */
        memcpy(seg, ckpt + j * N, sizeof(double) * (size_t)N);
        for (int64_t m = 1; m < len; ++m) step_varcoef(&g, faces, seg + (m - 1) * N, seg + m * N);
        for (int64_t m = len - 1; m >= 0; --m) {
            const double* ut = seg + m * N;     /* u_t, t = t0 + m */
            const double* lam = grad_u0;        /* lambda_{t+1} */
            /* dL/dc_f[p] += lambda_{t+1}[p] (u_t[p+e_f] - u_t[p]) */
#pragma omp parallel for schedule(static)
            for (int64_t i0 = 0; i0 < g.n[0]; ++i0) {
                for (int64_t rem = 0; rem < plane; ++rem) {
                    int64_t p = i0 * plane + rem;
                    int64_t cp[3];
                    coords(&g, p, cp);
                    if (!is_interior(&g, cp, 1)) continue;
                    for (int f = 0; f < nf; ++f)
                        grad_faces[(int64_t)f * N + p] += lam[p] * (ut[p + fst[f]] - ut[p]);
                }
            }
            /* lambda_t = A^T lambda_{t+1} */
            step_varcoef_T(&g, faces, grad_u0, nxt);
            memcpy(grad_u0, nxt, sizeof(double) * (size_t)N);
        }
    }
    free(ckpt); free(seg); free(cur); free(nxt);
    return 0;
}

/* 1/2 ||u - target||^2 */
double oracle_loss(int64_t n, const double* u, const double* target) {
    double L = 0.0;
    for (int64_t i = 0; i < n; ++i) { double d = u[i] - target[i]; L += d * d; }
    return 0.5 * L;
}
