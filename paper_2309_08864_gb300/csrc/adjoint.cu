// adjoint.cu -- differentiation form of the out-of-core sweep.
//
// For u_{t+1} = A u_t (the variable-coefficient 7-point stencil, centre weight
// 1 - sum of the six face weights) and L = 1/2 ||u_T - u*||^2:
//   lambda_T = u_T - u*,  lambda_t = A^T lambda_{t+1},  dL/du_0 = lambda_0,
//   (A^T l)[q] = [q not in I] l[q] + [q in I] c_c[q] l[q]
//                + sum_f [q - e_f in I] c_f[q - e_f] l[q - e_f],
//   dL/dc_f[p] = sum_t lambda_{t+1}[p] (u_t[p + e_f] - u_t[p]),  p in I.
// Everything runs through the same chunked pipeline as the forward sweep
// (Algorithm 1: chunks along axis 0, region sharing through circular device
// buffers, bounded by the plan's device budget):
//   1. forward rounds of C = checkpoint_every steps keep u_{jC} in host memory;
//   2. a loss pass forms lambda_T and reduces L in FP64 on the device;
//   3. per segment, last first: single-step rounds recompute the segment's
//      states into host memory, then single-step adjoint rounds run the
//      transposed stencil backward in time, updating lambda in place and
//      accumulating dL/dc_f on the cells each chunk owns (the overlap is
//      computed by both neighbours, so accumulating it twice would be wrong).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "kernels.hpp"
#include "run.hpp"

using namespace so2dr;

namespace so2dr {

constexpr int kPartialBlocks = 256;  // FP64 partial sums per chunk (fixed: deterministic order)

// ------------------------------------------------------------------ kernels

struct PlaneRef {  // planes of a (possibly circular) arena buffer
    const void* base;
    int64_t cap, slot0, lo;  // plane z sits in slot (slot0 + z - lo) % cap
    int64_t field_stride;    // elements between fields
    __device__ __forceinline__ int64_t off(int64_t z, int64_t plane) const {
        return ((slot0 + (z - lo)) % cap) * plane;
    }
};

struct AdjStepArgs {
    PlaneRef lam, coef, u, grad;  // lambda_{t+1}, faces, u_t (radius-1 halo); gradient slab
    void* lam_out;                // lambda_t on planes [s, e), slot z - s
    int64_t s, e;                 // planes of lambda_t this launch computes
    int64_t gs, ge;               // owned planes: the gradient accumulates here only
    int64_t n0, ny, nx;
    int first;                    // start the gradient from zero
};

__device__ __forceinline__ bool interior3(int64_t z, int64_t y, int64_t x, int64_t n0, int64_t ny, int64_t nx) {
    return z >= 1 && z < n0 - 1 && y >= 1 && y < ny - 1 && x >= 1 && x < nx - 1;
}

template <typename T>
__global__ void __launch_bounds__(256) adjoint_step_kernel(const AdjStepArgs a) {
    const int64_t plane = a.ny * a.nx;
    const int64_t n = (a.e - a.s) * plane;
    const T* lam = static_cast<const T*>(a.lam.base);
    const T* cf = static_cast<const T*>(a.coef.base);
    const T* u = static_cast<const T*>(a.u.base);
    T* g = static_cast<T*>(const_cast<void*>(a.grad.base));
    T* lo = static_cast<T*>(a.lam_out);
    const int64_t dz[6] = {-1, 1, 0, 0, 0, 0}, dy[6] = {0, 0, -1, 1, 0, 0}, dx[6] = {0, 0, 0, 0, -1, 1};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t z = a.s + i / plane, rem = i % plane, y = rem / a.nx, x = rem % a.nx;
        const int64_t c = y * a.nx + x;
        const int64_t lz = a.lam.off(z, plane), cz = a.coef.off(z, plane), uz = a.u.off(z, plane);
        const bool qi = interior3(z, y, x, a.n0, a.ny, a.nx);
        const T lq = lam[lz + c];
        T acc;
        if (qi) {
            T csum = cf[cz + c] + cf[a.coef.field_stride + cz + c];
            for (int f = 2; f < 6; ++f) csum = csum + cf[f * a.coef.field_stride + cz + c];
            acc = ((T)1 - csum) * lq;
        } else {
            acc = lq;
        }
        // neighbour p = q - e_f weighs u[q] with c_f[p]
        for (int f = 0; f < 6; ++f) {
            const int64_t pz = z - dz[f], py = y - dy[f], px = x - dx[f];
            if (!interior3(pz, py, px, a.n0, a.ny, a.nx)) continue;
            const int64_t pc = py * a.nx + px;
            acc = fma_c(cf[f * a.coef.field_stride + a.coef.off(pz, plane) + pc], lam[a.lam.off(pz, plane) + pc], acc);
        }
        lo[(z - a.s) * plane + c] = acc;
        // dL/dc_f[q] += lambda_{t+1}[q] (u_t[q + e_f] - u_t[q]) on the owned cells
        if (z < a.gs || z >= a.ge) continue;
        const int64_t gs = (z - a.gs) * plane + c;
        const T uq = u[uz + c];
        for (int f = 0; f < 6; ++f) {
            T gv = a.first ? (T)0 : g[f * a.grad.field_stride + gs];
            if (qi) {
                const int64_t nz = z + dz[f], nc = (y + dy[f]) * a.nx + (x + dx[f]);
                gv = fma_c(lq, u[a.u.off(nz, plane) + nc] - uq, gv);
            }
            g[f * a.grad.field_stride + gs] = gv;
        }
    }
}

// Block sum in a fixed order (deterministic): shuffles within warps, then warps.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
    return r;
}

// lambda = u - target on owned planes; FP64 partial sums of (u - target)^2,
// the difference formed in FP64
template <typename T>
__global__ void __launch_bounds__(256) residual_kernel(const T* u, const T* tg, T* lam, int64_t n, double* partial) {
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        // lambda_T in the storage precision; the loss from the FP64 difference
        if (lam) lam[i] = u[i] - tg[i];
        const double d = (double)u[i] - (double)tg[i];
        acc = fma(d, d, acc);
    }
    double b = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = b;
}

// FP64 partial inner products
template <typename T>
__global__ void __launch_bounds__(256) dot_kernel(const T* x, const T* y, int64_t n, double* partial) {
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc = fma((double)x[i], (double)y[i], acc);
    double b = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = b;
}

// out[0] = (accumulate ? out[0] : 0) + scale * sum of partial[0..n), fixed order
__global__ void __launch_bounds__(256) reduce_kernel(const double* partial, int64_t n, double scale, double* out,
                                                     int accumulate) {
    double acc = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
    double b = block_sum(acc);
    if (threadIdx.x == 0) out[0] = (accumulate ? out[0] : 0.0) + scale * b;
}

// ------------------------------------------------------------------ op lists

namespace {

enum AdjHost : int { kHU0 = 0, kHCoef = 1, kHTarget = 2, kHLam = 3, kHGrad = 4, kHWork = 5 };

// Buffers of the loss / dot pass: U, TG, LAM (x2 by chunk parity), partials, result.
enum { kLU0 = 0, kLT0 = 2, kLL0 = 4, kLPart = 6, kLRes = 7 };

size_t place(std::vector<Buffer>& b, int id, int64_t cap, int64_t pb, int nf, int64_t& off) {
    if ((int)b.size() <= id) b.resize(id + 1);
    b[id].offset = off;
    b[id].cap = cap;
    b[id].plane_bytes = pb;
    b[id].nfields = nf;
    off += align_up(cap * pb);
    return (size_t)off;
}

// Loss pass over chunks of `q`: lambda = u - target (written to host array
// lam_arr unless it is negative) and L = 1/2 sum lambda^2 into the result slot.
bool build_loss_list(const Plan& q, RunList& rl, size_t budget, int u_arr, int lam_arr) {
    rl.ops.clear();
    rl.bufs.clear();
    int64_t pmax = 0;
    for (int i = 0; i < q.d; ++i) pmax = std::max(pmax, q.starts[i + 1] - q.starts[i]);
    int64_t off = 0;
    for (int k = 0; k < 2; ++k) {
        place(rl.bufs, kLU0 + k, pmax, q.plane_bytes, 1, off);
        place(rl.bufs, kLT0 + k, pmax, q.plane_bytes, 1, off);
        place(rl.bufs, kLL0 + k, lam_arr >= 0 ? pmax : 0, q.plane_bytes, 1, off);
    }
    place(rl.bufs, kLPart, 1, (int64_t)q.d * kPartialBlocks * 8, 1, off);
    place(rl.bufs, kLRes, 1, 8, 1, off);
    off += kAlign;
    rl.arena_bytes = (size_t)off;
    if (budget && rl.arena_bytes > budget) return false;
    const int nbuf = (int)rl.bufs.size();
    Emitter em(rl, nbuf + std::max<int>(kHWork, std::max(u_arr, lam_arr)) + 1, nbuf);
    for (int i = 0; i < q.d; ++i) {
        const int64_t s = q.starts[i], e = q.starts[i + 1];
        const int k = i % 2;
        for (int f = 0; f < 2; ++f) {
            Op op = make_op(kOpH2D, kStreamH2D, 0, i);
            op.host_array = f ? kHTarget : u_arr;
            op.pub.src_lo = op.pub.dst_lo = s;
            op.pub.src_hi = op.pub.dst_hi = e;
            op.pub.src_slot0 = s;
            op.pub.dst_buf = (f ? kLT0 : kLU0) + k;
            op.pub.dst_slot0 = 0;
            em.tr.access(em.host_res(op.host_array), s, e, false);
            em.tr.access(op.pub.dst_buf, 0, e - s, true);
            em.emit(op);
        }
        Op op = make_op(kOpKernel, kStreamCompute, 0, i);
        op.fn = kFnResidual;
        op.pub.src_buf = kLU0 + k;
        op.pub.src_lo = s;
        op.pub.src_hi = e;
        op.aux_buf = kLT0 + k;
        op.pub.dst_buf = lam_arr >= 0 ? kLL0 + k : -1;
        op.pub.dst_lo = s;
        op.pub.dst_hi = e;
        op.arg0 = (int64_t)i * kPartialBlocks;
        em.tr.access(kLU0 + k, 0, e - s, false);
        em.tr.access(kLT0 + k, 0, e - s, false);
        if (lam_arr >= 0) em.tr.access(kLL0 + k, 0, e - s, true);
        em.tr.access(kLPart, i, i + 1, true);
        em.emit(op);
        if (lam_arr >= 0) {
            Op d = make_op(kOpD2H, kStreamD2H, 0, i);
            d.host_array = lam_arr;
            d.pub.src_buf = kLL0 + k;
            d.pub.src_lo = d.pub.dst_lo = s;
            d.pub.src_hi = d.pub.dst_hi = e;
            d.pub.src_slot0 = 0;
            d.pub.dst_slot0 = s;
            em.tr.access(kLL0 + k, 0, e - s, false);
            em.tr.access(em.host_res(lam_arr), s, e, true);
            em.emit(d);
        }
    }
    Op r = make_op(kOpKernel, kStreamCompute, 0, 0);
    r.fn = kFnReduce;
    r.arg0 = (int64_t)q.d * kPartialBlocks;
    r.arg1 = 0;   // scale 1/2, no accumulation
    r.aux_lo = 0;
    em.tr.access(kLPart, 0, q.d, false);
    em.tr.access(kLRes, 0, 1, true);
    em.emit(r);
    return true;
}

// Buffers of the adjoint rounds: circular region-shared inputs (lambda, the
// face fields, the K states u_t), gradient and final-lambda slabs by chunk
// parity, and two slabs for the intermediate lambdas of a round.
enum { kALam = 0, kACoef = 1, kAG0 = 2, kAL0 = 4, kAX = 6, kAY = 7, kAU0 = 8 };

// Capacity of the circular input buffers for rounds of K steps: a chunk's
// inputs [s - K, e + K) and the next chunk's new planes, so that transfers
// run one chunk ahead of the kernels.
int64_t adjoint_cin(const Plan& q, int K) {
    int64_t cin = 0;
    for (int i = 0; i < q.d; ++i) {
        ChunkGeom g = chunk_geom(q, i, K);
        int64_t next_hi = (i + 1 < q.d) ? chunk_geom(q, i + 1, K).hi : q.n0 + chunk_geom(q, 0, K).hi;
        cin = std::max(cin, std::max(g.b - g.a, next_hi - g.a));
    }
    return std::max<int64_t>(cin, 1);
}

size_t adjoint_layout(const Plan& q, int K, std::vector<Buffer>* out) {
    std::vector<Buffer> b;
    int64_t pmax = 0;
    for (int i = 0; i < q.d; ++i) pmax = std::max(pmax, q.starts[i + 1] - q.starts[i]);
    int64_t cin = adjoint_cin(q, K), off = 0;
    place(b, kALam, cin, q.plane_bytes, 1, off);
    place(b, kACoef, cin, 6 * q.plane_bytes, 6, off);
    for (int k = 0; k < 2; ++k) place(b, kAG0 + k, pmax, 6 * q.plane_bytes, 6, off);
    for (int k = 0; k < 2; ++k) place(b, kAL0 + k, pmax, q.plane_bytes, 1, off);
    place(b, kAX, K >= 2 ? pmax + 2 * K : 0, q.plane_bytes, 1, off);
    place(b, kAY, K >= 3 ? pmax + 2 * K : 0, q.plane_bytes, 1, off);
    for (int k = 0; k < K; ++k) place(b, kAU0 + k, cin, q.plane_bytes, 1, off);
    off += kAlign;
    if (out) *out = b;
    return (size_t)off;
}

// Adjoint rounds for times t_hi-1 down to t_lo, K steps per round (the last
// round of the span may be shorter).  A round reads lambda_{t+1} at its top
// time, the face fields and its K states u_t, with a K-plane halo through the
// circular buffers (each plane crosses the link once per round), runs K
// single-step launches of the transposed stencil on the shrinking trapezoid,
// accumulates dL/dc_f of all K steps on the chunk's owned planes in a device
// slab, and sends lambda and the gradient back once.  state_arr(t) is the
// host array holding u_t.
template <typename F>
void build_adjoint_list(const Plan& q, RunList& rl, int64_t t_lo, int64_t t_hi, int64_t T, int K, int nhost,
                        F state_arr) {
    rl.ops.clear();
    rl.arena_bytes = adjoint_layout(q, K, &rl.bufs);
    const int nbuf = (int)rl.bufs.size();
    Emitter em(rl, nbuf + nhost, nbuf);
    const int64_t cin = rl.bufs[kALam].cap;
    int64_t g = 0;
    int rho = 0;
    for (int64_t top = t_hi; top > t_lo; top -= K, ++rho) {
        const int kk = (int)std::min<int64_t>(K, top - t_lo);
        const int64_t V = (int64_t)rho * q.n0;
        for (int i = 0; i < q.d; ++i, ++g) {
            ChunkGeom cg = chunk_geom(q, i, kk);
            const int k = (int)(g % 2);
            // region-shared inputs: lambda_{top}, the face fields, u_{top-1} .. u_{top-kk}
            if (cg.hi > cg.lo) {
                for (int f = 0; f < 2 + kk; ++f) {
                    const int buf = f == 0 ? kALam : f == 1 ? kACoef : kAU0 + (f - 2);
                    const int arr = f == 0 ? kHLam : f == 1 ? kHCoef : state_arr(top - 1 - (f - 2));
                    Op op = make_op(kOpH2D, kStreamH2D, rho, i);
                    op.host_array = arr;
                    op.nfields = f == 1 ? 6 : 1;
                    op.pub.src_lo = op.pub.dst_lo = cg.lo;
                    op.pub.src_hi = op.pub.dst_hi = cg.hi;
                    op.pub.src_slot0 = cg.lo;
                    op.pub.dst_buf = buf;
                    op.pub.dst_slot0 = floor_mod(V + cg.lo, cin);
                    em.tr.access(em.host_res(arr), cg.lo, cg.hi, false);
                    add_buf_access(em.tr, buf, cg.lo, cg.hi, op.pub.dst_slot0, cin, true);
                    em.emit(op);
                }
            }
            // the gradient accumulated so far on the owned planes
            if (top != T) {
                Op op = make_op(kOpH2D, kStreamH2D, rho, i);
                op.host_array = kHGrad;
                op.nfields = 6;
                op.pub.src_lo = op.pub.dst_lo = cg.s;
                op.pub.src_hi = op.pub.dst_hi = cg.e;
                op.pub.src_slot0 = cg.s;
                op.pub.dst_buf = kAG0 + k;
                op.pub.dst_slot0 = 0;
                em.tr.access(em.host_res(kHGrad), cg.s, cg.e, false);
                em.tr.access(kAG0 + k, 0, cg.e - cg.s, true);
                em.emit(op);
            }
            // kk launches: lambda_{top-1-m} on [s - (kk-1-m), e + (kk-1-m))
            int src = kALam;
            int64_t in_lo = cg.a, in_hi = cg.b, src_slot0 = floor_mod(V + cg.a, cin), scap = cin;
            const int stream = (g % 2) ? kStreamCompute2 : kStreamCompute;
            for (int m = 0; m < kk; ++m) {
                const bool last = m + 1 == kk;
                const int64_t h = kk - 1 - m;
                const int64_t lo = std::max<int64_t>(0, cg.s - h), hi = std::min<int64_t>(q.n0, cg.e + h);
                const int dst = last ? kAL0 + k : ((m % 2 == 0) ? kAX : kAY);
                Op op = make_op(kOpKernel, stream, rho, i);
                op.fn = kFnAdjoint;
                op.pub.depth = 1;
                op.pub.src_buf = src;
                op.pub.src_lo = in_lo;
                op.pub.src_hi = in_hi;
                op.pub.src_slot0 = src_slot0;
                op.aux_buf = kACoef;
                op.aux_lo = cg.a;
                op.aux_slot0 = floor_mod(V + cg.a, cin);
                op.aux2_buf = kAU0 + m;
                op.aux2_lo = cg.a;
                op.aux2_slot0 = floor_mod(V + cg.a, cin);
                op.aux3_buf = kAG0 + k;
                op.aux3_lo = cg.s;
                op.aux3_slot0 = 0;
                op.arg2 = cg.e;
                op.pub.dst_buf = dst;
                op.pub.dst_lo = lo;
                op.pub.dst_hi = hi;
                op.arg1 = (top == T && m == 0);
                add_buf_access(em.tr, src, in_lo, in_hi, src_slot0, scap, false);
                add_buf_access(em.tr, kACoef, cg.a, cg.b, op.aux_slot0, cin, false);
                add_buf_access(em.tr, kAU0 + m, cg.a, cg.b, op.aux2_slot0, cin, false);
                em.tr.access(kAG0 + k, 0, cg.e - cg.s, true);
                em.tr.access(dst, 0, hi - lo, true);
                em.emit(op);
                src = dst;
                in_lo = lo;
                in_hi = hi;
                src_slot0 = 0;
                scap = rl.bufs[dst].cap;
            }
            // lambda_{top-kk} and the gradient back to the host (every owned
            // plane: the adjoint also changes the boundary cells of lambda)
            for (int f = 0; f < 2; ++f) {
                Op d = make_op(kOpD2H, kStreamD2H, rho, i);
                d.host_array = f ? kHGrad : kHLam;
                d.nfields = f ? 6 : 1;
                d.pub.src_buf = (f ? kAG0 : kAL0) + k;
                d.pub.src_lo = d.pub.dst_lo = cg.s;
                d.pub.src_hi = d.pub.dst_hi = cg.e;
                d.pub.src_slot0 = 0;
                d.pub.dst_slot0 = cg.s;
                em.tr.access(d.pub.src_buf, 0, cg.e - cg.s, false);
                em.tr.access(em.host_res(d.host_array), cg.s, cg.e, true);
                em.emit(d);
            }
        }
    }
}

// Smallest d >= dmin for which `arena(q)` fits `limit`.
template <typename F>
int fit_d(Plan& q, int dmin, size_t limit, F arena) {
    int64_t M = q.n0 - 2 * q.r;
    int dmax = (int)std::max<int64_t>(1, M);
    auto fits = [&](int d) {
        q.d = d;
        partition_planes(q);
        return arena(q) <= limit;
    };
    int lo = std::max(1, std::min(dmin, dmax));
    if (!fits(dmax)) return 0;
    if (fits(lo)) return lo;
    int a = lo, b = dmax;
    while (b - a > 1) {
        int m = a + (b - a) / 2;
        if (fits(m)) b = m; else a = m;
    }
    fits(b);
    return b;
}

}  // namespace

size_t adjoint_arena_bytes(const Plan& q) { return adjoint_layout(q, 1, nullptr); }

size_t adjoint_workspace_bytes(const Plan& p) {
    if (p.kind != SO2DR_VARCOEF_STAR) return (size_t)(p.n0 * p.plane_bytes);
    int64_t C = std::max(1, p.k_off), S = std::max<int64_t>(1, (p.T + C - 1) / C);
    return (size_t)((S + C - 1) * p.n0 * p.plane_bytes);
}

// ------------------------------------------------------------------ launch hook

int enqueue_aux_kernel(so2dr_plan_s* P, const RunList& rl, const Op& op, cudaStream_t s) {
    const Plan& p = P->p;
    const bool f64 = p.dtype == SO2DR_F64;
    const int64_t plane = p.plane_cells;
    auto buf = [&](int id) { return P->arena + rl.bufs[id].offset; };
    const int nblk = 4 * std::max(1, P->sm_count);
    cudaError_t e = cudaSuccess;
    if (op.fn == kFnStencil) return enqueue_stencil(P, rl, op, s);
    if (op.fn == kFnAdjoint) {
        AdjStepArgs a;
        std::memset(&a, 0, sizeof(a));
        auto ref = [&](int id, int64_t lo, int64_t slot0) {
            PlaneRef r;
            r.base = buf(id);
            r.cap = rl.bufs[id].cap;
            r.slot0 = slot0 % r.cap;
            r.lo = lo;
            r.field_stride = r.cap * plane;
            return r;
        };
        const so2dr_op_t& o = op.pub;
        a.lam = ref(o.src_buf, o.src_lo, o.src_slot0);
        a.coef = ref(op.aux_buf, op.aux_lo, op.aux_slot0);
        a.u = ref(op.aux2_buf, op.aux2_lo, op.aux2_slot0);
        a.grad = ref(op.aux3_buf, op.aux3_lo, op.aux3_slot0);
        a.lam_out = buf(o.dst_buf);
        a.s = o.dst_lo;
        a.e = o.dst_hi;
        a.gs = op.aux3_lo;
        a.ge = op.arg2;
        a.n0 = p.n0;
        a.ny = p.ny;
        a.nx = p.nx;
        a.first = (int)op.arg1;
        if (f64) adjoint_step_kernel<double><<<nblk, 256, 0, s>>>(a);
        else adjoint_step_kernel<float><<<nblk, 256, 0, s>>>(a);
    } else if (op.fn == kFnResidual) {
        const so2dr_op_t& o = op.pub;
        int64_t n = (o.src_hi - o.src_lo) * plane;
        double* part = reinterpret_cast<double*>(buf(kLPart)) + op.arg0;
        void* lam = o.dst_buf >= 0 ? buf(o.dst_buf) : nullptr;
        if (f64)
            residual_kernel<double><<<kPartialBlocks, 256, 0, s>>>((const double*)buf(o.src_buf),
                                                                   (const double*)buf(op.aux_buf), (double*)lam, n, part);
        else
            residual_kernel<float><<<kPartialBlocks, 256, 0, s>>>((const float*)buf(o.src_buf),
                                                                  (const float*)buf(op.aux_buf), (float*)lam, n, part);
    } else if (op.fn == kFnDot) {
        const so2dr_op_t& o = op.pub;
        int64_t n = op.arg1;
        double* part = reinterpret_cast<double*>(buf(kLPart)) + op.arg0;
        if (f64 || o.depth == 8)
            dot_kernel<double><<<kPartialBlocks, 256, 0, s>>>((const double*)buf(o.src_buf),
                                                              (const double*)buf(op.aux_buf), n, part);
        else
            dot_kernel<float><<<kPartialBlocks, 256, 0, s>>>((const float*)buf(o.src_buf),
                                                             (const float*)buf(op.aux_buf), n, part);
    } else if (op.fn == kFnReduce) {
        // arg0: partials to sum; arg1 bit 0: scale 1 (else 1/2); bit 1: accumulate;
        // aux_lo: first partial
        reduce_kernel<<<1, 256, 0, s>>>(reinterpret_cast<const double*>(buf(kLPart)) + op.aux_lo, op.arg0,
                                        (op.arg1 & 1) ? 1.0 : 0.5, reinterpret_cast<double*>(buf(kLRes)),
                                        (int)((op.arg1 >> 1) & 1));
    } else {
        return set_error(SO2DR_E_INVAL, "unknown kernel program");
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? SO2DR_OK : cuda_fail(e, "auxiliary kernel launch");
}

// Reads the FP64 result slot of a loss/dot list.
int read_result(so2dr_plan_s* P, const RunList& rl, double* out) {
    cudaError_t e = cudaMemcpy(out, P->arena + rl.bufs[kLRes].offset, sizeof(double), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? SO2DR_OK : cuda_fail(e, "reading the FP64 result");
}

}  // namespace so2dr

namespace {

// Host-array table shared by the pipelines of one adjoint/loss call.
struct HostTable {
    std::vector<char*> base;
    std::vector<int64_t> plane_bytes, field_bytes;
    void set(int i, const void* p, int64_t pb, int64_t fb) {
        if ((int)base.size() <= i) {
            base.resize(i + 1, nullptr);
            plane_bytes.resize(i + 1, 0);
            field_bytes.resize(i + 1, 0);
        }
        base[i] = static_cast<char*>(const_cast<void*>(p));
        plane_bytes[i] = pb;
        field_bytes[i] = fb;
    }
};

void add_stats(so2dr_stats_t* acc, const so2dr_stats_t& s) {
    if (!acc) return;
    acc->total_ms += s.total_ms;
    acc->kernel_ms += s.kernel_ms;
    acc->h2d_ms += s.h2d_ms;
    acc->d2h_ms += s.d2h_ms;
    acc->h2d_bytes += s.h2d_bytes;
    acc->d2h_bytes += s.d2h_bytes;
    acc->launches += s.launches;
    acc->ops += s.ops;
}

int run_list(so2dr_plan_s* P, const RunList& rl, const HostTable& h, so2dr_stats_t* acc) {
    so2dr_stats_t st;
    std::memset(&st, 0, sizeof(st));
    int rc = execute(P, rl, h.base.data(), h.plane_bytes.data(), h.field_bytes.data(), acc ? &st : nullptr,
                     enqueue_aux_kernel);
    if (rc) return rc;
    add_stats(acc, st);
    return SO2DR_OK;
}

// Forward pipeline of `steps` steps from host array src to host array dst
// (then in place on dst), rounds of k steps, fitted into `limit` arena bytes.
int forward_pipeline(so2dr_plan_s* P, int64_t steps, int k, int src, int dst, const HostTable& h, size_t limit,
                     so2dr_stats_t* acc) {
    if (steps <= 0) return SO2DR_OK;
    Plan q = P->p;
    q.T = steps;
    q.k_off = k;
    q.k_on = std::min(k, std::min(P->p.k_on, q.max_kon));
    q.rounds = (int)((steps + k - 1) / k);
    if (!fit_d(q, 1, limit, [](const Plan& x) { return forward_arena_bytes(x); }))
        return set_error(SO2DR_E_INFEASIBLE, "forward rounds do not fit the bound arena");
    ForwardOpts o;
    o.all_planes = true;
    o.coef_array = kHCoef;
    for (int t = 0; t < q.rounds; ++t) {
        o.src_array.push_back(t == 0 ? src : dst);
        o.dst_array.push_back(dst);
    }
    RunList rl;
    if (!build_forward_ooc_ex(q, rl, limit, o)) return set_error(SO2DR_E_INFEASIBLE, "forward rounds do not fit");
    Plan saved = P->p;
    P->p = q;  // the executor reads the chunking and k_on of the running list from the plan
    int rc = run_list(P, rl, h, acc);
    P->p = saved;
    return rc;
}

}  // namespace

extern "C" {

int so2dr_loss(so2dr_plan_t P, const void* host_u0, const void* host_coeff_fields, const void* host_target,
               void* host_workspace, size_t workspace_bytes, double* loss_out) {
    if (!P || !loss_out) return set_error(SO2DR_E_INVAL, "NULL argument");
    const Plan& p = P->p;
    if (!P->arena || P->device < 0) return set_error(SO2DR_E_NOT_BOUND, "plan is not bound (so2dr_bind)");
    if (p.kind != SO2DR_VARCOEF_STAR) return set_error(SO2DR_E_UNSUPPORTED, "so2dr_loss needs a VARCOEF_STAR plan");
    size_t need = (size_t)(p.n0 * p.plane_bytes);
    if (workspace_bytes < need) return set_error(SO2DR_E_INVAL, "workspace smaller than one grid");
    int rc;
    for (const void* q : {host_u0, host_coeff_fields, host_target, (const void*)host_workspace})
        if ((rc = check_pinned(q, "host buffer"))) return rc;
    HostTable h;
    const int64_t cb = p.dtype == SO2DR_F64 ? 8 : 4;
    h.set(kHU0, host_u0, p.plane_bytes, 0);
    h.set(kHCoef, host_coeff_fields, p.plane_cells * cb, p.n0 * p.plane_cells * cb);
    h.set(kHTarget, host_target, p.plane_bytes, 0);
    h.set(kHWork, host_workspace, p.plane_bytes, 0);
    const size_t limit = P->arena_bytes;
    if (p.T > 0) {
        rc = forward_pipeline(P, p.T, p.k_off, kHU0, kHWork, h, limit, nullptr);
        if (rc) return rc;
    }
    Plan q = p;
    if (!fit_d(q, 1, limit, [](const Plan& x) {
            RunList r;
            build_loss_list(x, r, 0, kHU0, -1);
            return r.arena_bytes;
        }))
        return set_error(SO2DR_E_INFEASIBLE, "loss pass does not fit the bound arena");
    RunList rl;
    build_loss_list(q, rl, limit, p.T > 0 ? kHWork : kHU0, -1);
    Plan saved = P->p;
    P->p = q;
    rc = run_list(P, rl, h, nullptr);
    P->p = saved;
    if (rc) return rc;
    return read_result(P, rl, loss_out);
}

int so2dr_adjoint(so2dr_plan_t P, const void* host_u0, const void* host_coeff_fields, const void* host_target,
                  void* host_grad_u0, void* host_grad_coeffs, void* host_workspace, size_t workspace_bytes,
                  int checkpoint_every, double* loss_out, so2dr_stats_t* stats) {
    if (!P || !loss_out) return set_error(SO2DR_E_INVAL, "NULL argument");
    const Plan& p = P->p;
    if (!P->arena || P->device < 0) return set_error(SO2DR_E_NOT_BOUND, "plan is not bound (so2dr_bind)");
    if (p.kind != SO2DR_VARCOEF_STAR) return set_error(SO2DR_E_UNSUPPORTED, "so2dr_adjoint needs a VARCOEF_STAR plan");
    if (checkpoint_every < 1) return set_error(SO2DR_E_INVAL, "checkpoint_every must be >= 1");
    const int64_t T = p.T, C = checkpoint_every, S = std::max<int64_t>(1, (T + C - 1) / C);
    const int64_t grid = p.n0 * p.plane_bytes;
    const size_t need = (size_t)((S + C - 1) * grid);
    if (workspace_bytes < need) return set_error(SO2DR_E_INVAL, "workspace smaller than (segments + C - 1) grids");
    int rc;
    for (const void* q : {host_u0, host_coeff_fields, host_target, (const void*)host_grad_u0,
                          (const void*)host_grad_coeffs, (const void*)host_workspace})
        if ((rc = check_pinned(q, "host buffer"))) return rc;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    HostTable h;
    const int64_t cb = p.dtype == SO2DR_F64 ? 8 : 4;
    h.set(kHU0, host_u0, p.plane_bytes, 0);
    h.set(kHCoef, host_coeff_fields, p.plane_cells * cb, p.n0 * p.plane_cells * cb);
    h.set(kHTarget, host_target, p.plane_bytes, 0);
    h.set(kHLam, host_grad_u0, p.plane_bytes, 0);
    h.set(kHGrad, host_grad_coeffs, p.plane_cells * cb, p.n0 * p.plane_cells * cb);
    // workspace: checkpoints u_{C}, ..., u_{(S-1)C}, u_T, then segment states 1..C-1
    char* ws = static_cast<char*>(host_workspace);
    for (int64_t j = 0; j < S + C - 1; ++j) h.set((int)(kHWork + j), ws + j * grid, p.plane_bytes, 0);
    auto ckpt_arr = [&](int64_t j) { return j == 0 ? (int)kHU0 : (int)(kHWork + j - 1); };  // u_{jC}; j = S: u_T
    auto seg_arr = [&](int64_t m) { return (int)(kHWork + S + m - 1); };                    // u_{t0+m}, m >= 1
    const size_t limit = P->arena_bytes;
    auto t0 = std::chrono::steady_clock::now();

    // 1. forward sweep keeping u at every multiple of C, and u_T
    for (int64_t j = 0; j < S; ++j) {
        int64_t len = std::min(C, T - j * C);
        if (len <= 0) break;
        rc = forward_pipeline(P, len, (int)len, ckpt_arr(j), ckpt_arr(j + 1), h, limit, stats);
        if (rc) return rc;
    }
    const int uT = T > 0 ? ckpt_arr(S) : (int)kHU0;
    // 2. lambda_T = u_T - u*, L = 1/2 ||lambda_T||^2
    {
        Plan q = p;
        if (!fit_d(q, 1, limit, [](const Plan& x) {
                RunList r;
                build_loss_list(x, r, 0, kHU0, kHLam);
                return r.arena_bytes;
            }))
            return set_error(SO2DR_E_INFEASIBLE, "loss pass does not fit the bound arena");
        RunList rl;
        build_loss_list(q, rl, limit, uT, kHLam);
        Plan saved = P->p;
        P->p = q;
        rc = run_list(P, rl, h, stats);
        P->p = saved;
        if (rc) return rc;
        if ((rc = read_result(P, rl, loss_out))) return rc;
    }
    if (T == 0) {
        // no step: dL/du_0 = lambda_T (written above) and dL/dc = 0
        std::memset(host_grad_coeffs, 0, (size_t)(6 * p.n0 * p.plane_cells * cb));
        return SO2DR_OK;
    }
    // 3. segments, last first: recompute states, then adjoint rounds.  The
    // rounds take K steps (K <= C) where the budget admits it: per round the
    // face fields and lambda cross the link once and the gradient once each
    // way, so K steps per round divide that traffic by K; the cost below
    // weighs those bytes against the per-chunk copy and launch overhead of the
    // smaller chunks a larger K forces.
    int K = 0;
    Plan qa = p;
    {
        // SO2DR_ADJOINT_STEPS pins K (or the largest K below it that fits)
        const char* ek = std::getenv("SO2DR_ADJOINT_STEPS");
        const int kpin = ek ? (int)std::min<int64_t>(std::max(1, std::atoi(ek)), C) : 0;
        double best = 0;
        for (int k = 1; k <= (int)std::min<int64_t>(C, 16); ++k) {
            if (kpin > 0 && k > kpin) continue;
            Plan q = p;
            if (!fit_d(q, 1, limit, [k](const Plan& x) { return adjoint_layout(x, k, nullptr); })) continue;
            const double grid_b = (double)p.n0 * p.plane_bytes;
            const double link_s = grid_b * (14.0 + k) / 170e9;           // inputs of one round
            const double ops_s = (double)q.d * (24.0 + 2.0 * k) * 4e-6;  // copies and launches
            const double cost = kpin > 0 ? -k : (link_s + ops_s) * std::ceil((double)C / k);
            if (K == 0 || cost < best) {
                K = k;
                best = cost;
                qa = q;
            }
        }
    }
    if (!K) return set_error(SO2DR_E_INFEASIBLE, "adjoint rounds do not fit the bound arena");
    for (int64_t j = S - 1; j >= 0; --j) {
        const int64_t ts = j * C, len = std::min(C, T - ts);
        // u_{ts+m}, m = 1..len-1, into the segment states: one round of
        // single-step launches that sends every intermediate state back, or,
        // where that round does not fit, one round per step
        if (len >= 2) {
            ForwardOpts o;
            o.all_planes = true;
            o.coef_array = kHCoef;
            o.src_array.push_back(ckpt_arr(j));
            o.dst_array.push_back(seg_arr(len - 1));
            for (int64_t m = 1; m + 1 < len; ++m) o.state_array.push_back(seg_arr(m));
            Plan q = p;
            q.T = len - 1;
            q.k_off = (int)(len - 1);
            q.k_on = 1;
            q.rounds = 1;
            RunList rl;
            if (fit_d(q, 1, limit, [](const Plan& x) { return forward_arena_bytes(x); }) &&
                build_forward_ooc_ex(q, rl, limit, o)) {
                Plan saved = P->p;
                P->p = q;
                rc = run_list(P, rl, h, stats);
                P->p = saved;
                if (rc) return rc;
            } else {
                for (int64_t m = 1; m < len; ++m) {
                    rc = forward_pipeline(P, 1, 1, m == 1 ? ckpt_arr(j) : seg_arr(m - 1), seg_arr(m), h, limit,
                                          stats);
                    if (rc) return rc;
                }
            }
        }
        RunList rl;
        build_adjoint_list(qa, rl, ts, ts + len, T, K, (int)h.base.size(),
                           [&](int64_t t) { return t == ts ? ckpt_arr(j) : seg_arr(t - ts); });
        if (rl.arena_bytes > limit) return set_error(SO2DR_E_INFEASIBLE, "adjoint rounds do not fit");
        Plan saved = P->p;
        P->p = qa;
        rc = run_list(P, rl, h, stats);
        P->p = saved;
        if (rc) return rc;
    }
    if (stats) {
        stats->total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        // forward + adjoint cell updates per second (interior cells x 2T)
        double inner = (double)std::max<int64_t>(0, p.n0 - 2) * std::max<int64_t>(0, p.ny - 2) *
                       std::max<int64_t>(0, p.nx - 2);
        stats->gcells_per_s = stats->total_ms > 0 ? 2.0 * inner * T / (stats->total_ms * 1e-3) / 1e9 : 0;
    }
    return SO2DR_OK;
}

int so2dr_dot(so2dr_plan_t P, const void* host_a, const void* host_b, int64_t n, int dtype, double* out) {
    if (!P || !host_a || !host_b || !out || n < 0) return set_error(SO2DR_E_INVAL, "invalid argument");
    if (dtype != SO2DR_F32 && dtype != SO2DR_F64) return set_error(SO2DR_E_UNSUPPORTED, "F32 or F64 only");
    if (!P->arena || P->device < 0) return set_error(SO2DR_E_NOT_BOUND, "plan is not bound (so2dr_bind)");
    int rc;
    if ((rc = check_pinned(host_a, "host_a")) || (rc = check_pinned(host_b, "host_b"))) return rc;
    const int64_t es = dtype == SO2DR_F64 ? 8 : 4;
    // two pieces of each operand in flight (by parity); per piece, 256 FP64
    // partials, added in piece order into one FP64 slot (deterministic)
    const int64_t fixed = 2 * align_up(kPartialBlocks * 8) + align_up(8) + 6 * kAlign;
    if ((int64_t)P->arena_bytes < fixed + 4 * 4096) return set_error(SO2DR_E_INFEASIBLE, "arena too small for so2dr_dot");
    int64_t piece = ((int64_t)P->arena_bytes - fixed) / (4 * es);
    piece = std::min<int64_t>(piece / 64 * 64, (int64_t)1 << 26);
    const int64_t npieces = n > 0 ? (n + piece - 1) / piece : 0;
    RunList rl;
    int64_t off = 0;
    for (int k = 0; k < 2; ++k) {
        place(rl.bufs, kLU0 + k, 1, piece * es, 1, off);
        place(rl.bufs, kLT0 + k, 1, piece * es, 1, off);
    }
    place(rl.bufs, kLPart, 1, 2 * kPartialBlocks * 8, 1, off);
    place(rl.bufs, kLRes, 1, 8, 1, off);
    off += kAlign;
    rl.arena_bytes = (size_t)off;
    if (rl.arena_bytes > P->arena_bytes) return set_error(SO2DR_E_INFEASIBLE, "dot buffers do not fit the bound arena");
    cudaError_t e = cudaSetDevice(P->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    cudaStream_t sc = P->st[kStreamCompute], sh = P->st[kStreamH2D];
    char* ab[2] = {static_cast<char*>(const_cast<void*>(host_a)), static_cast<char*>(const_cast<void*>(host_b))};
    // event j%2 of the pool: copy of piece j landed; event 2+j%2: kernel of piece j done
    cudaEvent_t* ev = P->ev.data();
    if (npieces == 0) {
        e = cudaMemsetAsync(P->arena + rl.bufs[kLRes].offset, 0, 8, sc);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    }
    for (int64_t i = 0; i < npieces; ++i) {
        const int64_t lo = i * piece, cnt = std::min(n, lo + piece) - lo;
        const int k = (int)(i % 2);
        if (i >= 2 && (e = cudaStreamWaitEvent(sh, ev[2 + k], 0)) != cudaSuccess) return cuda_fail(e, "wait");
        for (int f = 0; f < 2; ++f) {
            e = cudaMemcpyAsync(P->arena + rl.bufs[(f ? kLT0 : kLU0) + k].offset, ab[f] + lo * es, (size_t)(cnt * es),
                                cudaMemcpyHostToDevice, sh);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
        }
        if ((e = cudaEventRecord(ev[k], sh)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        if ((e = cudaStreamWaitEvent(sc, ev[k], 0)) != cudaSuccess) return cuda_fail(e, "wait");
        Op op = make_op(kOpKernel, kStreamCompute, 0, (int)i);
        op.fn = kFnDot;
        op.pub.depth = (int)es;
        op.pub.src_buf = kLU0 + k;
        op.aux_buf = kLT0 + k;
        op.arg0 = (int64_t)k * kPartialBlocks;
        op.arg1 = cnt;
        if ((rc = enqueue_aux_kernel(P, rl, op, sc))) return rc;
        Op r = make_op(kOpKernel, kStreamCompute, 0, (int)i);
        r.fn = kFnReduce;
        r.aux_lo = (int64_t)k * kPartialBlocks;
        r.arg0 = kPartialBlocks;
        r.arg1 = 1 | (i > 0 ? 2 : 0);
        if ((rc = enqueue_aux_kernel(P, rl, r, sc))) return rc;
        if ((e = cudaEventRecord(ev[2 + k], sc)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    }
    if ((e = cudaEventRecord(P->join[1], sc)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    rc = bounded_wait({P->join[1]}, wait_timeout_s());
    if (rc) return rc;
    return read_result(P, rl, out);
}

}  // extern "C"
