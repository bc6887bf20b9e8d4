// run.cu -- executor of a plan's op list and the C ABI (so2dr.h).
//
// The executor replays the op list the planner built (plan.cpp): copies on a
// host-to-device and a device-to-host stream, kernels on a compute stream,
// with the precomputed cross-stream waits as CUDA events.  This is the stream
// pipeline of Algorithm 1 / Sec. IV-C: transfers in both directions overlap
// kernel execution.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "kernels.hpp"
#include "plan.hpp"
#include "run.hpp"

using namespace so2dr;

// ------------------------------------------------------------- error state

namespace {
thread_local std::string g_last_error;
}

namespace so2dr {

int set_error(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return set_error(SO2DR_E_CUDA, m);
}

double wait_timeout_s() {
    const char* v = std::getenv("SO2DR_TIMEOUT_S");
    double t = v ? std::atof(v) : 0.0;
    return t > 0 ? t : 600.0;
}

// Polls the events until all have completed or the deadline passes.
int bounded_wait(const std::vector<cudaEvent_t>& evs, double timeout_s) {
    auto t0 = std::chrono::steady_clock::now();
    size_t done = 0;
    std::vector<char> ok(evs.size(), 0);
    int spins = 0;
    while (done < evs.size()) {
        for (size_t i = 0; i < evs.size(); ++i) {
            if (ok[i]) continue;
            cudaError_t e = cudaEventQuery(evs[i]);
            if (e == cudaSuccess) { ok[i] = 1; ++done; }
            else if (e != cudaErrorNotReady) return cuda_fail(e, "stream completion");
        }
        if (done == evs.size()) break;
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > timeout_s) return set_error(SO2DR_E_TIMEOUT, "device work did not complete within the time limit");
        if (++spins > 64) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    return SO2DR_OK;
}

int check_pinned(const void* p, const char* what) {
    if (!p) return set_error(SO2DR_E_INVAL, std::string(what) + " is NULL");
    if (std::getenv("SO2DR_ALLOW_PAGEABLE")) return SO2DR_OK;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(SO2DR_E_NOT_PINNED, std::string(what) + " is not a CUDA-visible pointer");
    }
    if (at.type != cudaMemoryTypeHost)
        return set_error(SO2DR_E_NOT_PINNED, std::string(what) + " is not page-locked host memory");
    return SO2DR_OK;
}

}  // namespace so2dr

// ------------------------------------------------------------- plan object

so2dr_plan_s::~so2dr_plan_s() { unbind(); }

void so2dr_plan_s::unbind() {
    if (device >= 0) {
        int cur = -1;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        for (cudaEvent_t e : tev) cudaEventDestroy(e);
        for (cudaEvent_t e : join) cudaEventDestroy(e);
        for (int s = 0; s < kNumStreams; ++s)
            if (own[s] && st[s]) cudaStreamDestroy(st[s]);
        if (cur >= 0) cudaSetDevice(cur);
    }
    ev.clear();
    tev.clear();
    for (auto& row : occ_cache)
        for (int& v : row) v = 0;
    join.clear();
    for (int s = 0; s < kNumStreams; ++s) { st[s] = nullptr; own[s] = false; }
    arena = nullptr;
    arena_bytes = 0;
    device = -1;
}

namespace so2dr {

int ensure_timing_events(so2dr_plan_s* P, size_t n) {
    while (P->tev.size() < n) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return cuda_fail(err, "cudaEventCreate");
        P->tev.push_back(e);
    }
    return SO2DR_OK;
}

namespace {

int shape_of(const Plan& p) {
    if (p.kind == SO2DR_VARCOEF_STAR) return kVarcoef3D;
    if (p.kind == SO2DR_BOX) return kBox2D;
    return p.ndim == 3 ? kStar3D : kStar2D;
}

// Copies planes [lo, hi) between host and a (possibly circular) device buffer.
cudaError_t copy_planes(const Buffer& b, char* arena, char* host, int64_t host_plane_bytes,
                        int64_t host_field_bytes, int nfields, int64_t lo, int64_t hi, int64_t slot0,
                        bool to_device, cudaStream_t s) {
    int64_t n = hi - lo;
    int64_t pb = b.plane_bytes / b.nfields;  // bytes per plane per field
    int64_t fstride = b.cap * pb;            // device bytes between fields
    int64_t s0 = slot0 % b.cap;
    int64_t first = std::min(n, b.cap - s0);
    for (int f = 0; f < nfields; ++f) {
        char* h = host + f * host_field_bytes + lo * host_plane_bytes;
        char* d = arena + b.offset + f * fstride;
        int64_t segs[2][3] = {{s0, 0, first}, {0, first, n - first}};
        for (auto& sg : segs) {
            if (sg[2] <= 0) continue;
            char* dp = d + sg[0] * pb;
            char* hp = h + sg[1] * host_plane_bytes;
            cudaError_t e = to_device ? cudaMemcpyAsync(dp, hp, sg[2] * pb, cudaMemcpyHostToDevice, s)
                                      : cudaMemcpyAsync(hp, dp, sg[2] * pb, cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

}  // namespace

int enqueue_stencil(so2dr_plan_s* P, const RunList& rl, const Op& op, cudaStream_t s) {
    const Plan& p = P->p;
    const so2dr_op_t& o = op.pub;
    int shape = shape_of(p);
    int csize = p.dtype == SO2DR_F64 ? 8 : 4;
    LaunchShape ls = stencil_launch_shape(shape, p.r, o.depth, p.ny, p.nx, csize, (int)p.elem_bytes);
    ls.grid.z = 1;
    if (!ls.ok) return set_error(SO2DR_E_UNSUPPORTED, "fused depth too large for the stencil kernel");
    // host-side argument checks (the kernel trusts them)
    int64_t h = (int64_t)p.r * o.depth;
    int64_t vlo = o.edge_lo ? 0 : o.src_lo + h, vhi = o.edge_hi ? p.n0 : o.src_hi - h;
    if (o.src_hi <= o.src_lo || o.dst_lo < vlo || o.dst_hi > vhi || o.dst_hi <= o.dst_lo ||
        (o.edge_lo && o.src_lo != 0) || (o.edge_hi && o.src_hi != p.n0))
        return set_error(SO2DR_E_DEVICE_CHECK, "kernel op ranges are inconsistent");
    const Buffer& bi = rl.bufs[o.src_buf];
    const Buffer& bo = rl.bufs[o.dst_buf];
    if (o.src_hi - o.src_lo > bi.cap || o.dst_slot0 < 0 || o.dst_slot0 + (o.dst_hi - o.dst_lo) > bo.cap)
        return set_error(SO2DR_E_DEVICE_CHECK, "kernel op exceeds its buffer");
    StencilArgs a;
    std::memset(&a, 0, sizeof(a));
    a.in = P->arena + bi.offset;
    a.in_cap = bi.cap;
    a.in_slot0 = o.src_slot0 % bi.cap;
    a.in_lo = o.src_lo;
    a.in_hi = o.src_hi;
    a.out = P->arena + bo.offset + o.dst_slot0 * bo.plane_bytes;  // plane out_lo sits in slot dst_slot0
    a.out_lo = o.dst_lo;
    a.out_hi = o.dst_hi;
    if (op.aux_buf >= 0) {
        const Buffer& bc = rl.bufs[op.aux_buf];
        a.coef = P->arena + bc.offset;
        a.coef_cap = bc.cap;
        a.coef_slot0 = op.aux_slot0 % bc.cap;
        a.coef_lo = op.aux_lo;
        a.coef_field_stride = bc.cap * p.plane_cells;
    }
    a.n0 = p.n0;
    a.ny = p.ny;
    a.nx = p.nx;
    a.depth = o.depth;
    a.edge_lo = o.edge_lo;
    a.edge_hi = o.edge_hi;
    a.lx = ls.lx;
    a.ly = ls.ly;
    a.tx = ls.tx;
    a.ty = ls.ty;
    a.status = reinterpret_cast<int*>(P->arena + rl.arena_bytes - kAlign);  // the run list's status word
    if (op.host_src >= 0) {
        // zero-copy input: the device mapping of the host array
        if (op.host_src >= (int)P->host_dev.size() || !P->host_dev[op.host_src])
            return set_error(SO2DR_E_DEVICE_CHECK, "zero-copy launch without a mapped host grid");
        a.host_in = P->host_dev[op.host_src];
        a.host_lo = op.host_lo;
        a.host_hi = op.host_hi;
    }
    for (size_t k = 0; k < p.coeffs.size() && k < (size_t)kMaxCoeffsDev; ++k) {
        a.c[k] = p.coeffs[k];
        a.cf[k] = (float)p.coeffs[k];
        a.cf2[k] = make_float2(a.cf[k], a.cf[k]);
    }
    if (ls.fast) {
        // split the work so that the grid fills the SMs evenly
        int& occ = P->occ_cache[1][o.depth];
        if (!occ) occ = stencil_occupancy(p.dtype, shape, p.r, o.depth, ls);
        if (ls.fast == kFastStar3D) {
            choose_work_split(ls, o.dst_hi - o.dst_lo, p.r, o.depth, P->sm_count, occ, &a.split);
            // the round split's piece counter: one per stream (the launches
            // of a stream run one after another), beside the status word
            if (a.split && o.stream >= 0 && o.stream < kNumStreams)
                a.work_ctr = reinterpret_cast<unsigned*>(P->arena + rl.arena_bytes - kAlign + kWorkCtrOff +
                                                         8 * o.stream);
        } else {
            int64_t tiles = (int64_t)ls.grid.x * ls.grid.y;
            ls.grid.z = (unsigned)choose_segments(tiles, o.dst_hi - o.dst_lo, p.r, o.depth, P->sm_count, occ, false);
        }
    } else {
        // generic kernel: axis-0 segments too, so that a launch of few tiles
        // (a narrow 2D grid) still spreads over the SMs (one CTA per SM
        // counted; its shared memory varies with the tile)
        int64_t tiles = (int64_t)ls.grid.x * ls.grid.y;
        ls.grid.z = (unsigned)choose_segments(tiles, o.dst_hi - o.dst_lo, p.r, o.depth, P->sm_count, 1, false);
    }
    cudaError_t e = launch_stencil(p.dtype, shape, p.r, a, ls, s);
    if (e != cudaSuccess) return cuda_fail(e, "stencil launch");
    return SO2DR_OK;
}

// Replays an op list.  hosts[i] is the base pointer of host array i.
int execute(so2dr_plan_s* P, const RunList& rl, char* const* hosts, const int64_t* host_plane_bytes,
            const int64_t* host_field_bytes, so2dr_stats_t* stats, const KernelHook& hook) {
    if (!P->arena || P->device < 0) return set_error(SO2DR_E_NOT_BOUND, "plan is not bound");
    if (P->arena_bytes < rl.arena_bytes) return set_error(SO2DR_E_NOT_BOUND, "bound arena is smaller than the plan needs");
    cudaError_t e = cudaSetDevice(P->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    const size_t E = P->ev.size();
    const size_t nops = rl.ops.size();
    bool timing = stats != nullptr;
    if (timing) {
        int rc = ensure_timing_events(P, 2 * nops + 2);
        if (rc) return rc;
    }
    cudaStream_t* st = P->st;
    // device status word (the last kAlign bytes of the run list's arena): a
    // kernel whose bounded wait for a copy gave up sets it
    // (and, after it, the round split's piece counters of the streams)
    int* status = reinterpret_cast<int*>(P->arena + rl.arena_bytes - kAlign);
    if ((e = cudaMemsetAsync(status, 0, kWorkCtrOff + 8 * kNumStreams, st[kStreamH2D])) != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync(status)");
    // start marker: the compute and D2H streams start after everything the
    // caller queued on the H2D stream
    cudaEvent_t start = P->join[0];
    if ((e = cudaEventRecord(start, st[kStreamH2D])) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    for (int s = 1; s < kNumStreams; ++s)
        if ((e = cudaStreamWaitEvent(st[s], start, 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    cudaEvent_t tstart = timing ? P->tev[2 * nops] : nullptr;
    if (timing && (e = cudaEventRecord(tstart, st[kStreamH2D])) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    double h2d_bytes = 0, d2h_bytes = 0;
    int64_t launches = 0;
    for (size_t j = 0; j < nops; ++j) {
        const Op& op = rl.ops[j];
        const so2dr_op_t& o = op.pub;
        cudaStream_t s = st[o.stream];
        for (int w = 0; w < kNumStreams; ++w) {
            if (o.wait_op[w] < 0 || w == o.stream) continue;
            e = cudaStreamWaitEvent(s, P->ev[(size_t)o.wait_op[w] % E], 0);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
        }
        if (timing && (e = cudaEventRecord(P->tev[2 * j], s)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        if (o.kind == kOpD2D) {
            const Buffer& bs = rl.bufs[o.src_buf];
            const Buffer& bd = rl.bufs[o.dst_buf];
            const int64_t n = o.src_hi - o.src_lo;
            if (o.src_slot0 < 0 || o.dst_slot0 < 0 || o.src_slot0 + n > bs.cap || o.dst_slot0 + n > bd.cap)
                return set_error(SO2DR_E_DEVICE_CHECK, "on-device copy exceeds its buffer");
            e = cudaMemcpyAsync(P->arena + bd.offset + o.dst_slot0 * bd.plane_bytes,
                                P->arena + bs.offset + o.src_slot0 * bs.plane_bytes, (size_t)(n * bs.plane_bytes),
                                cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return cuda_fail(e, "on-device copy");
        } else if (o.kind == kOpH2D || o.kind == kOpD2H) {
            bool h2d = o.kind == kOpH2D;
            int bid = h2d ? o.dst_buf : o.src_buf;
            const Buffer& b = rl.bufs[bid];
            int64_t lo = h2d ? o.dst_lo : o.src_lo, hi = h2d ? o.dst_hi : o.src_hi;
            int64_t slot0 = h2d ? o.dst_slot0 : o.src_slot0;
            char* host = hosts[op.host_array];
            int nf = std::max(1, op.nfields);
            e = copy_planes(b, P->arena, host, host_plane_bytes[op.host_array], host_field_bytes[op.host_array],
                            nf, lo, hi, slot0, h2d, s);
            if (e != cudaSuccess) return cuda_fail(e, h2d ? "host-to-device copy" : "device-to-host copy");
            double bytes = (double)(hi - lo) * (double)(b.plane_bytes / b.nfields) * nf;
            (h2d ? h2d_bytes : d2h_bytes) += bytes;
        } else {
            int rc = hook ? hook(P, rl, op, s) : enqueue_stencil(P, rl, op, s);
            if (rc) return rc;
            ++launches;
        }
        if (timing && (e = cudaEventRecord(P->tev[2 * j + 1], s)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        if (op.waited && (e = cudaEventRecord(P->ev[j % E], s)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    }
    // join
    std::vector<cudaEvent_t> ends;
    for (int s = 0; s < kNumStreams; ++s) {
        if ((e = cudaEventRecord(P->join[1 + s], st[s])) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        ends.push_back(P->join[1 + s]);
    }
    cudaEvent_t tend = timing ? P->tev[2 * nops + 1] : nullptr;
    if (timing) {
        for (int s = 0; s < kNumStreams; ++s)
            if (s != kStreamD2H && (e = cudaStreamWaitEvent(st[kStreamD2H], P->join[1 + s], 0)) != cudaSuccess)
                return cuda_fail(e, "cudaStreamWaitEvent");
        if ((e = cudaEventRecord(tend, st[kStreamD2H])) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        ends.push_back(tend);
    }
    int rc = bounded_wait(ends, wait_timeout_s());
    if (rc) return rc;
    int hstatus = 0;
    if ((e = cudaMemcpy(&hstatus, status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "status read");
    if (hstatus) return set_error(SO2DR_E_TIMEOUT, "a kernel's wait for a staged plane gave up");
    if (timing) {
        float ms = 0;
        std::memset(stats, 0, sizeof(*stats));
        cudaEventElapsedTime(&ms, tstart, tend);
        stats->total_ms = ms;
        P->tl_start.assign(nops, 0.0);
        P->tl_end.assign(nops, 0.0);
        for (size_t j = 0; j < nops; ++j) {
            float d = 0, t0 = 0, t1 = 0;
            cudaEventElapsedTime(&d, P->tev[2 * j], P->tev[2 * j + 1]);
            cudaEventElapsedTime(&t0, tstart, P->tev[2 * j]);
            cudaEventElapsedTime(&t1, tstart, P->tev[2 * j + 1]);
            P->tl_start[j] = t0;
            P->tl_end[j] = t1;
            const so2dr_op_t& o = rl.ops[j].pub;
            if (o.kind == kOpH2D) stats->h2d_ms += d;
            else if (o.kind == kOpD2H) stats->d2h_ms += d;
            else {
                stats->kernel_ms += d;
                const Plan& pp = P->p;
                const bool rr = &rl == &pp.rr;  // the result-reuse code runs depth-1 launches only
                if (o.depth == (rr ? 1 : pp.k_on) && rl.ops[j].fn == kFnStencil) {
                    // algorithmic cells: the chunk's owned planes (the whole grid in-core;
                    // the launch's own output planes in the result-reuse code)
                    int64_t owned = (&rl == &pp.ooc || &rl == &pp.zc) ? pp.starts[o.chunk + 1] - pp.starts[o.chunk]
                                                     : rr ? o.dst_hi - o.dst_lo : pp.n0;
                    stats->main_kernel_ms += d;
                    stats->main_kernel_launches += 1;
                    stats->main_kernel_cells += (double)owned * (double)pp.plane_cells;
                }
            }
        }
        stats->h2d_bytes = h2d_bytes;
        stats->d2h_bytes = d2h_bytes;
        stats->launches = launches;
        stats->ops = (int64_t)nops;
    }
    return SO2DR_OK;
}

}  // namespace so2dr

namespace so2dr {

int plan_create(so2dr_plan_t* out, int ndim, const int64_t* dims, int radius, int kind, const double* coeffs,
                int ncoeffs, int64_t time_steps, int min_chunks, int k_on, int k_off, size_t device_budget_bytes,
                int storage, double link_h2d_gbs, double link_d2h_gbs, double hbm_gbs, const PlanSearch* search) {
    if (!out) return set_error(SO2DR_E_INVAL, "out is NULL");
    *out = nullptr;
    so2dr_plan_s* P = new (std::nothrow) so2dr_plan_s();
    if (!P) return set_error(SO2DR_E_NOMEM, "plan allocation failed");
    std::string err;
    int csize = storage == SO2DR_F64 ? 8 : 4;
    int shape = kind == SO2DR_VARCOEF_STAR ? kVarcoef3D : kind == SO2DR_BOX ? kBox2D : (ndim == 3 ? kStar3D : kStar2D);
    int maxd = (radius >= 1 && radius <= kMaxRadius) ? stencil_max_depth(shape, radius, csize) : kMaxKon;
    int rc;
    try {
        P->p.max_kon = maxd;
        // the automatic choice stays within the register-streaming kernel when
        // it covers this stencil (the generic kernel is far slower)
        if (shape == kStar3D && storage != SO2DR_F64 && ndim == 3 && dims && dims[2] % 4 == 0) {
            int fm = 0;
            for (int d = 1; d <= kMaxKon; ++d)
                if (fast_star3d_supported(radius, d)) fm = d;
            if (fm > 0) P->p.max_kon_auto = fm;
        }
        if (shape == kBox2D && storage != SO2DR_F64 && ndim == 2 && dims && dims[1] % 4 == 0) {
            int fm = 0;
            for (int d = 1; d <= kMaxKon; ++d)
                if (fast_box2d_supported(radius, d)) fm = d;
            if (fm > 0) P->p.max_kon_auto = fm;
        }
        rc = build_plan(P->p, ndim, dims, radius, kind, coeffs, ncoeffs, time_steps, min_chunks, k_on, k_off,
                        device_budget_bytes, storage, link_h2d_gbs, link_d2h_gbs, hbm_gbs, &err, search);
    } catch (const std::bad_alloc&) {
        delete P;
        return set_error(SO2DR_E_NOMEM, "host allocation failed while planning");
    }
    if (rc) {
        delete P;
        return set_error(rc, err);
    }
    *out = P;
    return SO2DR_OK;
}

}  // namespace so2dr

// ==================================================================== C ABI

extern "C" {

int so2dr_abi_version(void) { return 5; }

const char* so2dr_strerror(int status) {
    switch (status) {
        case SO2DR_OK: return "ok";
        case SO2DR_E_INVAL: return "invalid argument";
        case SO2DR_E_INFEASIBLE: return "infeasible: no chunking fits the device budget";
        case SO2DR_E_NOT_BOUND: return "plan not bound to a large enough device arena";
        case SO2DR_E_CUDA: return "CUDA runtime error";
        case SO2DR_E_TIMEOUT: return "bounded wait on the device timed out";
        case SO2DR_E_DEVICE_CHECK: return "device-side argument or index check failed";
        case SO2DR_E_NOMEM: return "host allocation failed";
        case SO2DR_E_NOT_PINNED: return "host buffer is not page-locked";
        case SO2DR_E_UNSUPPORTED: return "unsupported configuration";
        default: return "unknown status";
    }
}

const char* so2dr_last_error(void) { return g_last_error.c_str(); }

int so2dr_plan_ex(so2dr_plan_t* out, int ndim, const int64_t* dims, int radius, int kind,
                  const double* coeffs, int ncoeffs, int64_t time_steps, int min_chunks, int k_on,
                  int k_off, size_t device_budget_bytes, int storage, double link_h2d_gbs,
                  double link_d2h_gbs, double hbm_gbs) {
    return so2dr::plan_create(out, ndim, dims, radius, kind, coeffs, ncoeffs, time_steps, min_chunks, k_on,
                              k_off, device_budget_bytes, storage, link_h2d_gbs, link_d2h_gbs, hbm_gbs, nullptr);
}

int so2dr_plan(so2dr_plan_t* out, int ndim, const int64_t* dims, int radius, int kind, const double* coeffs,
               int ncoeffs, int64_t time_steps, int min_chunks, int k_on, int k_off,
               size_t device_budget_bytes, int storage) {
    return so2dr_plan_ex(out, ndim, dims, radius, kind, coeffs, ncoeffs, time_steps, min_chunks, k_on, k_off,
                         device_budget_bytes, storage, 0, 0, 0);
}

int so2dr_plan_info(so2dr_plan_t P, so2dr_plan_info_t* info) {
    if (!P || !info) return set_error(SO2DR_E_INVAL, "NULL argument");
    const Plan& p = P->p;
    std::memset(info, 0, sizeof(*info));
    info->ndim = p.ndim;
    info->dims[0] = p.n0;
    info->dims[1] = p.ndim == 3 ? p.ny : p.nx;
    info->dims[2] = p.ndim == 3 ? p.nx : 1;
    info->radius = p.r;
    info->kind = p.kind;
    info->dtype = p.dtype;
    info->time_steps = p.T;
    info->k_off = p.k_off;
    info->k_on = p.k_on;
    info->rounds = p.rounds;
    info->chunks = p.d;
    info->n_streams = kNumStreams;
    int64_t pm = 0;
    for (int i = 0; i < p.d; ++i) pm = std::max(pm, p.starts[i + 1] - p.starts[i]);
    info->max_chunk_planes = pm;
    info->ring_planes = p.ring_planes;
    info->plane_bytes = p.plane_bytes;
    info->arena_bytes = p.ooc.arena_bytes;
    info->arena_bytes_in_core = p.ic.arena_bytes;
    info->host_workspace_bytes = adjoint_workspace_bytes(p);
    info->ops_per_run = (int64_t)p.ooc.ops.size();
    int64_t launches = 0;
    double hb = 0, db = 0;
    for (const Op& op : p.ooc.ops) {
        const so2dr_op_t& o = op.pub;
        if (o.kind == kOpKernel) ++launches;
        else {
            const Buffer& b = p.ooc.bufs[o.kind == kOpH2D ? o.dst_buf : o.src_buf];
            double bytes = (double)(o.src_hi - o.src_lo) * (double)b.plane_bytes;
            (o.kind == kOpH2D ? hb : db) += bytes;
        }
    }
    info->launches_per_run = launches;
    info->h2d_bytes_per_run = hb;
    info->d2h_bytes_per_run = db;
    info->cell_updates_per_run = p.cell_updates();
    info->redundancy = p.redundancy;
    info->lookahead = p.lookahead;
    info->out_slabs = p.n_out;
    info->arena_bytes_result_reuse = p.rr_chunks ? p.rr.arena_bytes : 0;
    info->result_reuse_chunks = p.rr_chunks;
    info->zero_copy = p.zc_ok ? 1 : 0;
    return SO2DR_OK;
}

int so2dr_run_timeline(so2dr_plan_t P, double* start_ms, double* end_ms, int64_t max_ops, int64_t* n_ops) {
    if (!P || !n_ops) return set_error(SO2DR_E_INVAL, "NULL argument");
    *n_ops = (int64_t)P->tl_start.size();
    if (!start_ms && !end_ms) return SO2DR_OK;
    if (!start_ms || !end_ms) return set_error(SO2DR_E_INVAL, "start_ms and end_ms must both be given");
    if (max_ops < *n_ops) return set_error(SO2DR_E_INVAL, "arrays too small");
    for (int64_t j = 0; j < *n_ops; ++j) {
        start_ms[j] = P->tl_start[(size_t)j];
        end_ms[j] = P->tl_end[(size_t)j];
    }
    return SO2DR_OK;
}

int so2dr_plan_chunks(so2dr_plan_t P, int64_t* starts, int max_entries) {
    if (!P || !starts) return set_error(SO2DR_E_INVAL, "NULL argument");
    if (max_entries < P->p.d + 1) return set_error(SO2DR_E_INVAL, "starts array too small");
    for (int i = 0; i <= P->p.d; ++i) starts[i] = P->p.starts[i];
    return SO2DR_OK;
}

int so2dr_plan_ops(so2dr_plan_t P, int in_core, so2dr_op_t* ops, int64_t max_ops, int64_t* n_ops) {
    if (!P || !n_ops) return set_error(SO2DR_E_INVAL, "NULL argument");
    const RunList& rl = in_core == 3 ? P->p.zc : in_core == 2 ? P->p.rr : (in_core ? P->p.ic : P->p.ooc);
    *n_ops = (int64_t)rl.ops.size();
    if (!ops) return SO2DR_OK;
    if (max_ops < *n_ops) return set_error(SO2DR_E_INVAL, "ops array too small");
    for (size_t j = 0; j < rl.ops.size(); ++j) ops[j] = rl.ops[j].pub;
    return SO2DR_OK;
}

int so2dr_plan_buffers(so2dr_plan_t P, int in_core, so2dr_buffer_t* bufs, int max_bufs, int* n_bufs) {
    if (!P || !n_bufs) return set_error(SO2DR_E_INVAL, "NULL argument");
    const RunList& rl = in_core == 3 ? P->p.zc : in_core == 2 ? P->p.rr : (in_core ? P->p.ic : P->p.ooc);
    *n_bufs = (int)rl.bufs.size();
    if (!bufs) return SO2DR_OK;
    if (max_bufs < *n_bufs) return set_error(SO2DR_E_INVAL, "bufs array too small");
    for (size_t i = 0; i < rl.bufs.size(); ++i) {
        bufs[i].offset_bytes = rl.bufs[i].offset;
        bufs[i].capacity_planes = rl.bufs[i].cap;
    }
    return SO2DR_OK;
}

int so2dr_bind(so2dr_plan_t P, void* device_arena, size_t arena_bytes, void* const* cuda_streams, int nstreams) {
    if (!P || !device_arena) return set_error(SO2DR_E_INVAL, "NULL argument");
    if (nstreams != 3 && nstreams != 4) return set_error(SO2DR_E_INVAL, "three or four streams are required");
    if (reinterpret_cast<uintptr_t>(device_arena) % 256) return set_error(SO2DR_E_INVAL, "arena must be 256-byte aligned");
    P->unbind();
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    cudaPointerAttributes at;
    e = cudaPointerGetAttributes(&at, device_arena);
    if (e != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return set_error(SO2DR_E_INVAL, "arena is not device memory");
    }
    P->device = dev;
    if (cudaDeviceGetAttribute(&P->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        P->sm_count = 0;
    }
    for (int s = 0; s < kNumStreams; ++s) {
        if (cuda_streams && s < nstreams && cuda_streams[s]) {
            P->st[s] = static_cast<cudaStream_t>(cuda_streams[s]);
        } else {
            e = cudaStreamCreateWithFlags(&P->st[s], cudaStreamNonBlocking);
            if (e != cudaSuccess) { P->unbind(); return cuda_fail(e, "cudaStreamCreate"); }
            P->own[s] = true;
        }
    }
    const size_t E = 256;
    for (size_t i = 0; i < E; ++i) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) { P->unbind(); return cuda_fail(e, "cudaEventCreate"); }
        P->ev.push_back(ev);
    }
    for (int i = 0; i < 1 + kNumStreams; ++i) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) { P->unbind(); return cuda_fail(e, "cudaEventCreate"); }
        P->join.push_back(ev);
    }
    P->arena = static_cast<char*>(device_arena);
    P->arena_bytes = arena_bytes;
    return SO2DR_OK;
}

int so2dr_run(so2dr_plan_t P, void* host_grid, const void* host_coeff_fields, int in_core, so2dr_stats_t* stats) {
    if (!P) return set_error(SO2DR_E_INVAL, "plan is NULL");
    const Plan& p = P->p;
    if (!P->arena || P->device < 0) return set_error(SO2DR_E_NOT_BOUND, "plan is not bound (so2dr_bind)");
    if (!host_grid) return set_error(SO2DR_E_INVAL, "host_grid is NULL");
    int rc = check_pinned(host_grid, "host_grid");
    if (rc) return rc;
    bool vc = p.kind == SO2DR_VARCOEF_STAR;
    if (vc) {
        rc = check_pinned(host_coeff_fields, "host_coeff_fields");
        if (rc) return rc;
    }
    if (in_core < 0 || in_core > 3) return set_error(SO2DR_E_INVAL, "mode must be 0, 1, 2 or 3");
    if (in_core == 2 && p.rr_chunks == 0)
        return set_error(SO2DR_E_UNSUPPORTED, "the result-reuse code needs a constant-coefficient plan that fits");
    if (in_core == 3 && !p.zc_ok)
        return set_error(SO2DR_E_UNSUPPORTED, "zero-copy input needs a 3D constant-coefficient star on the 3D star kernel");
    const RunList& rl = in_core == 3 ? p.zc : in_core == 2 ? p.rr : (in_core ? p.ic : p.ooc);
    P->host_dev.assign(1, nullptr);
    if (in_core == 3) {
        void* d = nullptr;
        cudaError_t e = cudaHostGetDevicePointer(&d, host_grid, 0);
        if (e != cudaSuccess || !d) return cuda_fail(e, "cudaHostGetDevicePointer(host_grid)");
        P->host_dev[0] = static_cast<char*>(d);
    }
    char* hosts[2] = {static_cast<char*>(host_grid), const_cast<char*>(static_cast<const char*>(host_coeff_fields))};
    int64_t cb = p.dtype == SO2DR_F64 ? 8 : 4;
    int64_t hpb[2] = {p.plane_bytes, p.plane_cells * cb};
    int64_t hfb[2] = {0, p.n0 * p.plane_cells * cb};
    rc = execute(P, rl, hosts, hpb, hfb, stats, KernelHook());
    if (rc) return rc;
    if (stats) stats->gcells_per_s = stats->total_ms > 0 ? p.cell_updates() / (stats->total_ms * 1e-3) / 1e9 : 0;
    return SO2DR_OK;
}

void so2dr_destroy(so2dr_plan_t P) { delete P; }

}  // extern "C"
