// tune.cu -- the run-time parameter search of Sec. IV-C: the cost model's
// ranked candidate list, plans built from one candidate, and the measured
// autotune that times the best candidates on the device (the trade-off that
// Sec. V-B's Fig. 5 measures), and the host-link / HBM measurement they use.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <initializer_list>
#include <vector>

#include "run.hpp"

using namespace so2dr;

namespace {

void to_entry(const Candidate& c, so2dr_tune_entry_t* e) {
    e->k_off = c.k_off;
    e->k_on = c.k_on;
    e->chunks = c.d;
    e->lookahead = c.lookahead;
    e->out_slabs = c.n_out;
    e->status = SO2DR_OK;
    e->predicted_ms = c.predicted_ms;
    e->measured_ms = -1.0;
}

struct Problem {
    int ndim;
    const int64_t* dims;
    int radius, kind;
    const double* coeffs;
    int ncoeffs;
    int64_t T;
    int min_chunks, k_on, k_off;
    size_t budget;
    int storage;
};

// Every feasible candidate, cheapest predicted first.
int rank(const Problem& q, double h2d, double d2h, double hbm, std::vector<Candidate>& out) {
    PlanSearch s;
    s.ranked = &out;
    so2dr_plan_t P = nullptr;
    int rc = plan_create(&P, q.ndim, q.dims, q.radius, q.kind, q.coeffs, q.ncoeffs, q.T, q.min_chunks, q.k_on,
                         q.k_off, q.budget, q.storage, h2d, d2h, hbm, &s);
    if (P) so2dr_destroy(P);
    if (rc) return rc;
    std::stable_sort(out.begin(), out.end(),
                     [](const Candidate& a, const Candidate& b) { return a.predicted_ms < b.predicted_ms; });
    return SO2DR_OK;
}

int plan_for(const Problem& q, const so2dr_tune_entry_t& e, double h2d, double d2h, double hbm,
             so2dr_plan_t* out) {
    if (e.k_off < 1 || e.k_on < 1 || e.chunks < 1 || (e.lookahead != 0 && e.lookahead != 1) ||
        (e.out_slabs != 1 && e.out_slabs != 2))
        return set_error(SO2DR_E_INVAL, "table entry out of range");
    PlanSearch s;
    s.lookahead = e.lookahead;
    s.n_out = e.out_slabs;
    int rc = plan_create(out, q.ndim, q.dims, q.radius, q.kind, q.coeffs, q.ncoeffs, q.T, e.chunks, e.k_on, e.k_off,
                         q.budget, q.storage, h2d, d2h, hbm, &s);
    if (rc) return rc;
    so2dr_plan_info_t info;
    so2dr_plan_info(*out, &info);
    if (info.chunks != e.chunks) {
        so2dr_destroy(*out);
        *out = nullptr;
        return set_error(SO2DR_E_INFEASIBLE, "the entry's chunk count does not fit the budget");
    }
    return SO2DR_OK;
}

// Least time of `reps` copies of `bytes` (ms), or a negative status.
int time_copy(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s, int reps,
              double* best_ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return cuda_fail(e, "event creation");
    }
    int rc = SO2DR_OK;
    *best_ms = -1.0;
    for (int i = 0; i < reps && rc == SO2DR_OK; ++i) {
        e = cudaEventRecord(a, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, kind, s);
        if (e == cudaSuccess) e = cudaEventRecord(b, s);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "link measurement copy");
            break;
        }
        rc = bounded_wait({b}, wait_timeout_s());
        float ms = 0.f;
        if (rc == SO2DR_OK && cudaEventElapsedTime(&ms, a, b) == cudaSuccess && ms > 0.f)
            if (*best_ms < 0 || ms < *best_ms) *best_ms = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return rc;
}

bool fatal(int rc) { return rc == SO2DR_E_CUDA || rc == SO2DR_E_TIMEOUT || rc == SO2DR_E_DEVICE_CHECK; }

// SM-driven copy of n 16-byte vectors (grid-stride, 4 vectors in flight per
// thread); either side may be mapped host memory
__global__ void __launch_bounds__(512) link_copy_kernel(const int4* __restrict__ src, int4* __restrict__ dst,
                                                        size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        const int4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
        dst[i] = a;
        dst[i + stride] = b;
        dst[i + 2 * stride] = c;
        dst[i + 3 * stride] = d;
    }
    for (; i < n; i += stride) dst[i] = src[i];
}

struct Xfer {
    void* dst;
    const void* src;
    cudaMemcpyKind kind;  // copy engine, or cudaMemcpyDefault for the SM kernel
};

// Runs one or two transfers at once (one stream each), `reps` times; best
// GB/s of each in gbs[] (0 on no timing).
int time_xfers(const Xfer* x, int nx, size_t bytes, int ctas, int reps, cudaStream_t* st, cudaEvent_t* ev,
               double* gbs) {
    for (int k = 0; k < nx; ++k) gbs[k] = 0;
    for (int r = 0; r < reps; ++r) {
        for (int k = 0; k < nx; ++k) {
            cudaError_t e = cudaEventRecord(ev[2 * k], st[k]);
            if (e == cudaSuccess) {
                if (x[k].kind == cudaMemcpyDefault) {
                    link_copy_kernel<<<ctas, 512, 0, st[k]>>>(static_cast<const int4*>(x[k].src),
                                                              static_cast<int4*>(x[k].dst), bytes / 16);
                    e = cudaGetLastError();
                } else {
                    e = cudaMemcpyAsync(x[k].dst, x[k].src, bytes, x[k].kind, st[k]);
                }
            }
            if (e == cudaSuccess) e = cudaEventRecord(ev[2 * k + 1], st[k]);
            if (e != cudaSuccess) return cuda_fail(e, "link measurement");
        }
        std::vector<cudaEvent_t> ends;
        for (int k = 0; k < nx; ++k) ends.push_back(ev[2 * k + 1]);
        int rc = bounded_wait(ends, wait_timeout_s());
        if (rc) return rc;
        for (int k = 0; k < nx; ++k) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]) == cudaSuccess && ms > 0.f)
                gbs[k] = std::max(gbs[k], bytes / (ms * 1e-3) / 1e9);
        }
    }
    return SO2DR_OK;
}

}  // namespace

extern "C" {

int so2dr_plan_candidates(int ndim, const int64_t* dims, int radius, int kind, const double* coeffs, int ncoeffs,
                          int64_t time_steps, int min_chunks, int k_on, int k_off, size_t device_budget_bytes,
                          int storage, double link_h2d_gbs, double link_d2h_gbs, double hbm_gbs,
                          so2dr_tune_entry_t* table, int table_cap, int* table_len) {
    if (!table_len) return set_error(SO2DR_E_INVAL, "table_len is NULL");
    *table_len = 0;
    if (table_cap > 0 && !table) return set_error(SO2DR_E_INVAL, "table is NULL");
    Problem q{ndim, dims, radius, kind, coeffs, ncoeffs, time_steps, min_chunks, k_on, k_off,
              device_budget_bytes, storage};
    std::vector<Candidate> c;
    int rc = rank(q, link_h2d_gbs, link_d2h_gbs, hbm_gbs, c);
    if (rc) return rc;
    *table_len = (int)c.size();
    for (int i = 0; i < (int)c.size() && i < table_cap; ++i) to_entry(c[i], &table[i]);
    return SO2DR_OK;
}

int so2dr_plan_tuned(so2dr_plan_t* out, int ndim, const int64_t* dims, int radius, int kind, const double* coeffs,
                     int ncoeffs, int64_t time_steps, const so2dr_tune_entry_t* entry, size_t device_budget_bytes,
                     int storage) {
    if (!out) return set_error(SO2DR_E_INVAL, "out is NULL");
    *out = nullptr;
    if (!entry) return set_error(SO2DR_E_INVAL, "entry is NULL");
    Problem q{ndim, dims, radius, kind, coeffs, ncoeffs, time_steps, 1, 0, 0, device_budget_bytes, storage};
    return plan_for(q, *entry, 0, 0, 0, out);
}

int so2dr_measure_link(void* host_a, void* host_b, void* device_arena, size_t bytes, int sm_ctas, int repeats,
                       double* out) {
    if (!host_a || !host_b || !device_arena || !out) return set_error(SO2DR_E_INVAL, "NULL argument");
    if (bytes < ((size_t)1 << 20) || bytes % 16) return set_error(SO2DR_E_INVAL, "bytes must be >= 1 MiB and a multiple of 16");
    if (sm_ctas < 1 || repeats < 1) return set_error(SO2DR_E_INVAL, "sm_ctas and repeats must be >= 1");
    int rc = check_pinned(host_a, "host_a");
    if (rc == SO2DR_OK) rc = check_pinned(host_b, "host_b");
    if (rc) return rc;
    for (int k = 0; k < 9; ++k) out[k] = -1.0;
    void *ma = nullptr, *mb = nullptr;  // device views of the pinned buffers
    const bool mapped = cudaHostGetDevicePointer(&ma, host_a, 0) == cudaSuccess &&
                        cudaHostGetDevicePointer(&mb, host_b, 0) == cudaSuccess;
    if (!mapped) cudaGetLastError();
    char* d0 = static_cast<char*>(device_arena);
    char* d1 = d0 + bytes;
    cudaStream_t st[2] = {nullptr, nullptr};
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&st[k], cudaStreamNonBlocking);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventCreate(&ev[k]);
    if (e != cudaSuccess) rc = cuda_fail(e, "stream or event creation");
    double g[2];
    auto run = [&](std::initializer_list<Xfer> xs, int o0) {
        if (rc) return;
        std::vector<Xfer> v(xs);
        rc = time_xfers(v.data(), (int)v.size(), bytes, sm_ctas, repeats, st, ev, g);
        for (size_t k = 0; k < v.size() && rc == SO2DR_OK; ++k) out[o0 + k] = g[k];
    };
    run({{d0, host_a, cudaMemcpyHostToDevice}}, 0);
    run({{host_b, d1, cudaMemcpyDeviceToHost}}, 1);
    run({{d0, host_a, cudaMemcpyHostToDevice}, {host_b, d1, cudaMemcpyDeviceToHost}}, 2);
    if (mapped) {
        run({{d0, ma, cudaMemcpyDefault}}, 4);
        run({{mb, d1, cudaMemcpyDefault}}, 5);
        run({{d0, ma, cudaMemcpyDefault}, {mb, d1, cudaMemcpyDefault}}, 6);
    }
    run({{d1, d0, cudaMemcpyDeviceToDevice}}, 8);
    if (rc == SO2DR_OK && out[8] > 0) out[8] *= 2.0;  // read + write
    for (int k = 0; k < 4; ++k)
        if (ev[k]) cudaEventDestroy(ev[k]);
    for (int k = 0; k < 2; ++k)
        if (st[k]) cudaStreamDestroy(st[k]);
    return rc;
}

int so2dr_autotune(int ndim, const int64_t* dims, int radius, int kind, const double* coeffs, int ncoeffs,
                   int64_t time_steps, int min_chunks, int k_on, int k_off, size_t device_budget_bytes, int storage,
                   void* device_arena, void* const* cuda_streams, int nstreams, void* scratch_host_grid,
                   int max_candidates, int repeats, so2dr_tune_entry_t* table, int table_cap, int* table_len,
                   double* link_gbs) {
    if (!table_len) return set_error(SO2DR_E_INVAL, "table_len is NULL");
    *table_len = 0;
    if (table_cap > 0 && !table) return set_error(SO2DR_E_INVAL, "table is NULL");
    if (!device_arena) return set_error(SO2DR_E_INVAL, "device_arena is NULL");
    if (max_candidates < 1 || repeats < 1) return set_error(SO2DR_E_INVAL, "max_candidates and repeats must be >= 1");
    if (kind == SO2DR_VARCOEF_STAR) return set_error(SO2DR_E_UNSUPPORTED, "autotune covers constant-coefficient stencils");
    if (device_budget_bytes == 0) return set_error(SO2DR_E_INVAL, "the autotune needs a finite device budget");
    if (nstreams != 3 && nstreams != 4) return set_error(SO2DR_E_INVAL, "nstreams must be 3 or 4");
    Problem q{ndim, dims, radius, kind, coeffs, ncoeffs, time_steps, min_chunks, k_on, k_off,
              device_budget_bytes, storage};
    std::vector<Candidate> cands;
    int rc = rank(q, 0, 0, 0, cands);  // validates the problem before any device work
    if (rc) return rc;
    rc = check_pinned(scratch_host_grid, "scratch_host_grid");
    if (rc) return rc;
    const int64_t cells = dims[0] * dims[1] * (ndim == 3 ? dims[2] : 1);
    const size_t grid_bytes = (size_t)cells * (size_t)elem_size(storage);

    // 1. link and HBM rates on the caller's buffers
    cudaStream_t sh = nullptr, sd = nullptr;
    bool own_h = false, own_d = false;
    if (cuda_streams && cuda_streams[0]) sh = (cudaStream_t)cuda_streams[0];
    if (cuda_streams && cuda_streams[2]) sd = (cudaStream_t)cuda_streams[2];
    cudaError_t ce = cudaSuccess;
    if (!sh && (ce = cudaStreamCreateWithFlags(&sh, cudaStreamNonBlocking)) == cudaSuccess) own_h = true;
    if (ce == cudaSuccess && !sd && (ce = cudaStreamCreateWithFlags(&sd, cudaStreamNonBlocking)) == cudaSuccess)
        own_d = true;
    double h2d = 0, d2h = 0, hbm = 0;
    if (ce != cudaSuccess) rc = cuda_fail(ce, "stream creation");
    const size_t gib = (size_t)1 << 30;
    size_t link_bytes = std::min(std::min(grid_bytes, device_budget_bytes), gib) & ~(size_t)4095;
    size_t half = std::min(device_budget_bytes / 2, gib) & ~(size_t)4095;
    double ms = -1.0;
    if (rc == SO2DR_OK && link_bytes >= ((size_t)1 << 20)) {
        rc = time_copy(device_arena, scratch_host_grid, link_bytes, cudaMemcpyHostToDevice, sh, 3, &ms);
        if (rc == SO2DR_OK && ms > 0) h2d = link_bytes / (ms * 1e-3) / 1e9;
        if (rc == SO2DR_OK) rc = time_copy(scratch_host_grid, device_arena, link_bytes, cudaMemcpyDeviceToHost, sd, 3, &ms);
        if (rc == SO2DR_OK && ms > 0) d2h = link_bytes / (ms * 1e-3) / 1e9;
    }
    if (rc == SO2DR_OK && half >= ((size_t)1 << 20)) {
        rc = time_copy((char*)device_arena + half, device_arena, half, cudaMemcpyDeviceToDevice, sh, 3, &ms);
        if (rc == SO2DR_OK && ms > 0) hbm = 2.0 * half / (ms * 1e-3) / 1e9;  // read + write
    }
    if (own_h) cudaStreamDestroy(sh);
    if (own_d) cudaStreamDestroy(sd);
    if (rc) return rc;
    if (link_gbs) {
        link_gbs[0] = h2d;
        link_gbs[1] = d2h;
        link_gbs[2] = hbm;
    }

    // 2. the model's ranking with the measured rates
    cands.clear();
    rc = rank(q, h2d, d2h, hbm, cands);
    if (rc) return rc;
    std::vector<so2dr_tune_entry_t> tab(cands.size());
    for (size_t i = 0; i < cands.size(); ++i) to_entry(cands[i], &tab[i]);

    // 3. time the best few
    const int n = std::min<int>(max_candidates, (int)tab.size());
    for (int i = 0; i < n; ++i) {
        so2dr_tune_entry_t& e = tab[i];
        so2dr_plan_t P = nullptr;
        int s = plan_for(q, e, h2d, d2h, hbm, &P);
        if (s == SO2DR_OK) s = so2dr_bind(P, device_arena, device_budget_bytes, cuda_streams, nstreams);
        double best = -1.0;
        for (int r = 0; r < repeats && s == SO2DR_OK; ++r) {
            so2dr_stats_t st;
            std::memset(&st, 0, sizeof(st));
            s = so2dr_run(P, scratch_host_grid, nullptr, 0, &st);
            if (s == SO2DR_OK && (best < 0 || st.total_ms < best)) best = st.total_ms;
        }
        if (P) so2dr_destroy(P);
        e.status = s;
        e.measured_ms = s == SO2DR_OK ? best : -1.0;
        if (fatal(s)) return s;
    }
    std::stable_sort(tab.begin(), tab.end(), [](const so2dr_tune_entry_t& a, const so2dr_tune_entry_t& b) {
        const bool ta = a.measured_ms >= 0, tb = b.measured_ms >= 0;
        if (ta != tb) return ta;
        return ta ? a.measured_ms < b.measured_ms : a.predicted_ms < b.predicted_ms;
    });
    *table_len = (int)tab.size();
    for (int i = 0; i < (int)tab.size() && i < table_cap; ++i) table[i] = tab[i];
    return SO2DR_OK;
}

}  // extern "C"
