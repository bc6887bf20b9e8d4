// run.hpp -- the plan object behind so2dr_plan_t and the executor interface.
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <string>
#include <vector>

#include "plan.hpp"

struct so2dr_plan_s {
    so2dr::Plan p;
    // binding (so2dr_bind)
    char* arena = nullptr;
    size_t arena_bytes = 0;
    cudaStream_t st[so2dr::kNumStreams] = {nullptr, nullptr, nullptr};
    bool own[so2dr::kNumStreams] = {false, false, false};
    std::vector<cudaEvent_t> ev;    // completion events, op j uses ev[j % size]
    std::vector<cudaEvent_t> join;  // start marker + one per stream
    std::vector<cudaEvent_t> tev;   // timing events (2 per op), created on demand
    int device = -1;
    int sm_count = 0;
    int occ_cache[2][17] = {};      // CTAs per SM of the fast / generic launch per depth
    std::vector<double> tl_start, tl_end;  // per-op times of the last timed op list (ms from its start)
    std::vector<char*> host_dev;    // device mappings of the run's host arrays (zero-copy input)

    ~so2dr_plan_s();
    void unbind();
};

namespace so2dr {

int set_error(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
int check_pinned(const void* p, const char* what);
double wait_timeout_s();
int bounded_wait(const std::vector<cudaEvent_t>& evs, double timeout_s);

// Enqueues a kernel op (non-stencil programs of the adjoint pipeline).
using KernelHook = std::function<int(so2dr_plan_s*, const RunList&, const Op&, cudaStream_t)>;

int enqueue_stencil(so2dr_plan_s* P, const RunList& rl, const Op& op, cudaStream_t s);

// Replays an op list.  hosts[i] is the base of host array i, host_plane_bytes[i]
// its bytes per plane and host_field_bytes[i] the bytes between its fields.
int execute(so2dr_plan_s* P, const RunList& rl, char* const* hosts, const int64_t* host_plane_bytes,
            const int64_t* host_field_bytes, so2dr_stats_t* stats, const KernelHook& hook);

size_t adjoint_workspace_bytes(const Plan& p);

// so2dr_plan_ex with search controls (pinned buffer options, candidate list).
int plan_create(so2dr_plan_t* out, int ndim, const int64_t* dims, int radius, int kind, const double* coeffs,
                int ncoeffs, int64_t time_steps, int min_chunks, int k_on, int k_off, size_t device_budget_bytes,
                int storage, double link_h2d_gbs, double link_d2h_gbs, double hbm_gbs, const PlanSearch* search);

}  // namespace so2dr
