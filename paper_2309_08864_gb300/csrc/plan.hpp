// plan.hpp -- host-side plan of the SO2DR pipeline (no CUDA calls).
//
// A plan fixes the chunking along axis 0 (Sec. II-A, Fig. 1b), the rounds and
// launch-depth sequence of Algorithm 1, the arena layout and, for each run,
// the complete list of operations (copies and launches) with the cross-stream
// waits that make it race-free.  The executor (run.cu) only replays the list.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "so2dr.h"

namespace so2dr {

// streams: host-to-device, compute (even chunks), device-to-host, compute (odd chunks)
constexpr int kStreamH2D = 0, kStreamCompute = 1, kStreamD2H = 2, kStreamCompute2 = 3, kNumStreams = 4;
constexpr int kOpH2D = 0, kOpKernel = 1, kOpD2H = 2, kOpD2D = 3;
constexpr int kHost = -1;           // buffer id of the host array of a copy
constexpr int kMaxRadius = 4;
constexpr int kMaxKon = 16;
constexpr int kMaxCoeffs = 81;      // (2*4+1)^2 for the 2D box of radius 4

// Kernel programs an op can launch.
enum KernelFn : int {
    kFnStencil = 0,     // const-coefficient star/box, or varcoef forward
    kFnAdjoint = 1,     // transposed varcoef step + coefficient-gradient update
    kFnResidual = 2,    // lambda_T = u_T - u*, FP64 partial loss
    kFnDot = 3,         // FP64 partial inner products
    kFnReduce = 4,      // FP64 final sum of partials
    kFnZero = 5,        // clear a buffer region
};

// One operation, as enqueued.  Extends the public record with what the
// executor needs and the introspection API does not expose.
struct Op {
    so2dr_op_t pub;
    int fn = kFnStencil;
    int host_array = 0;     // copies: which host array (see the run's array table)
    int64_t field_elems = 0;// copies: element offset between fields (multi-field copies)
    int nfields = 1;        // copies: number of fields moved by this op
    int64_t buf_field_stride = 0; // copies/kernels: bytes between fields inside a buffer
    int aux_buf = -1;       // kernels: extra buffer (coefficients, states, gradients)
    int64_t aux_lo = 0, aux_slot0 = 0;
    int aux2_buf = -1;
    int64_t aux2_lo = 0, aux2_slot0 = 0;
    int aux3_buf = -1;
    int64_t aux3_lo = 0, aux3_slot0 = 0;
    int64_t arg0 = 0, arg1 = 0, arg2 = 0;  // kernel-specific integers
    int host_src = -1;      // zero-copy kernels: host array whose planes [host_lo, host_hi) they read
    int64_t host_lo = 0, host_hi = 0;
    bool waited = false;    // some later op waits on this op's completion event
};

struct Buffer {
    int64_t offset = 0;     // bytes from the arena base
    int64_t cap = 0;        // planes
    int64_t plane_bytes = 0;// bytes per plane (x fields)
    int nfields = 1;
};

// Interval access tracker used while emitting ops: finds, for each new op,
// the latest conflicting op of every other stream.
class Tracker {
public:
    explicit Tracker(int nres) : res_(nres) {}
    // Adds one access of the op being built; call for each access, then commit().
    void access(int res, int64_t lo, int64_t hi, bool write);
    // Fills wait_op[] for op index `op` on `stream`, records its accesses.
    void commit(int64_t op, int stream, int64_t wait_op[kNumStreams]);

private:
    struct Entry { int64_t lo, hi, op; int stream; bool write; };
    struct Pending { int res; int64_t lo, hi; bool write; };
    std::vector<std::vector<Entry>> res_;
    std::vector<Pending> pend_;
};

struct RunList {
    std::vector<Op> ops;
    std::vector<Buffer> bufs;
    size_t arena_bytes = 0;
};

struct Plan {
    // problem
    int ndim = 3;
    int64_t n0 = 0, ny = 1, nx = 1;   // axis 0, then the in-plane extents (ny = 1 in 2D)
    int r = 1, kind = SO2DR_STAR, dtype = SO2DR_F32;
    std::vector<double> coeffs;
    int64_t T = 0;
    // schedule
    int k_off = 1, k_on = 1, rounds = 0, d = 1;
    std::vector<int64_t> starts;      // d + 1 entries, partition of [0, n0)
    int64_t elem_bytes = 4, plane_cells = 0, plane_bytes = 0;
    size_t budget = 0;
    int64_t ring_planes = 0;
    // cost-model inputs
    double bw_h2d = 171.0, bw_d2h = 171.0, bw_hbm = 6781.0;
    // op lists of a forward run
    RunList ooc, ic;
    RunList rr;                       // redundancy-free comparison code (result reuse), if it fits
    int rr_chunks = 0;
    RunList zc;                       // zero-copy input (run mode 3), if the 3D star kernel runs every first launch
    bool zc_ok = false;
    double redundancy = 0.0;
    int max_kon = kMaxKon;            // deepest fused launch the kernels support
    int lookahead = 1;                // circular buffer holds the next chunk's new planes too (1) or not (0)
    int n_out = 2;                    // output slabs (2: D2H of a chunk overlaps the next chunk's last launch)
    int max_kon_auto = kMaxKon;       // deepest launch the automatic choice considers

    int64_t interior_planes() const { return n0 - 2 * r; }
    double cell_updates() const;
};

// One point of the planner's search: schedule parameters and the cost
// model's predicted time of a run.
struct Candidate {
    int k_off = 1, k_on = 1, d = 1, lookahead = 1, n_out = 2;
    double predicted_ms = 0.0;
};

// Search controls: pin the buffer options (-1 = choose; they override the
// SO2DR_LOOKAHEAD / SO2DR_NOUT variables) and, if `ranked` is set, collect
// every feasible candidate of the search (in search order).
struct PlanSearch {
    int lookahead = -1, n_out = -1;
    std::vector<Candidate>* ranked = nullptr;
};

// Builds a plan; returns SO2DR_OK or an error code (message in *err).
int build_plan(Plan& p, int ndim, const int64_t* dims, int radius, int kind, const double* coeffs,
               int ncoeffs, int64_t T, int min_chunks, int k_on, int k_off, size_t budget,
               int dtype, double bw_h2d, double bw_d2h, double bw_hbm, std::string* err,
               const PlanSearch* search = nullptr);

// Launch-depth sequence of a round of k steps with k_on-step kernels
// (Algorithm 1: floor(k/k_on) k_on-step launches, then one (k mod k_on)-step).
std::vector<int> launch_depths(int k, int k_on);

// Steps of round t (the last round runs n mod k_off when that is non-zero).
int round_steps(int64_t T, int k_off, int t);

int64_t elem_size(int dtype);
int num_coeffs(int ndim, int radius, int kind);

// Forward op list for the given chunking.  Fills rl; returns false if the
// buffers do not fit `budget` (budget 0 = unlimited).
bool build_forward_ooc(const Plan& p, RunList& rl, size_t budget);
void build_forward_in_core(const Plan& p, RunList& rl);

// The redundancy-free out-of-core code the paper compares against (result
// reuse, Sec. II-B Fig. 2b and Sec. V-A): single-step launches, each chunk a
// parallelogram that shifts down by r per step and reads, before every step,
// the previous chunk's top 2r planes of the previous step from a per-step
// region-sharing ring.  Returns false if it does not fit `budget`.
bool build_result_reuse(const Plan& p, RunList& rl, size_t budget, int* chunks_out);

// Options of a forward op list used inside the adjoint pipeline.
struct ForwardOpts {
    std::vector<int> src_array;  // host array each round reads (default: 0, in place)
    std::vector<int> dst_array;  // host array each round writes (default: 0)
    bool all_planes = false;     // write back the axis-0 boundary planes too
    int coef_array = 1;          // host array of the face fields
    // round 0 only, single-step launches: host array receiving the state after
    // launch j (j = 0 .. k'-2; the last state goes to dst_array[0])
    std::vector<int> state_array;
    // zero-copy input: no host-to-device copy of the grid; the first launch of
    // each chunk reads the chunk's new planes from the mapped host grid and
    // writes them into the circular buffer for the next chunk
    bool zero_copy = false;
};

// Forward op list with per-round source/destination host arrays.
bool build_forward_ooc_ex(const Plan& p, RunList& rl, size_t budget, const ForwardOpts& opt);

// Arena bytes of the forward op list for the plan's chunking.
size_t forward_arena_bytes(const Plan& p);

// Splits [0, n0) into d chunks (interior planes spread evenly).
void partition_planes(Plan& p);

// Arena bytes of the single-step adjoint rounds for q's chunking (adjoint.cu).
size_t adjoint_arena_bytes(const Plan& q);

// ------------------------------------------------------------- op helpers

constexpr int64_t kAlign = 256;
// the last kAlign bytes of a run list's arena: the device status word at 0,
// the round split's piece counters of the streams (two words each) from here
constexpr int64_t kWorkCtrOff = 16;
static_assert(kWorkCtrOff + 8 * kNumStreams <= kAlign, "status block layout");
inline int64_t align_up(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
inline int64_t floor_mod(int64_t a, int64_t m) { return ((a % m) + m) % m; }

// Physical slot ranges of grid planes [lo, hi) stored from slot0 in a buffer
// of capacity cap (split at the wrap).
inline void add_buf_access(Tracker& tr, int res, int64_t lo, int64_t hi, int64_t slot0, int64_t cap,
                           bool write) {
    int64_t n = hi - lo;
    if (n <= 0 || cap <= 0) return;
    int64_t s0 = floor_mod(slot0, cap);
    int64_t first = n < cap - s0 ? n : cap - s0;
    tr.access(res, s0, s0 + first, write);
    if (n > first) tr.access(res, 0, n - first, write);
}

// Appends ops to a RunList, computing each op's cross-stream waits.
// Resources: device buffers 0..nbuf-1, host arrays nbuf..nbuf+nhost-1.
struct Emitter {
    RunList& rl;
    Tracker tr;
    int host_res_base;
    Emitter(RunList& r, int nres, int host_base) : rl(r), tr(nres), host_res_base(host_base) {}
    int64_t emit(Op& op) {
        int64_t idx = (int64_t)rl.ops.size();
        tr.commit(idx, op.pub.stream, op.pub.wait_op);
        for (int s = 0; s < kNumStreams; ++s)
            if (op.pub.wait_op[s] >= 0) rl.ops[op.pub.wait_op[s]].waited = true;
        rl.ops.push_back(op);
        return idx;
    }
    int host_res(int arr) const { return host_res_base + arr; }
};

inline Op make_op(int kind, int stream, int round, int chunk) {
    Op op;
    so2dr_op_t& p = op.pub;
    p.kind = kind;
    p.stream = stream;
    p.round = round;
    p.chunk = chunk;
    p.depth = 0;
    p.edge_lo = p.edge_hi = 0;
    p.src_buf = p.dst_buf = kHost;
    p.src_lo = p.src_hi = p.src_slot0 = 0;
    p.dst_lo = p.dst_hi = p.dst_slot0 = 0;
    for (int s = 0; s < kNumStreams; ++s) p.wait_op[s] = -1;
    return op;
}

struct ChunkGeom {
    int64_t s, e;      // owned planes
    int64_t a, b;      // input planes of the round
    int64_t lo, hi;    // new planes sent this round
};

inline ChunkGeom chunk_geom(const Plan& p, int i, int kk) {
    ChunkGeom g;
    g.s = p.starts[i];
    g.e = p.starts[i + 1];
    int64_t h = (int64_t)p.r * kk;
    g.a = g.s - h > 0 ? g.s - h : 0;
    g.b = g.e + h < p.n0 ? g.e + h : p.n0;
    g.lo = (i == 0) ? 0 : (g.s + h < p.n0 ? g.s + h : p.n0);
    g.hi = (i == p.d - 1) ? p.n0 : (g.e + h < p.n0 ? g.e + h : p.n0);
    return g;
}

}  // namespace so2dr
