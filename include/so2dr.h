/*
 * so2dr.h -- C ABI of the SO2DR out-of-core stencil engine for one GB300.
 *
 * SO2DR (synergy between on- and off-chip data reuse; paper Sec. IV) runs n
 * iterations of a stencil over a grid that lives in pinned host memory.  The
 * grid is cut into d chunks along axis 0 (Sec. II-A, Fig. 1b).  Every round of
 * k_off time steps (Algorithm 1) sends each chunk to the GPU once, runs
 * k_off steps on it with k_on-step on-chip temporal-blocking kernels
 * (Sec. IV-A), and sends the chunk back.  Chunks overlap by the halo of the
 * round; the overlap is shared on the device (off-chip region sharing, Sec.
 * II-B, Fig. 2) and both neighbours compute it (redundant off-chip
 * computation, Sec. IV-B, Fig. 4), so no kernel waits on a neighbour.
 *
 * What one time step computes (Sec. II-A; the method only reorganises it):
 *   interior I = { p : r <= p_a < n_a - r for every axis a }
 *   u'[p] = sum_o c_o u[p + o]   for p in I;   u'[p] = u[p] otherwise.
 * The boundary ring of width r is a fixed Dirichlet boundary.
 *
 * Conventions
 *  - Grids are row-major, axis 0 slowest; ndim is 2 or 3.  A "plane" is one
 *    index of axis 0 (a row in 2D).  The chunk axis is axis 0.
 *  - All functions return SO2DR_OK (0) or a negative SO2DR_E_* code.  Nothing
 *    aborts or prints.  so2dr_strerror() names a code; so2dr_last_error()
 *    gives a one-line detail for the calling thread.
 *  - Host grids are owned by the caller and must stay valid (and, for the
 *    bandwidth the engine is built for, be pinned: cudaHostAlloc /
 *    cudaHostRegister / torch pin_memory) until the call returns.  The library
 *    never frees or reallocates them.  Calls are synchronous: every stream the
 *    call used is joined (with a bounded wait) before it returns.
 *  - Device memory and streams are owned by the caller and lent to a plan by
 *    so2dr_bind().  The library carves the arena; it allocates no device
 *    memory of its own.  It creates CUDA events (no memory) at bind time.
 *  - One plan is used by one host thread at a time.
 *  - Planes 0..r-1 and n0-r..n0-1 of axis 0 are never written by so2dr_run;
 *    boundary cells of the other axes are written back with their own,
 *    unchanged values.
 */
#ifndef SO2DR_H
#define SO2DR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define SO2DR_OK 0
#define SO2DR_E_INVAL (-1)        /* an argument is out of range or NULL        */
#define SO2DR_E_INFEASIBLE (-2)   /* no chunking fits the device budget/limits  */
#define SO2DR_E_NOT_BOUND (-3)    /* run before so2dr_bind, or arena too small  */
#define SO2DR_E_CUDA (-4)         /* a CUDA runtime call failed (see last_error)*/
#define SO2DR_E_TIMEOUT (-5)      /* a bounded wait on the device ran out       */
#define SO2DR_E_DEVICE_CHECK (-6) /* a kernel's own index/argument check failed */
#define SO2DR_E_NOMEM (-7)        /* host-side allocation failed                */
#define SO2DR_E_NOT_PINNED (-8)   /* a host buffer is not page-locked           */
#define SO2DR_E_UNSUPPORTED (-9)  /* valid request this build does not provide  */

/* ------------------------------------------------------------------ enums */
typedef enum { SO2DR_F64 = 0, SO2DR_F32 = 1, SO2DR_BF16 = 2, SO2DR_F16 = 3 } so2dr_dtype;

/*
 * Stencil kinds (Fig. 1a shows star and box types) and the order of their
 * coefficient tables:
 *  SO2DR_STAR: 1 + 2*r*ndim weights.  Index 0 is the centre, then for each
 *      axis a = 0..ndim-1 and j = 1..r: the weight of offset -j*e_a, then of
 *      +j*e_a.
 *  SO2DR_BOX: (2r+1)^ndim weights for every offset o with |o_a| <= r,
 *      lexicographic with axis 0 slowest, each component running -r..r.
 *  SO2DR_VARCOEF_STAR: radius 1, ndim 3, no table.  Six caller-supplied face
 *      fields c_f (f = 2a: offset -e_a; f = 2a+1: offset +e_a), each a full
 *      grid of the storage dtype's compute type (FP32, or FP64 for F64
 *      storage), laid out [6][n0][n1][n2].  The centre weight is
 *      1 - sum_f c_f[p], formed per cell in the compute type.
 * Weights are rounded once to the compute type: FP64 for F64 storage, FP32
 * otherwise.  Storage in BF16/F16 is converted to FP32 on load and rounded
 * (nearest even) only when a kernel stores its result.
 */
typedef enum { SO2DR_STAR = 0, SO2DR_BOX = 1, SO2DR_VARCOEF_STAR = 2 } so2dr_kind;

typedef struct so2dr_plan_s* so2dr_plan_t; /* opaque; library-owned host memory */

/* Filled by so2dr_plan_info(); every field is a property of the plan. */
typedef struct {
    int ndim;
    int64_t dims[3];
    int radius;
    int kind;
    int dtype;
    int64_t time_steps;      /* n in Algorithm 1                                    */
    int k_off;               /* TB steps per round in device memory (S_TB)          */
    int k_on;                /* steps fused in one kernel launch                    */
    int rounds;              /* N_t = ceil(n / k_off)                               */
    int chunks;              /* d                                                   */
    int n_streams;           /* 4: host-to-device, compute x2, device-to-host       */
    int64_t max_chunk_planes;/* largest chunk (owned planes)                        */
    int64_t ring_planes;     /* capacity of the circular region-sharing buffer      */
    int64_t plane_bytes;     /* bytes of one stored plane                           */
    size_t arena_bytes;      /* device bytes so2dr_bind must lend (out-of-core)     */
    size_t arena_bytes_in_core; /* device bytes the in-core mode needs              */
    size_t host_workspace_bytes; /* pinned host bytes so2dr_adjoint/so2dr_loss need */
    int64_t ops_per_run;     /* copies + launches one out-of-core run enqueues      */
    int64_t launches_per_run;
    double h2d_bytes_per_run;
    double d2h_bytes_per_run;
    double cell_updates_per_run; /* interior cells x time steps                    */
    double redundancy;       /* computed / useful cell updates - 1 (trapezoids)     */
    int lookahead;           /* 1: the circular buffer also holds the next chunk's new
                                planes, so transfers run a chunk ahead of the kernels */
    int out_slabs;           /* output slabs (2: a chunk's device-to-host copy overlaps
                                the next chunk's last launch)                        */
    size_t arena_bytes_result_reuse; /* arena of mode 2 of so2dr_run (0: unavailable) */
    int result_reuse_chunks; /* chunks mode 2 uses                                  */
    int zero_copy;           /* 1: mode 3 of so2dr_run (zero-copy input) is available */
} so2dr_plan_info_t;

/* Filled by so2dr_run / so2dr_adjoint when the caller passes a non-NULL pointer. */
typedef struct {
    double total_ms;     /* first enqueue to last completion, CUDA events          */
    double kernel_ms;    /* sum of kernel durations (event pairs per launch; in
                            mode 2 also the on-device region-sharing copies)     */
    double h2d_ms;       /* sum of host-to-device copy durations                   */
    double d2h_ms;       /* sum of device-to-host copy durations                   */
    double h2d_bytes;
    double d2h_bytes;
    int64_t launches;
    int64_t ops;
    double gcells_per_s; /* cell_updates / total_ms                                */
    double main_kernel_ms;      /* sum of durations of the k_on-deep launches (depth
                                   1 in the result-reuse code, mode 2)              */
    int64_t main_kernel_launches;
    double main_kernel_cells;   /* owned (useful) cells those launches produced     */
} so2dr_stats_t;

/*
 * One entry of a plan's operation list (host-only introspection, used by the
 * CPU schedule emulator in the tests).  Buffers: id -1 is the host array, ids
 * >= 0 are regions of the arena (see so2dr_plan_buffers).  A buffer access
 * covers grid planes [z_lo, z_hi); plane z sits in slot (slot0 + z - z_lo)
 * modulo the buffer's capacity.
 */
typedef struct {
    int kind;        /* 0 host-to-device copy, 1 kernel launch, 2 device-to-host copy,
                        3 on-device copy (region sharing of the result-reuse code)   */
    int stream;      /* 0 host-to-device, 1 compute (even chunks), 2 device-to-host,
                        3 compute (odd chunks)                                        */
    int round;
    int chunk;
    int depth;       /* kernels: fused time steps                                     */
    int edge_lo;     /* kernels: input starts at plane 0 (fixed bottom boundary)      */
    int edge_hi;     /* kernels: input ends at plane n0 (fixed top boundary)          */
    int src_buf;     /* copies: source buffer; kernels: input buffer                  */
    int dst_buf;     /* copies: destination buffer; kernels: output buffer            */
    int64_t src_lo, src_hi, src_slot0; /* planes read and where plane src_lo sits     */
    int64_t dst_lo, dst_hi, dst_slot0; /* planes written and where dst_lo sits        */
    int64_t wait_op[4];/* per stream: index of the latest op of that stream this op
                          must wait for (-1 none); same-stream order is implicit     */
} so2dr_op_t;

typedef struct {
    int64_t offset_bytes;  /* from the arena base                                   */
    int64_t capacity_planes;
} so2dr_buffer_t;

/*
 * Environment variables the library reads:
 *   SO2DR_TIMEOUT_S       limit of every bounded wait on the device, seconds
 *                         (default 600); past it a call returns
 *                         SO2DR_E_TIMEOUT instead of waiting on.
 *   SO2DR_LOOKAHEAD=0|1   pin the planner's look-ahead option (default: the
 *   SO2DR_NOUT=1|2        cost model chooses); likewise the output slabs.
 *   SO2DR_GENERIC_KERNEL  any value: launch the generic temporal-blocking
 *                         kernel even where a register-streaming one exists
 *                         (same per-cell summation order, same results).
 *   SO2DR_ALLOW_PAGEABLE  any value: skip the page-locked check on host
 *                         grids (copies from pageable memory are staged by
 *                         the driver and run slower).
 *   SO2DR_ADJOINT_STEPS=K backward steps per adjoint round (or the largest
 *                         K below it that fits the arena; default: chosen).
 *   SO2DR_WORK_SPLIT      how a 3D star launch spreads over the SMs (default:
 *                         chosen per launch): grid = one tile and axis-0
 *                         segment per CTA; rounds = one CTA per SM slot
 *                         taking (tile, segment) units in rounds; waves = the
 *                         grid split with segments counted in waves of
 *                         resident CTAs.  Results are the same bytes.
 * A kernel whose bounded wait for a staged plane gives up (after about two
 * seconds) sets the run list's device status word; so2dr_run then returns
 * SO2DR_E_TIMEOUT.
 */

/* ---------------------------------------------------------------- planning */

/*
 * Builds a plan (host only; no CUDA call).  Algorithm 1 takes d, n, k_off
 * and k_on as its inputs; Table I adds the sizes and the device capacity.
 *   ndim, dims     grid extents (ndim 2 or 3), boundary ring included.
 *   radius, kind   stencil radius r (1..4) and kind (see so2dr_kind).
 *   coeffs, ncoeffs constant-coefficient table (NULL/0 for VARCOEF_STAR).
 *   time_steps     n >= 0.
 *   min_chunks     lower bound on d (>= 1); the planner raises d until every
 *                  buffer fits device_budget_bytes (so2dr_plan_info reports
 *                  the chosen d).
 *   k_on           steps fused per launch (1..16), 0 = choose.
 *   k_off          steps per round (>= 1), 0 = choose from the cost model
 *                  (among the candidates predicted within 2% of the best, the
 *                  one with the fewest rounds; see so2dr_plan_candidates).
 *   device_budget_bytes  every device byte the out-of-core pipeline uses.
 *   storage        grid storage dtype.
 * Returns SO2DR_E_INFEASIBLE when no chunking fits the budget.
 */
int so2dr_plan(so2dr_plan_t* out, int ndim, const int64_t* dims, int radius, int kind,
               const double* coeffs, int ncoeffs, int64_t time_steps, int min_chunks,
               int k_on, int k_off, size_t device_budget_bytes, int storage);

/* Same, with the two link bandwidths (GB/s) and the HBM bandwidth the cost
 * model uses to pick k_off and k_on (the model of Sec. III). */
int so2dr_plan_ex(so2dr_plan_t* out, int ndim, const int64_t* dims, int radius, int kind,
                  const double* coeffs, int ncoeffs, int64_t time_steps, int min_chunks,
                  int k_on, int k_off, size_t device_budget_bytes, int storage,
                  double link_h2d_gbs, double link_d2h_gbs, double hbm_gbs);

int so2dr_plan_info(so2dr_plan_t plan, so2dr_plan_info_t* info);

/* Chunk c owns planes [starts[c], starts[c+1]) of axis 0; starts has chunks+1
 * entries and covers [0, n0). */
int so2dr_plan_chunks(so2dr_plan_t plan, int64_t* starts, int max_entries);

/* Operation list of one run (mode 0/1/2 as in so2dr_run) in enqueue order.
 * With ops NULL the call only reports the count in *n_ops. */
int so2dr_plan_ops(so2dr_plan_t plan, int in_core, so2dr_op_t* ops, int64_t max_ops,
                   int64_t* n_ops);

/* Arena regions used by the op list of one run (mode 0/1/2). */
int so2dr_plan_buffers(so2dr_plan_t plan, int in_core, so2dr_buffer_t* bufs, int max_bufs,
                       int* n_bufs);

/*
 * One point of the run-time parameter search (Sec. IV-C chooses d, k_off and
 * k_on so that kernel time and transfer time balance under the device
 * capacity; Sec. V-B's Fig. 5 measures that trade-off).
 */
typedef struct {
    int k_off;           /* steps per round                                      */
    int k_on;            /* steps fused per launch                               */
    int chunks;          /* d: the fewest chunks whose buffers fit the budget    */
    int lookahead;       /* circular buffer also holds the next chunk's planes   */
    int out_slabs;       /* output slabs (1 or 2)                                */
    int status;          /* SO2DR_OK, or why the candidate could not be timed    */
    double predicted_ms; /* cost model's time of one run                         */
    double measured_ms;  /* least measured time of one run; -1 if not timed      */
} so2dr_tune_entry_t;

/*
 * Every feasible (k_off, k_on, look-ahead, output slabs) point of the
 * planner's search for this problem, with its chunk count and predicted time,
 * sorted by predicted time (host only; no CUDA call).  Arguments as in
 * so2dr_plan_ex; k_on or k_off non-zero pins that parameter.  Writes at most
 * table_cap entries; *table_len receives how many exist.
 */
int so2dr_plan_candidates(int ndim, const int64_t* dims, int radius, int kind, const double* coeffs,
                          int ncoeffs, int64_t time_steps, int min_chunks, int k_on, int k_off,
                          size_t device_budget_bytes, int storage, double link_h2d_gbs,
                          double link_d2h_gbs, double hbm_gbs, so2dr_tune_entry_t* table,
                          int table_cap, int* table_len);

/*
 * Builds the plan of one table entry (its k_off, k_on, chunks, lookahead and
 * out_slabs; host only).  Returns SO2DR_E_INFEASIBLE if it does not fit the
 * budget.
 */
int so2dr_plan_tuned(so2dr_plan_t* out, int ndim, const int64_t* dims, int radius, int kind,
                     const double* coeffs, int ncoeffs, int64_t time_steps,
                     const so2dr_tune_entry_t* entry, size_t device_budget_bytes, int storage);

/* ------------------------------------------------------------- execution */

/*
 * Lends device memory and streams to the plan.  Sec. IV-C fixes three streams
 * so that transfers in both directions overlap kernel execution; here the
 * streams are host-to-device, compute, device-to-host and a second compute
 * stream that lets consecutive chunks' launches overlap.
 *   device_arena   caller-owned device memory of at least
 *                  so2dr_plan_info().arena_bytes (or arena_bytes_in_core for
 *                  in-core runs), 256-byte aligned.
 * *   cuda_streams   nstreams (3 or 4) cudaStream_t handles: host-to-device,
 *                  compute, device-to-host[, second compute].  NULL entries (and
 *                  the fourth stream when nstreams is 3) are created privately
 *                  and destroyed by so2dr_destroy.
 * Creates the plan's CUDA events on the current device.  Rebinding replaces
 * the previous binding.
 */
int so2dr_bind(so2dr_plan_t plan, void* device_arena, size_t arena_bytes,
               void* const* cuda_streams, int nstreams);

/*
 * Runs the plan's n time steps on host_grid in place (Algorithm 1).
 *   host_grid      caller-owned grid of the plan's dtype, dims[0]*dims[1]*dims[2]
 *                  elements, updated in place.
 *   host_coeff_fields  VARCOEF_STAR only: the six face fields (see so2dr_kind),
 *                  read-only; NULL otherwise.
 *   in_core        mode.  0: the out-of-core SO2DR pipeline (chunks, circular
 *                  region-sharing buffer, trapezoids).  1: the whole grid is
 *                  copied to the device once, the same launch-depth sequence
 *                  runs on it, and it is copied back (the in-core comparison
 *                  code of Sec. V-A); mode 0's result is bit-identical to it.
 *                  2: the redundancy-free out-of-core code the paper compares
 *                  against (result reuse, Sec. II-B Fig. 2b, Sec. V-A):
 *                  single-step launches, region sharing of intermediate
 *                  results before every step; same k_off rounds, its own
 *                  chunking (plan_info().result_reuse_chunks) and arena
 *                  (plan_info().arena_bytes_result_reuse); constant
 *                  coefficients only.
 *                  3: mode 0 with zero-copy input: no host-to-device copy
 *                  of the grid; the first launch of each chunk reads the
 *                  chunk's new planes from the pinned host grid through its
 *                  device mapping (cudaHostGetDevicePointer) and writes them
 *                  into the circular buffer, where the next chunk finds its
 *                  shared region (a GB300 option over NVLink-C2C, not in the
 *                  paper).  Same arena and result as mode 0; 3D constant-
 *                  coefficient stars with FP32/BF16/FP16 storage whose every
 *                  first launch runs the register-streaming kernel
 *                  (plan_info().zero_copy).
 *   stats          optional timings.
 */
int so2dr_run(so2dr_plan_t plan, void* host_grid, const void* host_coeff_fields, int in_core,
              so2dr_stats_t* stats);

/*
 * Timeline of the last run made with stats (tracing): for op j of the list
 * that run replayed (the order of so2dr_plan_ops for its mode; for
 * so2dr_adjoint and so2dr_loss, the last of their pipelines), the time its
 * stream reached it after its waits and the time it completed, in ms from the
 * run's start marker (CUDA events).  With both arrays NULL only *n_ops is
 * set; 0 ops before any timed run.
 */
int so2dr_run_timeline(so2dr_plan_t plan, double* start_ms, double* end_ms, int64_t max_ops, int64_t* n_ops);

/*
 * Measured autotune of the run-time parameters (Sec. IV-C's choice of d,
 * k_off and k_on, made by timing instead of by the model alone).
 *   1. Measures the host link (host-to-device and device-to-host copies of
 *      up to 1 GiB between scratch_host_grid and the arena, each alone, best
 *      of 3) and HBM (an on-device copy inside the arena); link_gbs receives
 *      {h2d, d2h, hbm} in GB/s (may be NULL).
 *   2. Ranks the candidates of so2dr_plan_candidates with those rates.
 *   3. Runs the best max_candidates of them (mode 0) on scratch_host_grid,
 *      each `repeats` times, with the given arena and streams.
 * scratch_host_grid is a pinned host grid of the problem's shape and dtype
 * whose contents are overwritten (the timings do not depend on its values);
 * device_arena must hold device_budget_bytes.  The table (at most table_cap
 * entries) is sorted by measured time, untimed entries last; build the
 * winner with so2dr_plan_tuned(table[0]).  Plain problems only (no
 * VARCOEF_STAR).  Synchronises the streams.
 */
int so2dr_autotune(int ndim, const int64_t* dims, int radius, int kind, const double* coeffs,
                   int ncoeffs, int64_t time_steps, int min_chunks, int k_on, int k_off,
                   size_t device_budget_bytes, int storage, void* device_arena,
                   void* const* cuda_streams, int nstreams, void* scratch_host_grid,
                   int max_candidates, int repeats, so2dr_tune_entry_t* table, int table_cap,
                   int* table_len, double* link_gbs);

/*
 * Host-link and HBM rates on the caller's buffers, in GB/s: the rates the
 * cost model of Sec. III balances, and the comparison of the copy engines
 * with SM-driven transfers over the mapped pinned buffer (on GB300 the
 * Grace-Blackwell C2C link; the zero-copy alternative to cudaMemcpyAsync).
 *   host_a, host_b  pinned host buffers of `bytes` each (contents overwritten).
 *   device_arena    device memory of 2 * bytes.
 *   bytes           transfer size, a multiple of 16, >= 1 MiB.
 *   sm_ctas         CTAs of the SM copy kernel (e.g. 64).
 *   repeats         timed transfers per figure (the best is kept), >= 1.
 *   out             9 rates: [0] copy-engine host-to-device, [1] copy-engine
 *                   device-to-host, [2] and [3] the same two at once (two
 *                   streams), [4] SM host-to-device, [5] SM device-to-host,
 *                   [6] and [7] the two SM directions at once, [8] HBM (an
 *                   on-device copy, read + write bytes).  SM figures are -1
 *                   when the host buffers have no device mapping.
 * Synchronises the device work it issues; uses its own streams.
 */
int so2dr_measure_link(void* host_a, void* host_b, void* device_arena, size_t bytes, int sm_ctas,
                       int repeats, double* out);

/*
 * Gradient of L = 1/2 ||u_T - u*||^2 (T = time_steps) for a VARCOEF_STAR plan,
 * through the same out-of-core pipeline: a forward sweep that keeps u every
 * checkpoint_every steps in host_workspace, then, segment by segment from the
 * last, recomputation of the segment's states (one round of single-step
 * launches that sends every state back) and the transposed stencil run
 * backward in time in rounds of K steps (K <= checkpoint_every, the largest
 * worth it under the budget; SO2DR_ADJOINT_STEPS pins it), accumulating
 * dL/dc_f of a round's K steps on the cells each chunk owns before it goes
 * back to the host.
 *   host_u0, host_coeff_fields, host_target   inputs (read-only).
 *   host_grad_u0     out: dL/du_0 for every cell (N elements, plan dtype).
 *   host_grad_coeffs out: dL/dc_f, [6][N] in the compute type; zero off I.
 *   host_workspace   pinned scratch of plan_info().host_workspace_bytes.
 *   loss_out         out: L, reduced in FP64 on the device.
 * Requires F32 or F64 storage.
 */
int so2dr_adjoint(so2dr_plan_t plan, const void* host_u0, const void* host_coeff_fields,
                  const void* host_target, void* host_grad_u0, void* host_grad_coeffs,
                  void* host_workspace, size_t workspace_bytes, int checkpoint_every,
                  double* loss_out, so2dr_stats_t* stats);

/* L = 1/2 ||u_T - u*||^2 only (forward sweep + FP64 device reduction).  The
 * workspace receives u_T (N elements). */
int so2dr_loss(so2dr_plan_t plan, const void* host_u0, const void* host_coeff_fields,
               const void* host_target, void* host_workspace, size_t workspace_bytes,
               double* loss_out);

/* FP64 inner product of two host arrays of n elements of dtype (F32 or F64),
 * streamed through the plan's arena and reduced on the device (used for the
 * finite-difference checks). */
int so2dr_dot(so2dr_plan_t plan, const void* host_a, const void* host_b, int64_t n, int dtype,
              double* out);

/*
 * Allocation-free in-core run (the paper has no counterpart: this entry point
 * exists for callers that cannot allocate memory -- code running while a CUDA
 * graph is captured, real-time loops that forbid allocation after start-up,
 * host runtimes that only hand out pre-registered device buffers).
 *
 * Runs `steps` time steps of a constant-coefficient star stencil (2D or 3D)
 * or 2D box stencil, of the given radius, coefficient table (see so2dr_kind)
 * and storage dtype, on a grid that is already on the device: d_in is read,
 * d_out receives the result (caller-owned device buffers of
 * dims[0]*dims[1](*dims[2]) elements, 16-byte aligned and not overlapping;
 * d_in is not modified).  The launches are floor(steps/k_on) launches of
 * depth k_on, then one of the remainder, on `stream` (a cudaStream_t; NULL =
 * the legacy default stream).  The call returns once the launches are queued;
 * it does not synchronise.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine, on the device
 * or the host.  Its one scratch grid lives in a file-scope device array of
 * 32 MiB that every GPU loading the library holds until the process exits.
 * Only runs of two or more launches use it: those are rejected with
 * SO2DR_E_INFEASIBLE when the grid is above 32 MiB (a run of one launch, or
 * of zero steps, takes any size).  The first such call on each device looks
 * up the array's device address (cudaGetSymbolAddress with the device
 * current) and caches it with the id of the current context; after a
 * cudaDeviceReset, or any re-creation of the device's primary context, the
 * next call looks it up again.  Make those calls before any stream capture.
 * Every call shares the array and leaves the last call's data in it (nothing
 * in it has to start at zero: each launch overwrites every cell it later
 * reads); calls whose work overlaps on the GPU race on it, so serialise them
 * (one stream, or events).
 */
int so2dr_run_device_noalloc(int ndim, const int64_t* dims, int radius, int kind, const double* coeffs,
                             int ncoeffs, int64_t steps, int k_on, int dtype, const void* d_in, void* d_out,
                             void* stream);

void so2dr_destroy(so2dr_plan_t plan);

const char* so2dr_strerror(int status);
const char* so2dr_last_error(void);

/* ABI version of this header (bumped on any incompatible change): 5. */
int so2dr_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SO2DR_H */
