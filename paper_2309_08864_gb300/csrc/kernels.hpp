// kernels.hpp -- host-side entry points of the device kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "so2dr.h"
#include "stencil.cuh"

namespace so2dr {

// Tiling and shared-memory size of a stencil launch for the plan's geometry.
struct LaunchShape {
    dim3 grid, block;
    size_t smem;
    int lx, ly, tx, ty;
    bool ok;
    int fast;    // 0 generic kernel, kFastStar3D (star3d_tb.cuh), kFastBox2D (box2d_fast.cuh)
};

constexpr int kFastStar3D = 1, kFastBox2D = 2;

// (R, K) pairs the register-streaming 3D star kernel is instantiated for.
bool fast_star3d_supported(int r, int depth);

// Whether the 3D star kernel can stage planes of this row length with TMA:
// rows must be a whole number of 16-byte units (nx % 4 == 0 for 4-byte
// storage, nx % 8 == 0 for 16-bit storage).
bool fast_star3d_row_ok(int64_t nx, int esize);

// TMA descriptor of a buffer of `cap` planes of ny x nx elements of `esize`
// bytes, with boxes of box_x columns x box_rows rows x 1 plane.  Host only.
cudaError_t encode_plane_map(CUtensorMap* map, int esize, const void* base, int64_t nx, int64_t ny, int64_t cap,
                             int box_x, int box_rows);

// (R, K) pairs the register-streaming 2D box kernel is instantiated for.
bool fast_box2d_supported(int r, int depth);

// csize: compute-type bytes; esize: storage-type bytes.
LaunchShape stencil_launch_shape(int shape, int r, int depth, int64_t ny, int64_t nx, int csize, int esize);

// Largest fused depth the stencil kernel supports for this geometry.
int stencil_max_depth(int shape, int r, int csize);

// Launches the temporal-blocking kernel.  Returns cudaSuccess or the error.
cudaError_t launch_stencil(int dtype, int shape, int r, const StencilArgs& a, const LaunchShape& ls,
                           cudaStream_t s);

// CTAs per SM of a launch shape (cudaOccupancyMaxActiveBlocksPerMultiprocessor).
int stencil_occupancy(int dtype, int shape, int r, int depth, const LaunchShape& ls);

// Axis-0 segments for a launch with `tiles` CTAs per segment, nout output
// planes and halo r*depth: the count that minimises the busiest SM's time.
// share_sm: the occ resident CTAs of an SM share its throughput, so the time
// goes with the CTAs the busiest SM receives times the planes each streams
// (the 3D star kernel, issue-bound); otherwise they run side by side and the
// time goes with the waves of sms * occ CTAs (the 2D box kernel, whose second
// resident CTA hides the first one's latency).
int choose_segments(int64_t tiles, int64_t nout, int r, int depth, int sms, int occ, bool share_sm);

// Work split of a 3D star kernel launch (ls.grid is tiles in x by tiles in
// y): either axis-0 segments per tile, one CTA each (choose_segments; *split
// = 0, grid.z = segments), or sms * occ CTAs (a 1D grid) that take the tiles
// x n (tile, segment) units in rounds, the units of the last, partial round
// cut into shorter axis-0 pieces (*split = n), whichever the cost model
// (busiest SM's CTAs times planes streamed, each piece paying the r * depth
// halo each side and the depth-deep pipeline fill) rates cheaper by 3%, with
// units of at most 384 planes.  SO2DR_WORK_SPLIT=grid|rounds pins the choice
// (waves: the grid split with segments counted in waves of resident CTAs).
void choose_work_split(LaunchShape& ls, int64_t nout, int r, int depth, int sms, int occ, int* split);

// Per-dtype instantiations (one translation unit each).
int occupancy_stencil_f64(int shape, int r, int depth, const LaunchShape& ls);
int occupancy_stencil_f32(int shape, int r, int depth, const LaunchShape& ls);
int occupancy_stencil_bf16(int shape, int r, int depth, const LaunchShape& ls);
int occupancy_stencil_f16(int shape, int r, int depth, const LaunchShape& ls);
cudaError_t launch_stencil_f64(int shape, int r, const StencilArgs& a, const LaunchShape& ls, cudaStream_t s);
cudaError_t launch_stencil_f32(int shape, int r, const StencilArgs& a, const LaunchShape& ls, cudaStream_t s);
cudaError_t launch_stencil_bf16(int shape, int r, const StencilArgs& a, const LaunchShape& ls, cudaStream_t s);
cudaError_t launch_stencil_f16(int shape, int r, const StencilArgs& a, const LaunchShape& ls, cudaStream_t s);

}  // namespace so2dr
