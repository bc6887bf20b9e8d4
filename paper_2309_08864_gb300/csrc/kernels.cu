// kernels.cu -- launch geometry and dtype dispatch of the stencil kernel.
#include "kernels.hpp"

namespace so2dr {

namespace {
constexpr int64_t kSmemLimit = 200 * 1024;

bool is3d(int shape) { return shape == kStar3D || shape == kVarcoef3D; }

// Loaded-tile edge for an in-plane halo H: at least 32 and at least 2H + 16.
int tile_edge(int H) {
    int e = 2 * H + 16;
    if (e < 32) e = 32;
    return (e + 7) / 8 * 8;
}
}  // namespace

LaunchShape stencil_launch_shape(int shape, int r, int depth, int64_t ny, int64_t nx, int csize) {
    LaunchShape ls;
    ls.ok = false;
    if (depth < 1) return ls;
    int H = r * depth;
    if (is3d(shape)) {
        ls.lx = ls.ly = tile_edge(H);
        ls.tx = ls.lx - 2 * H;
        ls.ty = ls.ly - 2 * H;
        ls.block = dim3(32, 8, 1);
    } else {
        ls.lx = 256;
        while (ls.lx - 2 * H < 64) ls.lx += 128;
        ls.ly = 1;
        ls.tx = ls.lx - 2 * H;
        ls.ty = 1;
        ls.block = dim3(256, 1, 1);
    }
    ls.smem = (size_t)stencil_smem_bytes(shape, r, depth, ls.lx, ls.ly, csize);
    if ((int64_t)ls.smem > kSmemLimit) return ls;
    int64_t gx = (nx + ls.tx - 1) / ls.tx;
    int64_t gy = is3d(shape) ? (ny + ls.ty - 1) / ls.ty : 1;
    if (gx > 2147483647 || gy > 65535) return ls;
    ls.grid = dim3((unsigned)gx, (unsigned)gy, 1);
    ls.ok = true;
    return ls;
}

int stencil_max_depth(int shape, int r, int csize) {
    int best = 0;
    for (int d = 1; d <= 16; ++d) {
        LaunchShape ls = stencil_launch_shape(shape, r, d, 1024, 1024, csize);
        if (ls.ok) best = d;
    }
    return best;
}

cudaError_t launch_stencil(int dtype, int shape, int r, const StencilArgs& a, const LaunchShape& ls,
                           cudaStream_t s) {
    switch (dtype) {
        case SO2DR_F64: return launch_stencil_f64(shape, r, a, ls, s);
        case SO2DR_F32: return launch_stencil_f32(shape, r, a, ls, s);
        case SO2DR_BF16: return launch_stencil_bf16(shape, r, a, ls, s);
        case SO2DR_F16: return launch_stencil_f16(shape, r, a, ls, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace so2dr
