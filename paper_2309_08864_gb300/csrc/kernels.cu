// kernels.cu -- launch geometry and dtype dispatch of the stencil kernel.
#include "kernels.hpp"
#include "box2d_fast.cuh"
#include "star3d_tb.cuh"

#include <cmath>
#include <cstdlib>
#include <cstring>

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

bool fast_star3d_supported(int r, int depth) {
    return (r == 1 && depth >= 1 && depth <= 4) || (r >= 2 && r <= 4 && depth >= 1 && depth <= 2);
}

bool fast_star3d_row_ok(int64_t nx, int esize) { return nx % (esize == 4 ? 4 : 8) == 0; }

bool fast_box2d_supported(int r, int depth) {
    return depth >= 1 && ((r == 1 && depth <= 8) || (r == 2 && depth <= 4) || (r == 3 && depth <= 3) ||
                          (r == 4 && depth <= 2));
}

namespace {
template <int R, int K> void box_shape(LaunchShape& ls, int64_t nx, int esize) {
    using S = BoxShape<R, K>;
    ls.lx = S::LX;
    ls.ly = 1;
    ls.tx = S::TX;
    ls.ty = 1;
    ls.block = dim3(S::NT, 1, 1);
    ls.smem = esize == 4 ? S::template smem<4>() : S::template smem<2>();
    ls.grid = dim3((unsigned)((nx + S::TX - 1) / S::TX), 1, 1);
    ls.ok = true;
    ls.fast = kFastBox2D;
}

template <int R, int K> void fast_shape(LaunchShape& ls, int64_t ny, int64_t nx, int esize) {
    using S = StarShape<R, K>;
    ls.lx = S::LX;
    ls.ly = S::LYT;
    ls.tx = S::TX;
    ls.ty = S::TY;
    ls.block = dim3(S::NT, 1, 1);
    ls.smem = esize == 4 ? S::template smem<4>() : S::template smem<2>();
    ls.grid = dim3((unsigned)((nx + S::TX - 1) / S::TX), (unsigned)((ny + S::TY - 1) / S::TY), 1);
    ls.ok = ls.grid.y <= 65535;
    ls.fast = kFastStar3D;
}
}  // namespace

LaunchShape stencil_launch_shape(int shape, int r, int depth, int64_t ny, int64_t nx, int csize, int esize) {
    LaunchShape ls;
    ls.ok = false;
    ls.fast = 0;
    if (depth < 1) return ls;
    if (shape == kBox2D && csize == 4 && nx % 4 == 0 && fast_box2d_supported(r, depth) &&
        !std::getenv("SO2DR_GENERIC_KERNEL")) {
        switch (r * 16 + depth) {
            case 17: box_shape<1, 1>(ls, nx, esize); break;
            case 18: box_shape<1, 2>(ls, nx, esize); break;
            case 19: box_shape<1, 3>(ls, nx, esize); break;
            case 20: box_shape<1, 4>(ls, nx, esize); break;
            case 21: box_shape<1, 5>(ls, nx, esize); break;
            case 22: box_shape<1, 6>(ls, nx, esize); break;
            case 23: box_shape<1, 7>(ls, nx, esize); break;
            case 24: box_shape<1, 8>(ls, nx, esize); break;
            case 33: box_shape<2, 1>(ls, nx, esize); break;
            case 34: box_shape<2, 2>(ls, nx, esize); break;
            case 35: box_shape<2, 3>(ls, nx, esize); break;
            case 36: box_shape<2, 4>(ls, nx, esize); break;
            case 49: box_shape<3, 1>(ls, nx, esize); break;
            case 50: box_shape<3, 2>(ls, nx, esize); break;
            case 51: box_shape<3, 3>(ls, nx, esize); break;
            case 65: box_shape<4, 1>(ls, nx, esize); break;
            case 66: box_shape<4, 2>(ls, nx, esize); break;
        }
        if (ls.ok) return ls;
    }
    if (shape == kStar3D && csize == 4 && fast_star3d_row_ok(nx, esize) && fast_star3d_supported(r, depth) &&
        !std::getenv("SO2DR_GENERIC_KERNEL")) {
        switch (r * 16 + depth) {
            case 17: fast_shape<1, 1>(ls, ny, nx, esize); break;
            case 18: fast_shape<1, 2>(ls, ny, nx, esize); break;
            case 19: fast_shape<1, 3>(ls, ny, nx, esize); break;
            case 20: fast_shape<1, 4>(ls, ny, nx, esize); break;
            case 33: fast_shape<2, 1>(ls, ny, nx, esize); break;
            case 34: fast_shape<2, 2>(ls, ny, nx, esize); break;
            case 49: fast_shape<3, 1>(ls, ny, nx, esize); break;
            case 50: fast_shape<3, 2>(ls, ny, nx, esize); break;
            case 65: fast_shape<4, 1>(ls, ny, nx, esize); break;
            case 66: fast_shape<4, 2>(ls, ny, nx, esize); break;
        }
        if (ls.ok) return ls;
    }
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
        LaunchShape ls = stencil_launch_shape(shape, r, d, 1024, 1024, csize, csize);
        if (ls.ok) best = d;
    }
    return best;
}

int stencil_occupancy(int dtype, int shape, int r, int depth, const LaunchShape& ls) {
    switch (dtype) {
        case SO2DR_F64: return occupancy_stencil_f64(shape, r, depth, ls);
        case SO2DR_F32: return occupancy_stencil_f32(shape, r, depth, ls);
        case SO2DR_BF16: return occupancy_stencil_bf16(shape, r, depth, ls);
        case SO2DR_F16: return occupancy_stencil_f16(shape, r, depth, ls);
        default: return 1;
    }
}

int choose_segments(int64_t tiles, int64_t nout, int r, int depth, int sms, int occ, bool share_sm) {
    if (tiles <= 0 || nout <= 0 || sms <= 0) return 1;
    const int64_t slots = (int64_t)sms * (share_sm || occ < 1 ? 1 : occ);
    int best = 1;
    double best_cost = 0;
    for (int n = 1; n <= 64 && n <= nout; ++n) {
        // share_sm: the CTAs resident on one SM share its throughput, so an
        // SM's time goes with the CTAs it receives (the busiest SM gets
        // ceil(tiles * n / sms)) times the planes each streams; otherwise the
        // occ resident CTAs of an SM run side by side, and the time goes with
        // the waves of sms * occ CTAs
        int64_t per_slot = (tiles * n + slots - 1) / slots;
        double len = (double)nout / n + 2.0 * r * depth + depth;
        double cost = (double)per_slot * len;
        if (n == 1 || cost < best_cost * 0.98) { best = n; best_cost = cost; }
    }
    return best;
}

// longest unit of the round split (planes; measured on GB300: units of 1024
// planes ran 1-5% slower than the grid split at fused depths 1-3, units of
// 341 planes 5% faster at depth 4)
constexpr double kMaxUnit = 384;

void choose_work_split(LaunchShape& ls, int64_t nout, int r, int depth, int sms, int occ, int* split) {
    *split = 0;
    const int64_t tiles = (int64_t)ls.grid.x * ls.grid.y;
    if (tiles <= 0 || nout <= 0 || sms <= 0) return;
    const char* pin = std::getenv("SO2DR_WORK_SPLIT");
    // grid split: segments by the shared-SM model, or by waves of resident
    // CTAs (SO2DR_WORK_SPLIT=waves)
    const bool waves = pin && std::strcmp(pin, "waves") == 0;
    const int nseg = choose_segments(tiles, nout, r, depth, sms, occ, !waves);
    const double ovh = 2.0 * r * depth + depth;
    const double cost_grid = (double)((tiles * nseg + sms - 1) / sms) * ((double)nout / nseg + ovh);
    // round split: G = sms * occ CTAs take the tiles x n units in rounds;
    // each unit of the last, partial round is cut into floor(G / rem) pieces
    const int64_t occ1 = occ > 0 ? occ : 1, G = (int64_t)sms * occ1;
    int best_n = 0;
    double best = 0;
    for (int n = 1; n <= 64 && n <= nout; ++n) {
        const int64_t units = tiles * n, F = units / G, rem = units - F * G;
        const double len = std::ceil((double)nout / n);
        // units of more than kMaxUnit planes let neighbouring CTAs drift
        // apart along axis 0, and the halo rows they share then miss in L2
        if (len > kMaxUnit && n < nout) continue;
        double cost = (double)F * (len + ovh);
        if (rem) cost += std::ceil(len / (double)(G / rem)) + ovh;
        cost *= (double)occ1;
        if (best_n == 0 || cost < best * 0.98) { best_n = n; best = cost; }
    }
    bool rounds = best_n > 0 && best < cost_grid * 0.97;
    if (pin && (std::strcmp(pin, "grid") == 0 || waves)) rounds = false;
    if (pin && std::strcmp(pin, "rounds") == 0) rounds = true;
    if (rounds) {
        ls.grid = dim3((unsigned)G, 1, 1);
        *split = best_n;
    } else {
        ls.grid.z = (unsigned)nseg;
    }
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
