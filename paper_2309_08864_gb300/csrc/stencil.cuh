// stencil.cuh -- k_on-step on-chip temporal-blocking stencil kernel (sm_103a).
//
// One launch advances a slab of planes (axis 0) by `depth` time steps without
// going back to device memory between them (on-chip data reuse, Sec. III and
// Sec. IV-A; the paper's kernels fuse 4 steps).  Each CTA owns a tile of the
// plane (axes 1, 2) plus an in-plane halo of r*depth cells and streams along
// axis 0: a plane is read from device memory once, every fused level keeps a
// (2r+1)-plane window of its own results in shared memory, and only the last
// level is stored.  The computed area shrinks by r per level in every
// direction that is not a domain edge (the compute-area adjustment of
// Algorithm 1, applied inside the launch as well as between launches).
//
// Arithmetic order is fixed per cell (explicit FMAs in coefficient-table
// order), so every chunking and tiling of a plan produces the same bits.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>

namespace so2dr {

constexpr int kMaxCoeffsDev = 81;

struct StencilArgs {
    // input: planes [in_lo, in_hi); plane z sits in slot (in_slot0 + z - in_lo) % in_cap
    const void* in;
    int64_t in_cap, in_slot0, in_lo, in_hi;
    // output: planes [out_lo, out_hi); plane z sits in slot z - out_lo
    void* out;
    int64_t out_lo, out_hi;
    // variable-coefficient face fields: field f, plane z at
    // coef + f * coef_field_stride + ((coef_slot0 + z - coef_lo) % coef_cap) * plane
    const void* coef;
    int64_t coef_cap, coef_slot0, coef_lo, coef_field_stride;
    // grid
    int64_t n0, ny, nx;   // ny = 1 for 2D grids
    int depth;
    int edge_lo, edge_hi; // input starts at plane 0 / ends at plane n0
    // tiling (chosen by the host)
    int lx, ly;           // loaded tile, halo included
    int tx, ty;           // output tile
    int* status;          // device status word (index checks)
    double c[kMaxCoeffsDev];
    float cf[kMaxCoeffsDev];   // the same weights rounded once to FP32
    float2 cf2[kMaxCoeffsDev]; // (cf, cf) pairs for packed FP32x2 FMAs
    // zero-copy input (3D star kernel): planes [host_lo, host_hi) are read
    // from host_in (mapped pinned host memory, plane z at host_in + z * plane)
    // instead of the input buffer, and written into the input buffer for the
    // launches that read them later
    const void* host_in;
    int64_t host_lo, host_hi;
    // 3D star kernel work split: 0 = one tile and axis-0 segment per CTA
    // (grid: tiles in x, tiles in y, segments); n > 0 = gridDim.x CTAs take
    // the tiles x n (tile, segment) units in rounds (the last round's units
    // cut shorter along axis 0)
    int split;
    // round split: {next piece, finished CTAs}, zero at launch; the CTAs take
    // pieces in order from this counter (null: CTA c takes pieces c, c + G, ...)
    // and the last CTA to finish zeroes both for the next launch on the stream
    unsigned* work_ctr;
};

template <typename T> struct Compute { using type = float; };
template <> struct Compute<double> { using type = double; };

template <typename T, typename C> __device__ __forceinline__ C load_as(const T* p) { return (C)(*p); }
template <> __device__ __forceinline__ float load_as<__nv_bfloat16, float>(const __nv_bfloat16* p) {
    return __bfloat162float(*p);
}
template <> __device__ __forceinline__ float load_as<__half, float>(const __half* p) { return __half2float(*p); }

template <typename T, typename C> __device__ __forceinline__ void store_as(T* p, C v) { *p = (T)v; }
template <> __device__ __forceinline__ void store_as<__nv_bfloat16, float>(__nv_bfloat16* p, float v) {
    *p = __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ void store_as<__half, float>(__half* p, float v) { *p = __float2half_rn(v); }

__device__ __forceinline__ float fma_c(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_c(double a, double b, double c) { return __fma_rn(a, b, c); }

enum StencilShape : int { kStar3D = 0, kStar2D = 1, kBox2D = 2, kVarcoef3D = 3 };

// Shared-memory bytes of one launch.
inline int64_t stencil_smem_bytes(int shape, int r, int depth, int lx, int ly, int csize) {
    (void)shape;
    return (int64_t)depth * (2 * r + 1) * lx * ly * csize;
}

template <typename T, int R, int SHAPE>
__global__ void __launch_bounds__(256) stencil_tb_kernel(const StencilArgs a) {
    using C = typename Compute<T>::type;
    constexpr int W = 2 * R + 1;
    extern __shared__ unsigned char smem_raw[];
    C* win = reinterpret_cast<C*>(smem_raw);  // [depth][W][ly][lx]

    const int lx = a.lx, ly = a.ly;
    const int64_t plane = a.ny * a.nx;
    const int64_t tile_cells = (int64_t)lx * ly;
    const int H = R * a.depth;
    const int64_t x0 = (int64_t)blockIdx.x * a.tx;  // output tile origin
    const int64_t y0 = (int64_t)blockIdx.y * a.ty;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthr = blockDim.x * blockDim.y;
    const T* in = static_cast<const T*>(a.in);
    T* out = static_cast<T*>(a.out);
    const C* coef = static_cast<const C*>(a.coef);

    C cst[SHAPE == kVarcoef3D ? 1 : (SHAPE == kBox2D ? W * W : (SHAPE == kStar2D ? 1 + 4 * R : 1 + 6 * R))];
#pragma unroll
    for (int k = 0; k < (int)(sizeof(cst) / sizeof(C)); ++k) cst[k] = (C)a.c[k];

    // axis-0 segment of this CTA (gridDim.z segments): outputs [zs, ze),
    // streamed over [za, zb), the outputs and the R*depth planes each side
    // (clipped to the launch's input; a clipped end keeps the launch's own
    // rule for which planes each level computes)
    const int64_t nout = a.out_hi - a.out_lo;
    const int64_t zs = a.out_lo + nout * blockIdx.z / gridDim.z;
    const int64_t ze = a.out_lo + nout * (blockIdx.z + 1) / gridDim.z;
    const int64_t za = zs - H > a.in_lo ? zs - H : a.in_lo;
    const int64_t zb = ze + H < a.in_hi ? ze + H : a.in_hi;
    const int64_t nsteps = (zb - za) + (int64_t)R * a.depth;
    for (int64_t s = 0; s < nsteps; ++s) {
        // ---- level 0: load input plane z0 into window 0
        const int64_t z0 = za + s;
        if (z0 < zb) {
            int64_t slot = (a.in_slot0 + (z0 - a.in_lo)) % a.in_cap;
            const T* src = in + slot * plane;
            C* w0 = win + ((z0 - a.in_lo) % W) * tile_cells;
            for (int64_t i = tid; i < tile_cells; i += nthr) {
                int ly_ = (int)(i / lx), lx_ = (int)(i % lx);
                int64_t gy = y0 - (SHAPE == kStar3D || SHAPE == kVarcoef3D ? H : 0) + ly_;
                int64_t gx = x0 - H + lx_;
                C v = (C)0;
                if (gy >= 0 && gy < a.ny && gx >= 0 && gx < a.nx) v = load_as<T, C>(src + gy * a.nx + gx);
                w0[i] = v;
            }
        }
        __syncthreads();
        // ---- fused levels 1..depth
        for (int l = 1; l <= a.depth; ++l) {
            const int64_t z = za + s - (int64_t)l * R;
            const int64_t lo_l = za > a.in_lo ? za + (int64_t)l * R : (a.edge_lo ? 0 : a.in_lo + (int64_t)l * R);
            const int64_t hi_l = zb < a.in_hi ? zb - (int64_t)l * R : (a.edge_hi ? a.n0 : a.in_hi - (int64_t)l * R);
            if (z >= lo_l && z < hi_l) {
                const C* wp = win + (int64_t)(l - 1) * W * tile_cells;  // level l-1 window
                const bool zint = z >= R && z < a.n0 - R;
                const int base = (int)((z - a.in_lo) % W);
                const bool last = l == a.depth;
                const bool store_z = last && z >= zs && z < ze;
                const int m = l * R;  // level-l in-plane margin inside the loaded tile
                const int yl0 = (SHAPE == kStar3D || SHAPE == kVarcoef3D) ? m : 0;
                const int yl1 = (SHAPE == kStar3D || SHAPE == kVarcoef3D) ? ly - m : ly;
                for (int64_t i = tid; i < tile_cells; i += nthr) {
                    int ly_ = (int)(i / lx), lx_ = (int)(i % lx);
                    if (ly_ < yl0 || ly_ >= yl1 || lx_ < m || lx_ >= lx - m) continue;
                    int64_t gy = y0 - (SHAPE == kStar3D || SHAPE == kVarcoef3D ? H : 0) + ly_;
                    int64_t gx = x0 - H + lx_;
                    if (gy < 0 || gy >= a.ny || gx < 0 || gx >= a.nx) continue;
                    auto W_ = [&](int dz, int dy, int dx) -> C {
                        int sl = (base + dz + W) % W;
                        return wp[(int64_t)sl * tile_cells + (int64_t)(ly_ + dy) * lx + (lx_ + dx)];
                    };
                    C v;
                    bool inter = zint && gx >= R && gx < a.nx - R;
                    if (SHAPE == kStar3D || SHAPE == kVarcoef3D) inter = inter && gy >= R && gy < a.ny - R;
                    if (!inter) {
                        v = W_(0, 0, 0);
                    } else if (SHAPE == kStar3D) {
                        // streaming order: axis 0 from -R up to -1, centre,
                        // axis 1 (-j,+j), axis 2 (-j,+j), then axis 0 +1..+R
                        v = cst[1 + 2 * (R - 1)] * W_(-R, 0, 0);
#pragma unroll
                        for (int j = R - 1; j >= 1; --j) v = fma_c(cst[1 + 2 * (j - 1)], W_(-j, 0, 0), v);
                        v = fma_c(cst[0], W_(0, 0, 0), v);
#pragma unroll
                        for (int j = 1; j <= R; ++j) {
                            v = fma_c(cst[1 + 2 * R + 2 * (j - 1)], W_(0, -j, 0), v);
                            v = fma_c(cst[2 + 2 * R + 2 * (j - 1)], W_(0, j, 0), v);
                        }
#pragma unroll
                        for (int j = 1; j <= R; ++j) {
                            v = fma_c(cst[1 + 4 * R + 2 * (j - 1)], W_(0, 0, -j), v);
                            v = fma_c(cst[2 + 4 * R + 2 * (j - 1)], W_(0, 0, j), v);
                        }
#pragma unroll
                        for (int j = 1; j <= R; ++j) v = fma_c(cst[2 + 2 * (j - 1)], W_(j, 0, 0), v);
                    } else if (SHAPE == kStar2D) {
                        v = cst[0] * W_(0, 0, 0);
                        int k = 1;
#pragma unroll
                        for (int j = 1; j <= R; ++j) { v = fma_c(cst[k], W_(-j, 0, 0), v); ++k; v = fma_c(cst[k], W_(j, 0, 0), v); ++k; }
#pragma unroll
                        for (int j = 1; j <= R; ++j) { v = fma_c(cst[k], W_(0, 0, -j), v); ++k; v = fma_c(cst[k], W_(0, 0, j), v); ++k; }
                    } else if (SHAPE == kBox2D) {
                        v = cst[0] * W_(-R, 0, -R);
#pragma unroll
                        for (int k = 1; k < W * W; ++k) v = fma_c(cst[k], W_(k / W - R, 0, k % W - R), v);
                    } else {  // kVarcoef3D: faces (-e0,+e0,-e1,+e1,-e2,+e2), centre 1 - sum
                        int64_t cs = (a.coef_slot0 + (z - a.coef_lo)) % a.coef_cap;
                        const C* cp = coef + cs * plane + gy * a.nx + gx;
                        C cf0 = cp[0], cf1 = cp[a.coef_field_stride], cf2 = cp[2 * a.coef_field_stride];
                        C cf3 = cp[3 * a.coef_field_stride], cf4 = cp[4 * a.coef_field_stride];
                        C cf5 = cp[5 * a.coef_field_stride];
                        C csum = cf0 + cf1;
                        csum = csum + cf2;
                        csum = csum + cf3;
                        csum = csum + cf4;
                        csum = csum + cf5;
                        v = ((C)1 - csum) * W_(0, 0, 0);
                        v = fma_c(cf0, W_(-1, 0, 0), v);
                        v = fma_c(cf1, W_(1, 0, 0), v);
                        v = fma_c(cf2, W_(0, -1, 0), v);
                        v = fma_c(cf3, W_(0, 1, 0), v);
                        v = fma_c(cf4, W_(0, 0, -1), v);
                        v = fma_c(cf5, W_(0, 0, 1), v);
                    }
                    if (!last) {
                        win[((int64_t)l * W + base) * tile_cells + i] = v;
                    } else if (store_z) {
                        int64_t oy = gy - y0, ox = gx - x0;
                        bool in_tile = ox >= 0 && ox < a.tx;
                        if (SHAPE == kStar3D || SHAPE == kVarcoef3D) in_tile = in_tile && oy >= 0 && oy < a.ty;
                        if (in_tile) store_as<T, C>(out + (z - a.out_lo) * plane + gy * a.nx + gx, v);
                    }
                }
            }
            __syncthreads();
        }
    }
}

}  // namespace so2dr
