// star3d_fast.cuh -- register-streaming temporal-blocking kernel for 3D star
// stencils (radius R, K fused steps per launch), FP32 arithmetic on FP32 /
// BF16 / FP16 storage.
//
// The on-chip temporal blocking of Sec. III / Sec. IV-A, laid out for sm_103a:
//  * a CTA owns a 128-wide x tile (32 lanes x float4) and NW*VY rows of y
//    (one warp per VY rows) and streams the planes of axis 0 through it;
//  * each input plane is read from device memory once: cp.async copies
//    (16-byte vectors, zero-fill outside the grid) stage it one plane ahead in
//    a double-buffered shared-memory plane that gives the y neighbours; x
//    neighbours come from warp shuffles;
//  * every fused level keeps only 2R partial sums per cell in registers: when
//    the previous level produces plane z', it is added into the targets
//    z'-R..z'+R (in-plane terms at z'), and target z'-R is complete.  Only
//    the last level is stored;
//  * control flow is uniform: the stream runs nin + K*R steps and feeds zeros
//    beyond the input, which only ever reach targets outside the valid
//    trapezoid.
// The computed area shrinks by R per level in y (rows) and x (columns),
// exactly the compute-area adjustment of Algorithm 1 applied inside a launch.
//
// Per-cell arithmetic order (identical in every launch, chunk and tile):
//   c(-R e0) u, then FMAs with c(-R+1 e0) ... c(-e0), c(0), c(-e1), c(+e1),
//   ..., c(-R e1), c(+R e1), c(-e2), c(+e2), ..., c(+e0), ..., c(+R e0).
#pragma once

#include "stencil.cuh"

namespace so2dr {

// Loaded-tile shape per (R, K): warps along y, VY rows per warp.
template <int R, int K> struct FastShape {
    // two rows per thread; 16 warps when the launch fuses several levels

    static constexpr int VY = 2;
    static constexpr int NW = (K == 1) ? 8 : 16;
    static constexpr int LX = 128;
    static constexpr int LYT = NW * VY;
    static constexpr int HXA = ((R * K + 3) / 4) * 4;   // x halo, whole float4s
    static constexpr int HY = R * (K - 1);             // computed-row halo in y
    static constexpr int TX = LX - 2 * HXA;
    static constexpr int TY = LYT - 2 * HY;
    static constexpr int INROWS = LYT + 2 * R;
    template <int ES> static constexpr int smem() { return 2 * INROWS * LX * ES + 2 * (K - 1) * LYT * LX * 4; }
};

// Input rows of a plane are staged with cp.async (zero-fill outside the grid).
template <typename T> __device__ __forceinline__ void cp_async_vec4(T* sdst, const T* gsrc, bool valid) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    int n = valid ? (int)(4 * sizeof(T)) : 0;
    if (sizeof(T) == 4)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gsrc), "r"(n));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gsrc), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 lds4(const __nv_bfloat16* p) {
    uint2 raw = *reinterpret_cast<const uint2*>(p);
    float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.x));
    float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 lds4(const __half* p) {
    uint2 raw = *reinterpret_cast<const uint2*>(p);
    float2 a = __half22float2(*reinterpret_cast<const __half2*>(&raw.x));
    float2 b = __half22float2(*reinterpret_cast<const __half2*>(&raw.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float4 ld4(const __nv_bfloat16* p) {
    uint2 raw = __ldg(reinterpret_cast<const uint2*>(p));
    float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.x));
    float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 ld4(const __half* p) {
    uint2 raw = __ldg(reinterpret_cast<const uint2*>(p));
    float2 a = __half22float2(*reinterpret_cast<const __half2*>(&raw.x));
    float2 b = __half22float2(*reinterpret_cast<const __half2*>(&raw.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ void st4(__nv_bfloat16* p, float4 v) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    uint2 raw;
    raw.x = *reinterpret_cast<unsigned*>(&a);
    raw.y = *reinterpret_cast<unsigned*>(&b);
    *reinterpret_cast<uint2*>(p) = raw;
}
__device__ __forceinline__ void st4(__half* p, float4 v) {
    __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
    uint2 raw;
    raw.x = *reinterpret_cast<unsigned*>(&a);
    raw.y = *reinterpret_cast<unsigned*>(&b);
    *reinterpret_cast<uint2*>(p) = raw;
}

__device__ __forceinline__ float f4get(const float4& v, int e) {
    return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
}

// Coefficient-table index of offset (axis, s*j), s = -1 or +1 (star order).
template <int R> __host__ __device__ constexpr int cidx(int axis, int s, int j) {
    return 1 + axis * 2 * R + 2 * (j - 1) + (s > 0 ? 1 : 0);
}

// One arrival of plane zp of the previous level: v holds its values on my
// cells, `rows` its smem copy (row 0 = thread-tile row 0 + row_shift; valid
// rows [rlo, rhi) of the copy).  Updates the 2R partial sums A and returns
// the completed target zp - R in `done`.
template <int R, int VY, typename ST>
__device__ __forceinline__ void level_arrival(float (&A)[2 * R][VY][4], const float (&v)[VY][4],
                                              const ST* rows, int row_shift, int rlo, int rhi,
                                              int my_row, int lane, const float* c,
                                              const unsigned inyx_mask, int64_t zp, int64_t n0,
                                              float (&done)[VY][4]) {
    // z-interior flags of the targets zp - R + t, t = 0..2R
    bool zi[2 * R + 1];
#pragma unroll
    for (int t = 0; t <= 2 * R; ++t) {
        int64_t zt = zp - R + t;
        zi[t] = zt >= R && zt < n0 - R;
    }
    // x neighbours from the adjacent lanes
    float lft[VY][4], rgt[VY][4];
#pragma unroll
    for (int y = 0; y < VY; ++y)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            lft[y][e] = (e >= 4 - R) ? __shfl_up_sync(0xffffffffu, v[y][e], 1) : 0.f;
            rgt[y][e] = (e < R) ? __shfl_down_sync(0xffffffffu, v[y][e], 1) : 0.f;
        }
    // y neighbours outside my VY rows, from shared memory
    float4 up[VY][R], dn[VY][R];
#pragma unroll
    for (int y = 0; y < VY; ++y)
#pragma unroll
        for (int j = 1; j <= R; ++j) {
            if (y - j < 0) {
                int r = my_row + y - j + row_shift;
                r = r < rlo ? rlo : (r >= rhi ? rhi - 1 : r);
                up[y][j - 1] = lds4(rows + (int64_t)r * 128 + lane * 4);
            }
            if (y + j >= VY) {
                int r = my_row + y + j + row_shift;
                r = r < rlo ? rlo : (r >= rhi ? rhi - 1 : r);
                dn[y][j - 1] = lds4(rows + (int64_t)r * 128 + lane * 4);
            }
        }
    float newacc[VY][4];
#pragma unroll
    for (int y = 0; y < VY; ++y)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const bool cin = (inyx_mask >> (y * 4 + e)) & 1u;
            const float x = v[y][e];
            // t = 2R: first contribution to target zp + R (offset -R on axis 0)
            newacc[y][e] = (cin && zi[2 * R]) ? c[cidx<R>(0, -1, R)] * x : 0.f;
            // R < t < 2R: offsets -(t-R) on axis 0
#pragma unroll
            for (int t = R + 1; t < 2 * R; ++t)
                if (cin && zi[t]) A[t][y][e] = __fmaf_rn(c[cidx<R>(0, -1, t - R)], x, A[t][y][e]);
            // t = R: centre and in-plane terms
            {
                float s = __fmaf_rn(c[0], x, A[R][y][e]);
#pragma unroll
                for (int j = 1; j <= R; ++j) {
                    float ym = (y - j >= 0) ? v[y - j][e] : f4get(up[y][j - 1], e);
                    float yp = (y + j < VY) ? v[y + j][e] : f4get(dn[y][j - 1], e);
                    s = __fmaf_rn(c[cidx<R>(1, -1, j)], ym, s);
                    s = __fmaf_rn(c[cidx<R>(1, +1, j)], yp, s);
                }
#pragma unroll
                for (int j = 1; j <= R; ++j) {
                    float xm = (e - j >= 0) ? v[y][e - j] : lft[y][4 + e - j];
                    float xp = (e + j < 4) ? v[y][e + j] : rgt[y][e + j - 4];
                    s = __fmaf_rn(c[cidx<R>(2, -1, j)], xm, s);
                    s = __fmaf_rn(c[cidx<R>(2, +1, j)], xp, s);
                }
                A[R][y][e] = (cin && zi[R]) ? s : x;
            }
            // 0 <= t < R: offsets +(R-t) on axis 0
#pragma unroll
            for (int t = 0; t < R; ++t)
                if (cin && zi[t]) A[t][y][e] = __fmaf_rn(c[cidx<R>(0, +1, R - t)], x, A[t][y][e]);
            done[y][e] = A[0][y][e];
        }
    // rotate: target zp - R is complete
#pragma unroll
    for (int q = 0; q < 2 * R - 1; ++q)
#pragma unroll
        for (int y = 0; y < VY; ++y)
#pragma unroll
            for (int e = 0; e < 4; ++e) A[q][y][e] = A[q + 1][y][e];
#pragma unroll
    for (int y = 0; y < VY; ++y)
#pragma unroll
        for (int e = 0; e < 4; ++e) A[2 * R - 1][y][e] = newacc[y][e];
}

template <typename T, int R, int K>
__global__ void __launch_bounds__(FastShape<R, K>::NW * 32, 1) star3d_fast_kernel(const StencilArgs a) {
    using S = FastShape<R, K>;
    constexpr int VY = S::VY, NW = S::NW, LX = S::LX, LYT = S::LYT, INROWS = S::INROWS;
    constexpr int RPW = (INROWS + NW - 1) / NW;
    constexpr int NC = 1 + 6 * R;
    extern __shared__ float4 smem4[];
    T* sin = reinterpret_cast<T*>(smem4);                                        // [2][INROWS][LX]
    float* slev = reinterpret_cast<float*>(smem4) + (2 * INROWS * LX * sizeof(T)) / 4;  // [K-1][2][LYT][LX]

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int my_row = warp * VY;
    const int64_t x0 = (int64_t)blockIdx.x * S::TX, y0 = (int64_t)blockIdx.y * S::TY;
    const int64_t xs = x0 - S::HXA, ys = y0 - S::HY;
    const int64_t ny = a.ny, nx = a.nx, n0 = a.n0, plane = ny * nx;
    const T* in = static_cast<const T*>(a.in);
    T* out = static_cast<T*>(a.out);

    float c[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) c[k] = (float)a.c[k];

    unsigned inyx = 0;
#pragma unroll
    for (int y = 0; y < VY; ++y)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            int64_t gy = ys + my_row + y, gx = xs + lane * 4 + e;
            if (gy >= R && gy < ny - R && gx >= R && gx < nx - R) inyx |= 1u << (y * 4 + e);
        }

    float A[K][2 * R][VY][4];
#pragma unroll
    for (int l = 0; l < K; ++l)
#pragma unroll
        for (int q = 0; q < 2 * R; ++q)
#pragma unroll
            for (int y = 0; y < VY; ++y)
#pragma unroll
                for (int e = 0; e < 4; ++e) A[l][q][y][e] = 0.f;

    const int64_t gx0 = xs + lane * 4;
    const bool xin = gx0 >= 0 && gx0 < nx;  // nx % 4 == 0: a vector is all in or all out
    // stage input plane z (zeros past the input or outside the grid) in buffer b
    auto stage_plane = [&](int64_t z, int b) {
        const bool zin = z < a.in_hi;
        const int64_t slot = zin ? (a.in_slot0 + (z - a.in_lo)) % a.in_cap : 0;
        const T* base = in + slot * plane;
        T* sb = sin + b * INROWS * LX;
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
            int row = warp + i * NW;
            if (row < INROWS) {
                int64_t gy = ys - R + row;
                bool ok = zin && xin && gy >= 0 && gy < ny;
                cp_async_vec4(sb + row * LX + lane * 4, ok ? base + gy * nx + gx0 : in, ok);
            }
        }
        cp_async_commit();
    };

    const int64_t nin = a.in_hi - a.in_lo;
    const int64_t nsteps = nin + (int64_t)K * R;
    stage_plane(a.in_lo, 0);
    for (int64_t s = 0; s < nsteps; ++s) {
        const int64_t zin = a.in_lo + s;
        const int buf = (int)(s & 1);
        const T* sbuf = sin + buf * INROWS * LX;
        cp_async_wait_all();
        __syncthreads();  // plane zin staged by everyone; step s-1 fully done
        if (s + 1 < nsteps) stage_plane(zin + 1, buf ^ 1);
        // ---- level 1: arrival of input plane zin
        float v[VY][4], done[VY][4];
#pragma unroll
        for (int y = 0; y < VY; ++y) {
            float4 q = lds4(sbuf + (my_row + y + R) * LX + lane * 4);
            v[y][0] = q.x; v[y][1] = q.y; v[y][2] = q.z; v[y][3] = q.w;
        }
        level_arrival<R, VY, T>(A[0], v, sbuf, R, 0, INROWS, my_row, lane, c, inyx, zin, n0, done);
        // ---- levels 2..K: arrival of the previous level's completed plane
#pragma unroll
        for (int l = 1; l < K; ++l) {
            float* lb = slev + ((l - 1) * 2 + buf) * LYT * LX;
#pragma unroll
            for (int y = 0; y < VY; ++y)
                *reinterpret_cast<float4*>(lb + (my_row + y) * LX + lane * 4) =
                    make_float4(done[y][0], done[y][1], done[y][2], done[y][3]);
            __syncthreads();
#pragma unroll
            for (int y = 0; y < VY; ++y)
#pragma unroll
                for (int e = 0; e < 4; ++e) v[y][e] = done[y][e];
            level_arrival<R, VY, float>(A[l], v, lb, 0, 0, LYT, my_row, lane, c, inyx, zin - (int64_t)l * R, n0, done);
        }
        // ---- store the last level's completed plane
        const int64_t zo = zin - (int64_t)K * R;
        if (zo >= a.out_lo && zo < a.out_hi) {
            const int lx0 = lane * 4;
            if (lx0 >= S::HXA && lx0 < S::HXA + S::TX && xin) {
                T* ob = out + (zo - a.out_lo) * plane;
#pragma unroll
                for (int y = 0; y < VY; ++y) {
                    int ty = my_row + y;
                    int64_t gy = ys + ty;
                    if (ty >= S::HY && ty < S::HY + S::TY && gy < ny)
                        st4(ob + gy * nx + gx0, make_float4(done[y][0], done[y][1], done[y][2], done[y][3]));
                }
            }
        }
    }
}

}  // namespace so2dr
