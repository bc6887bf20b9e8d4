// star3d_fast.cuh -- register-streaming temporal-blocking kernel for 3D star
// stencils (radius R, K fused steps per launch), FP32 arithmetic on FP32 /
// BF16 / FP16 storage.
//
// The on-chip temporal blocking of Sec. III / Sec. IV-A, laid out for sm_103a:
//  * a CTA owns a 128-wide x tile (32 lanes x float4) and NW*VY rows of y
//    (VY rows per warp) and streams the planes of axis 0 through it; a launch
//    may also split axis 0 into segments (gridDim.z) so that the grid fills
//    the SMs evenly;
//  * each input plane is read from device memory once: cp.async copies
//    (16-byte vectors, zero-fill outside the grid) stage it one plane ahead in
//    a double-buffered shared-memory plane; y neighbours come from shared
//    memory, x neighbours from warp shuffles;
//  * every fused level keeps 2R partial sums per cell in registers: when the
//    previous level produces plane z', it is added into the targets
//    z'-R..z'+R (in-plane terms at z') and target z'-R is complete.  The slot
//    of a target is fixed by its plane index modulo 2R and the plane loop is
//    unrolled 2R times, so the ring never moves data;
//  * levels are pipelined across planes: level l consumes what level l-1
//    completed in the previous phase, so one barrier per plane suffices;
//  * every cell is computed as if interior (no per-cell predicates); cells of
//    the fixed boundary never change, so on completion they take their input
//    value back from the launch's input buffer (rare, warp-uniform branch);
//  * control flow is uniform: the stream feeds zeros beyond the input, which
//    only ever reach targets outside the valid trapezoid.
// The computed area shrinks by R per level in y and x, the compute-area
// adjustment of Algorithm 1 applied inside a launch.
//
// Per-cell arithmetic order (identical in every launch, chunk and tile):
//   c(-R e0) u, then FMAs with c(-R+1 e0) ... c(-e0), c(0), c(-e1), c(+e1),
//   ..., c(-R e1), c(+R e1), c(-e2), c(+e2), ..., c(+e0), ..., c(+R e0).
#pragma once

#include <type_traits>

#include "stencil.cuh"

namespace so2dr {

// Loaded-tile shape per (R, K): 16 warps of 2 rows (8 warps for one level).
// Four fused levels fit 128 registers per thread this way, so a 512-thread
// CTA fills the register file: 16 warps per SM (against 8 warps of 4 rows,
// which needed 235 registers: 2.6% slower on 1024^3, 10% on 512^3).
template <int R, int K> struct FastShape {
    static constexpr int VY = 2;
    static constexpr int NW = K == 1 ? 8 : 16;
    static constexpr int LX = 128;
    static constexpr int LYT = NW * VY;
    static constexpr int HXA = ((R * K + 3) / 4) * 4;   // x halo, whole float4s
    static constexpr int HY = R * (K - 1);             // computed-row halo in y
    static constexpr int TX = LX - 2 * HXA;
    static constexpr int TY = LYT - 2 * HY;
    static constexpr int INROWS = LYT + 2 * R;
    static constexpr int LROWS = LYT + 2 * R;           // level planes with R spare rows each side
    // planes kept per level: the arrival of the current phase, the one being
    // written, and the R older ones whose values boundary cells take back on
    // completion
    static constexpr int NB = R + 2;
    template <int ES> static constexpr int smem() { return NB * INROWS * LX * ES + NB * (K - 1) * LROWS * LX * 4; }
};

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
__device__ __forceinline__ float ld1(const float* p) { return *p; }
__device__ __forceinline__ float ld1(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ld1(const __half* p) { return __half2float(*p); }

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
__host__ __device__ constexpr int pmod(int a, int m) { return ((a % m) + m) % m; }

template <typename T, int R, int K>
struct FastTB {
    using S = FastShape<R, K>;
    static constexpr int VY = S::VY, NW = S::NW, LX = S::LX, LYT = S::LYT, INROWS = S::INROWS;
    static constexpr int RPW = (INROWS + NW - 1) / NW, W2 = 2 * R, NC = 1 + 6 * R, LROWS = S::LROWS, NB = S::NB;

    const StencilArgs& a;
    T* sin;        // [NB][INROWS][LX] staged input planes (plane of phase p in slot p % NB)
    float* slev;   // [K-1][NB][LROWS][LX] completed planes of levels 0..K-2 (R spare rows each side)
    int rowoff[RPW];   // element offset of each staged row inside a plane
    unsigned rowok;    // bit i: staged row i lies inside the grid
    int lane, warp, my_row, n0, olo, ohi;
    int need_lo, need_hi;  // level L processes arrivals in [need_lo - (K-L)R, need_hi + (K-L)R), clipped at za
    int xs, ys, ny, nx, gx0, za, zb, slot_next;  // extents and plane indices fit in 32 bits
    int64_t plane;
    bool xin, warp_bnd;
    unsigned inyx;  // bit y*4+e: my cell is an interior cell of the plane
    const T* in;
    T* out;
    float2 A[K][W2][VY][2];  // 2R partial sums per cell per level, in x pairs

    __device__ __forceinline__ explicit FastTB(const StencilArgs& args) : a(args) {}

    // input plane z -> buffer b (zeros past zb or outside the grid)
    __device__ __forceinline__ void stage_plane(int z, int b) {
        if (z >= zb) return;  // past the input: the buffer keeps stale data that only phantom targets see
        const T* base = in + (int64_t)slot_next * plane;
        T* sb = sin + b * INROWS * LX + warp * LX + lane * 4;
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
            if (warp + i * NW < INROWS) {
                bool ok = (rowok >> i) & 1u;
                cp_async_vec4(sb + i * NW * LX, ok ? base + rowoff[i] : in, ok);
            }
        }
        cp_async_commit();
        if (++slot_next == a.in_cap) slot_next = 0;
    }

    // one arrival at level L of plane zp (phase PH = (zp - za) mod 2R); rows
    // is the arrival plane's smem copy, tile row t at row t + shift (rows
    // -R..LYT+R-1 of the tile exist; those outside the tile hold garbage that
    // only reaches cells outside the level's valid area)
    template <int L, int PH, typename ST>
    __device__ __forceinline__ void arrive(const float2 (&v)[VY][2], const ST* rows, int shift,
                                           float2 (&done)[VY][2]) {
        // x neighbours beyond my 4 cells, from the adjacent lanes
        float lft[VY][4], rgt[VY][4];
#pragma unroll
        for (int y = 0; y < VY; ++y)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float me = (e & 1) ? v[y][e >> 1].y : v[y][e >> 1].x;
                lft[y][e] = (e >= 4 - R) ? __shfl_up_sync(0xffffffffu, me, 1) : 0.f;
                rgt[y][e] = (e < R) ? __shfl_down_sync(0xffffffffu, me, 1) : 0.f;
            }
        // y neighbours outside my VY rows, from shared memory
        float4 up[VY][R], dn[VY][R];
#pragma unroll
        for (int y = 0; y < VY; ++y)
#pragma unroll
            for (int j = 1; j <= R; ++j) {
                if (y - j < 0) up[y][j - 1] = lds4(rows + (my_row + y - j + shift) * LX + lane * 4);
                if (y + j >= VY) dn[y][j - 1] = lds4(rows + (my_row + y + j + shift) * LX + lane * 4);
            }
        // value of x neighbour e (-R..3+R) of row y, and the pair starting there
        auto xval = [&](int y, int e) -> float {
            if (e < 0) return lft[y][4 + e];
            if (e > 3) return rgt[y][e - 4];
            return (e & 1) ? v[y][e >> 1].y : v[y][e >> 1].x;
        };
        auto xpair = [&](int y, int e) -> float2 {
            if (e == 0 || e == 2) return v[y][e >> 1];
            return make_float2(xval(y, e), xval(y, e + 1));
        };
        auto ypair = [&](int y, int j, int h) -> float2 {  // row y + j (j may be out of my rows)
            if (y + j >= 0 && y + j < VY) return v[y + j][h];
            const float4 q = (j < 0) ? up[y][-j - 1] : dn[y][j - 1];
            return h ? make_float2(q.z, q.w) : make_float2(q.x, q.y);
        };
        // target t is plane zp - R + t, kept in slot (PH - R + t) mod 2R.
        // Cells are processed in x pairs with packed FP32x2 FMAs (each lane
        // of a pair is an ordinary fused multiply-add rounded once, so the
        // per-cell order below is the same as the scalar one).
#pragma unroll
        for (int y = 0; y < VY; ++y)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int e0 = 2 * h;
                const float2 x = v[y][h];
#pragma unroll
                for (int t = R + 1; t < 2 * R; ++t) {
                    float2& acc = A[L][pmod(PH - R + t, W2)][y][h];
                    acc = __ffma2_rn(a.cf2[cidx<R>(0, -1, t - R)], x, acc);
                }
                {
                    float2& acc = A[L][pmod(PH, W2)][y][h];
                    float2 s2 = __ffma2_rn(a.cf2[0], x, acc);
#pragma unroll
                    for (int j = 1; j <= R; ++j) {
                        s2 = __ffma2_rn(a.cf2[cidx<R>(1, -1, j)], ypair(y, -j, h), s2);
                        s2 = __ffma2_rn(a.cf2[cidx<R>(1, +1, j)], ypair(y, +j, h), s2);
                    }
#pragma unroll
                    for (int j = 1; j <= R; ++j) {
                        s2 = __ffma2_rn(a.cf2[cidx<R>(2, -1, j)], xpair(y, e0 - j), s2);
                        s2 = __ffma2_rn(a.cf2[cidx<R>(2, +1, j)], xpair(y, e0 + j), s2);
                    }
                    acc = s2;
                }
#pragma unroll
                for (int t = 0; t < R; ++t) {
                    float2& acc = A[L][pmod(PH - R + t, W2)][y][h];
                    acc = __ffma2_rn(a.cf2[cidx<R>(0, +1, R - t)], x, acc);
                }
                float2& a0 = A[L][pmod(PH - R, W2)][y][h];
                done[y][h] = a0;
                a0 = __fmul2_rn(a.cf2[cidx<R>(0, -1, R)], x);  // first contribution to target zp + R
            }
    }

    // Boundary cells (and whole boundary planes) keep their value: on
    // completion they take back the value they had at their centre arrival,
    // R phases ago, still resident in slot `cs` of the arrival planes.
    template <typename ST>
    __device__ __forceinline__ void fixup(float2 (&done)[VY][2], int zt, const ST* cen) {
        const bool zbnd = zt < R || zt >= n0 - R;
        if (!(zbnd || warp_bnd)) return;
#pragma unroll
        for (int y = 0; y < VY; ++y) {
            const unsigned rowmask = (inyx >> (y * 4)) & 0xFu;
            if (zbnd || rowmask != 0xFu) {
                const float4 q = lds4(cen + (my_row + y + R) * LX + lane * 4);
                if (zbnd || !(rowmask & 1u)) done[y][0].x = q.x;
                if (zbnd || !(rowmask & 2u)) done[y][0].y = q.y;
                if (zbnd || !(rowmask & 4u)) done[y][1].x = q.z;
                if (zbnd || !(rowmask & 8u)) done[y][1].y = q.w;
            }
        }
    }

    __device__ __forceinline__ void emit(const float2 (&done)[VY][2], int zt) {
        if (zt < olo || zt >= ohi) return;
        const int lx0 = lane * 4;
        if (!(lx0 >= S::HXA && lx0 < S::HXA + S::TX && xin)) return;
        T* ob = out + (int64_t)(zt - (int)a.out_lo) * plane;
#pragma unroll
        for (int y = 0; y < VY; ++y) {
            int ty = my_row + y;
            int gy = ys + ty;
            if (ty >= S::HY && ty < S::HY + S::TY && gy < ny)
                st4(ob + (int64_t)gy * nx + gx0, make_float4(done[y][0].x, done[y][0].y, done[y][1].x, done[y][1].y));
        }
    }

    // level L of phase p (phase PH = p mod 2R): consumes input plane za + p
    // (L = 0) or what level L-1 completed in phase p-1 (plane za + p - L(R+1))
    template <int L, int PH>
    __device__ __forceinline__ void level(int p, const T* sbuf, int buf) {
        // buf = p % NB: the slot this phase writes (and, for level 0, reads);
        // arrivals from the level below were written in phase p-1
        // arrivals that can reach the requested output planes (uniform per CTA)
        const int zp = za + p - L * (R + 1);
        const int lo = need_lo - (K - L) * R, hi = need_hi + (K - L) * R;
        if (zp < za || zp < lo || zp >= hi) {
            if constexpr (L + 1 < K) level<L + 1, PH>(p, sbuf, buf);
            return;
        }
        float2 v[VY][2], done[VY][2];
        const int zt = za + p - L * (R + 1) - R;
        if constexpr (L == 0) {
#pragma unroll
            for (int y = 0; y < VY; ++y) {
                const float4 q = lds4(sbuf + (my_row + y + R) * LX + lane * 4);
                v[y][0] = make_float2(q.x, q.y);
                v[y][1] = make_float2(q.z, q.w);
            }
            arrive<0, PH>(v, sbuf, R, done);
            fixup(done, zt, sin + ((p - R + NB * R) % NB) * INROWS * LX);
        } else {
            const int pa = (p - 1 + NB) % NB;  // slot written in phase p-1
            const float* prev = slev + ((L - 1) * NB + pa) * LROWS * LX;
#pragma unroll
            for (int y = 0; y < VY; ++y) {
                const float4 q = lds4(prev + (my_row + y + R) * LX + lane * 4);
                v[y][0] = make_float2(q.x, q.y);
                v[y][1] = make_float2(q.z, q.w);
            }
            arrive<L, pmod(PH - L * (R + 1), W2)>(v, prev, R, done);
            fixup(done, zt, slev + ((L - 1) * NB + (p - 1 - R + NB * (R + 1)) % NB) * LROWS * LX);
        }
        if constexpr (L == K - 1) {
            emit(done, zt);
        } else {
            float* lb = slev + (L * NB + buf) * LROWS * LX;
#pragma unroll
            for (int y = 0; y < VY; ++y)
                *reinterpret_cast<float4*>(lb + (my_row + y + R) * LX + lane * 4) =
                    make_float4(done[y][0].x, done[y][0].y, done[y][1].x, done[y][1].y);
        }
        if constexpr (L + 1 < K) level<L + 1, PH>(p, sbuf, buf);
    }

    template <int PH>
    __device__ __forceinline__ void phase(int p0) {
        const int p = p0 + PH;
        cp_async_wait_all();
        __syncthreads();
        const int buf = p % NB;
        stage_plane(za + p + 1, (p + 1) % NB);
        level<0, PH>(p, sin + buf * INROWS * LX, buf);
        if constexpr (PH + 1 < W2) phase<PH + 1>(p0);
    }

    __device__ __forceinline__ void run(void* smem) {
        sin = reinterpret_cast<T*>(smem);
        slev = reinterpret_cast<float*>(smem) + (NB * INROWS * LX * sizeof(T)) / 4;
        lane = threadIdx.x & 31;
        warp = threadIdx.x >> 5;
        my_row = warp * VY;
        const int x0 = (int)blockIdx.x * S::TX, y0 = (int)blockIdx.y * S::TY;
        xs = x0 - S::HXA;
        ys = y0 - S::HY;
        ny = (int)a.ny;
        nx = (int)a.nx;
        plane = a.ny * a.nx;
        n0 = (int)a.n0;
        gx0 = xs + lane * 4;
        xin = gx0 >= 0 && gx0 < nx;  // nx % 4 == 0: a vector is all in or all out
        in = static_cast<const T*>(a.in);
        out = static_cast<T*>(a.out);
        inyx = 0;
#pragma unroll
        for (int y = 0; y < VY; ++y)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                int gy = ys + my_row + y, gx = gx0 + e;
                if (gy >= R && gy < ny - R && gx >= R && gx < nx - R) inyx |= 1u << (y * 4 + e);
            }
        warp_bnd = __any_sync(0xffffffffu, inyx != (1u << (4 * VY)) - 1u);
        rowok = 0;
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
            int gy = ys - R + warp + i * NW;
            rowoff[i] = gy * nx + gx0;
            if (xin && gy >= 0 && gy < ny) rowok |= 1u << i;
        }
#pragma unroll
        for (int l = 0; l < K; ++l)
#pragma unroll
            for (int q = 0; q < W2; ++q)
#pragma unroll
                for (int y = 0; y < VY; ++y)
#pragma unroll
                    for (int h = 0; h < 2; ++h) A[l][q][y][h] = make_float2(0.f, 0.f);
        // axis-0 segment of this CTA: outputs [zs, ze), stream over [za, zb)
        const int nseg = gridDim.z;
        const int nout = (int)(a.out_hi - a.out_lo), in_lo = (int)a.in_lo, in_hi = (int)a.in_hi;
        const int zs = (int)a.out_lo + (int)((int64_t)nout * blockIdx.z / nseg);
        const int ze = (int)a.out_lo + (int)((int64_t)nout * (blockIdx.z + 1) / nseg);
        za = zs - K * R > in_lo ? zs - K * R : in_lo;
        zb = ze + K * R < in_hi ? ze + K * R : in_hi;
        olo = zs;
        ohi = ze;
        slot_next = (int)((a.in_slot0 + (za - in_lo)) % a.in_cap);
        need_lo = zs > (int)a.out_lo ? zs : (int)a.out_lo;
        need_hi = ze < (int)a.out_hi ? ze : (int)a.out_hi;
        // last arrival any level needs: level K-1 at plane need_hi + R - 1
        const int nph0 = (need_hi + R - 1 - za) + (K - 1) * (R + 1) + 1;
        const int nph = (nph0 + W2 - 1) / W2 * W2;
        stage_plane(za, 0);
        for (int p0 = 0; p0 < nph; p0 += W2) phase<0>(p0);
        cp_async_wait_all();
    }
};

template <typename T, int R, int K>
__global__ void __launch_bounds__(FastShape<R, K>::NW * 32, 1) star3d_fast_kernel(const StencilArgs a) {
    extern __shared__ float4 smem4[];
    FastTB<T, R, K> k(a);
    k.run(smem4);
}

}  // namespace so2dr
