// star3d_tb.cuh -- register-streaming temporal-blocking kernel for 3D star
// stencils (radius R, K fused steps per launch), FP32 arithmetic on FP32 /
// BF16 / FP16 storage.
//
// The on-chip temporal blocking of Sec. III / Sec. IV-A, laid out for sm_103a:
//  * a CTA owns a 128-wide x tile (32 lanes x 4 cells) and NW*VY rows of y
//    (VY rows per warp) and streams the planes of axis 0 through it.  The
//    host picks the work split that loads the SMs most evenly: either one
//    tile and one axis-0 segment per CTA (gridDim.z segments), or one CTA
//    per SM slot taking (tile, segment) units in rounds, with the units of
//    the last, partial round cut into shorter axis-0 pieces so that no SM
//    idles while others finish a whole unit;
//  * each input plane is read from device memory once, as one TMA box
//    (cp.async.bulk.tensor, issued by one thread, landing on an mbarrier) of
//    the tile plus R halo rows, PD planes ahead of its use in an NI-slot ring;
//    the box reads zeros where it leaves the grid;
//  * every fused level keeps 2R partial sums per cell in registers: when the
//    level below produces plane z', it is added into the targets z'-R..z'+R
//    (the in-plane terms at z') and target z'-R is complete.  The register
//    slot of a target is fixed by its plane index modulo 2R and the plane
//    loop is unrolled 2R times, so the ring never moves data;
//  * levels are pipelined across planes: level L consumes what level L-1
//    completed in the previous phase, so one barrier per plane suffices.  A
//    thread's own cells of that plane stay in its registers (levels run from
//    the deepest down, so each reads them before they are replaced); only
//    the R rows at each end of a warp's rows go to shared memory (two plane
//    slots per level), for the neighbouring warps.  x neighbours come from
//    warp shuffles;
//  * every cell is computed as if interior.  Cells of the fixed boundary
//    (the in-plane ring of width R and the first and last R planes) keep
//    their value: the centre arrival of a boundary target stores the
//    arriving value and the later arrivals leave it alone.  Warps whose only
//    boundary cells are the ring's columns select those cells by a per-lane
//    predicate; warps with boundary rows, and phases with a fixed plane in
//    flight, select per cell on a slower path;
//  * a phase runs one body per boundary mode (no boundary cell, ring columns,
//    per-cell masks); for radius 1 the phases in which every level is active
//    run straight-line bodies without per-level tests, for larger radii (2R
//    phases of longer bodies) a uniform per-level test keeps the code inside
//    the instruction cache.
// The valid area shrinks by R per level in y and x: the compute-area
// adjustment of Algorithm 1 applied inside a launch.
//
// Per-cell arithmetic order (identical in every launch, chunk and tile, and
// the order of the generic kernel in stencil.cuh):
//   c(-R e0) u, then FMAs with c(-R+1 e0) ... c(-e0), c(0), c(-e1), c(+e1),
//   ..., c(-R e1), c(+R e1), c(-e2), c(+e2), ..., c(+e0), ..., c(+R e0).
#pragma once

#include "stencil.cuh"
#include "tb_common.cuh"

namespace so2dr {

// Tile shape per (R, K).  Fused depths: 8 warps of 4 rows, whose partial sums
// (K * 2R * 16 per thread) and carried cells fit the 255-register limit of a
// 256-thread CTA; radius 3 and 4 fuse two levels with 2 rows per warp (the
// 2R = 8 partial sums per cell and level leave no room for more).  One level:
// 8 warps of 2 rows, two CTAs per SM.
template <int R, int K> struct StarShape {
    static constexpr int VY = (K == 1 || R >= 3) ? 2 : 4;
    static constexpr int NW = 8;
    static constexpr int NT = NW * 32;
    static constexpr bool CARRY = K > 1;                // own cells of a level stay in registers
    static constexpr int LX = 128;                      // tile columns (32 lanes x 4)
    static constexpr int LYT = NW * VY;                 // tile rows
    static constexpr int HXA = ((R * K + 3) / 4) * 4;   // x halo, whole 4-cell vectors
    static constexpr int HY = R * (K - 1);              // rows lost per side to the y halo
    static constexpr int TX = LX - 2 * HXA;             // output columns per tile
    static constexpr int TY = LYT - 2 * HY;             // output rows per tile
    static constexpr int ROWS = LYT + 2 * R;            // staged input rows / level-plane rows
    // input plane slots: radius 4 at one level loads 6 (two CTAs per SM
    // still fit) and gains 4%; the other shapes lose occupancy or nothing
    static constexpr int NI = (R == 4 && K == 1) ? 6 : 4;
    static constexpr int PD = NI - 1;                   // planes loaded ahead
    static constexpr int NB = 2;                        // plane slots per intermediate level
    static constexpr int MINB = K == 1 ? 2 : 1;         // CTAs per SM the registers are sized for
    // staged columns: 16-bit boxes start on an 8-element boundary (16 bytes),
    // so they carry 8 spare columns and the tile starts 0 or 4 columns in
    template <int ES> static constexpr int lxb() { return ES == 4 ? LX : LX + 8; }
    template <int ES> static constexpr int box_bytes() { return lxb<ES>() * ROWS * ES; }
    template <int ES> static constexpr int in_slot_bytes() { return (box_bytes<ES>() + 127) / 128 * 128; }
    static constexpr int lev_bytes = ROWS * LX * 4;
    static constexpr int kBarBytes = 128;               // NI mbarriers, padded
    template <int ES> static constexpr int smem() {
        return kBarBytes + NI * in_slot_bytes<ES>() + (K - 1) * NB * lev_bytes;
    }
};

// How a warp treats the fixed boundary in a phase.
enum BndMode : int {
    kBndNone = 0,     // no boundary cell in the warp, no fixed plane in flight
    kBndColumns = 1,  // only the ring's columns: lanes holding column 0 or nx-1 select
    kBndCells = 2,    // boundary rows or fixed planes: per-cell masks
};

template <typename T, int R, int K, bool ZC>
struct StarTB {
    using S = StarShape<R, K>;
    static constexpr int VY = S::VY, NW = S::NW, LX = S::LX, LYT = S::LYT, ROWS = S::ROWS, NI = S::NI,
                         PD = S::PD, NB = S::NB, W2 = 2 * R, ES = (int)sizeof(T), LXB = S::template lxb<ES>(),
                         SLOT = S::template in_slot_bytes<ES>();
    static constexpr unsigned kAll = (1u << (4 * VY)) - 1u;
    static constexpr int kWorkOff = 64;  // work-split constants, behind the mbarriers
    static_assert(NI * 8 <= kWorkOff && kWorkOff + 8 * 4 <= S::kBarBytes, "barrier block layout");

    const StencilArgs& a;
    const CUtensorMap* tmap;
    uint32_t bar0, sin0;  // shared addresses: mbarrier 0, input slot 0
    const T* sin;         // [NI] slots of [ROWS][LXB] staged input
    float* slev;          // [K-1][NB][ROWS][LX] completed planes of levels 0..K-2
    int lane, warp, my_row, col0;
    int n0, ny, nx, xs, ys, gx0, bx0;
    int za, zb, olo, ohi, need_lo, need_hi;
    int ps_lo, ps_hi;     // phases in which every level is active
    int pfail;            // phase whose input copy did not land in time
    int gb;               // input copies issued by this CTA before the current piece
    unsigned par;         // bit s: parity of the next completion of mbarrier s
    int wmode;            // BndMode of my warp away from the fixed planes
    int64_t plane;
    bool xin;
    bool xl, xr;          // my lane holds column 0 / column nx-1 of the grid
    unsigned inyx;        // bit y*4+e: my cell (row y, column e) is interior in its plane
    T* out;
    const T* hin;         // zero-copy: mapped host grid (planes [hlo, hhi) come from there)
    int hlo, hhi;
    float2 A[K][W2][VY][2];                 // 2R partial sums per cell per level, in x pairs
    float2 C[K > 1 ? K - 1 : 1][VY][2];     // my cells of what levels 0..K-2 completed last phase

    __device__ __forceinline__ explicit StarTB(const StencilArgs& args, const CUtensorMap* m) : a(args), tmap(m) {}

    // first and one-past-last arrival plane level L needs
    __device__ __forceinline__ int lev_lo(int L) const {
        const int v = need_lo - (K - L) * R;
        return v > za ? v : za;
    }
    __device__ __forceinline__ int lev_hi(int L) const { return need_hi + (K - L) * R; }

    // boundary mask (bits y*4+e) of target plane zt: every cell of a fixed
    // plane, else the in-plane ring (and the cells outside the grid)
    __device__ __forceinline__ unsigned bmask(int zt) const {
        return (zt < R || zt >= n0 - R) ? kAll : (~inyx & kAll);
    }

    // one thread: TMA of the input plane of phase q into its slot
    // (the staging slot of phase q of a piece is (gb + q) mod NI: the slots
    // go round in issue order across the pieces of a CTA)
    __device__ __forceinline__ void issue(int q) {
        const int z = za + q;
        if (z >= zb) return;
        const int slot = (int)((a.in_slot0 + (int64_t)(z - (int)a.in_lo)) % a.in_cap);
        const int g = (gb + q) % NI;
        const uint32_t bar = bar0 + (uint32_t)g * 8u;
        mbar_arrive_expect_tx(bar, (uint32_t)S::template box_bytes<ES>());
        tma_load_3d(sin0 + (uint32_t)g * SLOT, tmap, bx0, ys - R, slot, bar);
    }

    // zero-copy input: plane z comes from the mapped host grid
    __device__ __forceinline__ bool host_plane(int z) const { return z < zb && z >= hlo && z < hhi; }

    // all threads: 16-byte cp.async copies of the box of phase q (the same
    // rows and columns the TMA box covers, zeros outside the grid) from the
    // mapped host grid into its slot
    __device__ __forceinline__ void stage_host(int q) {
        constexpr int VEC = 16 / ES, NV = LXB / VEC;
        const int z = za + q;
        const T* base = hin + (int64_t)z * plane;
        T* sb = const_cast<T*>(sin) + ((gb + q) % NI) * (SLOT / ES);
        for (int v = threadIdx.x; v < ROWS * NV; v += S::NT) {
            const int row = v / NV, cv = v - row * NV;
            const int gy = ys - R + row, gx = bx0 + cv * VEC;
            const bool ok = gy >= 0 && gy < ny && gx >= 0 && gx < nx;
            cp_async16(sb + row * LXB + cv * VEC, ok ? base + (int64_t)gy * nx + gx : base, ok);
        }
    }

    // all threads: the tile's own part of the host plane of phase p (rows
    // [y0, y0 + TY), columns [x0, x0 + TX): the tiles partition the plane) goes
    // into the input buffer, where later launches read it
    __device__ __forceinline__ void write_back(int p) {
        constexpr int VEC = 16 / ES, NV = S::TX / VEC;
        const int z = za + p;
        const int slot = (int)((a.in_slot0 + (int64_t)(z - (int)a.in_lo)) % a.in_cap);
        T* dst = const_cast<T*>(static_cast<const T*>(a.in)) + (int64_t)slot * plane;
        const T* sb = sin + ((gb + p) % NI) * (SLOT / ES);
        const int x0 = xs + S::HXA, y0 = ys + S::HY;
        for (int v = threadIdx.x; v < S::TY * NV; v += S::NT) {
            const int r = v / NV, cv = v - r * NV;
            const int gy = y0 + r, gx = x0 + cv * VEC;
            if (gy < ny && gx < nx)
                *reinterpret_cast<uint4*>(dst + (int64_t)gy * nx + gx) =
                    *reinterpret_cast<const uint4*>(sb + (gy - ys + R) * LXB + (gx - bx0));
        }
    }

    // keep (boundary) or nv, per element of a pair: per-cell mask bits
    // (kBndCells) or the column predicates of my lane (kBndColumns)
    template <int MODE>
    __device__ __forceinline__ float2 pick(unsigned m, int y, int h, float2 keep, float2 nv) const {
        const int e0 = 2 * h, bit = 4 * y + e0;
        if constexpr (MODE == kBndCells) {
            return make_float2(((m >> bit) & 1u) ? keep.x : nv.x, ((m >> (bit + 1)) & 1u) ? keep.y : nv.y);
        } else if constexpr (MODE == kBndColumns) {
            // columns 0..R-1 are cells e < R of the lane holding column 0,
            // columns nx-R..nx-1 cells e >= 4-R of the lane holding nx-1
            const bool p0 = (e0 < R && xl) || (e0 >= 4 - R && xr);
            const bool p1 = (e0 + 1 < R && xl) || (e0 + 1 >= 4 - R && xr);
            return make_float2(p0 ? keep.x : nv.x, p1 ? keep.y : nv.y);
        } else {
            return nv;
        }
    }

    // One arrival at level L whose target phase is PHL = (zp - za) mod 2R:
    // v holds my cells of the arriving plane, `rows` its shared-memory copy
    // (tile row t at row t + R, my first column at element col).  Masks
    // mz[t] (t = 0..R, kBndCells only) belong to targets zp - R + t.
    template <int L, int PHL, int MODE, typename ST>
    __device__ __forceinline__ void arrive(const float2 (&v)[VY][2], const ST* rows, int pitch, int col,
                                           float2 (&done)[VY][2], const unsigned (&mz)[R + 1]) {
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
                if (y - j < 0) up[y][j - 1] = lds4(rows + (my_row + y - j + R) * pitch + col);
                if (y + j >= VY) dn[y][j - 1] = lds4(rows + (my_row + y + j + R) * pitch + col);
            }
        auto xval = [&](int y, int e) -> float {
            if (e < 0) return lft[y][4 + e];
            if (e > 3) return rgt[y][e - 4];
            return (e & 1) ? v[y][e >> 1].y : v[y][e >> 1].x;
        };
        auto xpair = [&](int y, int e) -> float2 {
            if (e == 0 || e == 2) return v[y][e >> 1];
            return make_float2(xval(y, e), xval(y, e + 1));
        };
        auto ypair = [&](int y, int j, int h) -> float2 {
            if (y + j >= 0 && y + j < VY) return v[y + j][h];
            const float4 q = (j < 0) ? up[y][-j - 1] : dn[y][j - 1];
            return h ? make_float2(q.z, q.w) : make_float2(q.x, q.y);
        };
        // target t is plane zp - R + t, kept in slot (PHL - R + t) mod 2R;
        // cells go in x pairs through packed FP32x2 FMAs (each lane an
        // ordinary fused multiply-add, so the per-cell order is unchanged)
#pragma unroll
        for (int y = 0; y < VY; ++y)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int e0 = 2 * h;
                const float2 x = v[y][h];
#pragma unroll
                for (int t = R + 1; t < 2 * R; ++t) {
                    float2& acc = A[L][pmod(PHL - R + t, W2)][y][h];
                    acc = __ffma2_rn(a.cf2[cidx<R>(0, -1, t - R)], x, acc);
                }
                {
                    float2& acc = A[L][pmod(PHL, W2)][y][h];
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
                    // a boundary target keeps the value of its centre arrival
                    acc = pick<MODE>(mz[R], y, h, x, s2);
                }
#pragma unroll
                for (int t = 1; t < R; ++t) {
                    float2& acc = A[L][pmod(PHL - R + t, W2)][y][h];
                    acc = pick<MODE>(mz[t], y, h, acc, __ffma2_rn(a.cf2[cidx<R>(0, +1, R - t)], x, acc));
                }
                float2& a0 = A[L][pmod(PHL - R, W2)][y][h];
                done[y][h] = pick<MODE>(mz[0], y, h, a0, __ffma2_rn(a.cf2[cidx<R>(0, +1, R)], x, a0));
                a0 = __fmul2_rn(a.cf2[cidx<R>(0, -1, R)], x);  // first contribution to target zp + R
            }
    }

    __device__ __forceinline__ void emit(const float2 (&done)[VY][2], int zt) {
        if (zt < olo || zt >= ohi) return;
        const int lx0 = lane * 4;
        if (!(lx0 >= S::HXA && lx0 < S::HXA + S::TX && xin)) return;
        T* ob = out + (int64_t)(zt - (int)a.out_lo) * plane;
#pragma unroll
        for (int y = 0; y < VY; ++y) {
            const int ty = my_row + y, gy = ys + ty;
            if (ty >= S::HY && ty < S::HY + S::TY && gy < ny)
                st4(ob + (int64_t)gy * nx + gx0, make_float4(done[y][0].x, done[y][0].y, done[y][1].x, done[y][1].y));
        }
    }

    // level L of phase p (PH = p mod 2R; p0 is a multiple of 2R, so the
    // parity of p is that of PH): consumes input plane za + p (L = 0) or what
    // level L-1 completed in phase p-1 (plane za + p - L(R+1))
    template <int L, int PH, int MODE>
    __device__ __forceinline__ void level_body(int p) {
        const int zp = za + p - L * (R + 1);
        unsigned mz[R + 1];
#pragma unroll
        for (int t = 0; t <= R; ++t) mz[t] = MODE == kBndCells ? bmask(zp - R + t) : 0u;
        float2 v[VY][2], done[VY][2];
        constexpr int PHL = pmod(PH - L * (R + 1), W2);
        if constexpr (L == 0) {
            const T* rows = sin + ((gb + p) % NI) * (SLOT / ES);
#pragma unroll
            for (int y = 0; y < VY; ++y) {
                const float4 q = lds4(rows + (my_row + y + R) * LXB + col0);
                v[y][0] = make_float2(q.x, q.y);
                v[y][1] = make_float2(q.z, q.w);
            }
            arrive<0, PHL, MODE>(v, rows, LXB, col0, done, mz);
        } else {
            const float* prev = slev + ((L - 1) * NB + ((PH + 1) & 1)) * ROWS * LX;  // slot of phase p-1
#pragma unroll
            for (int y = 0; y < VY; ++y) {
                if constexpr (S::CARRY) {
                    v[y][0] = C[L - 1][y][0];
                    v[y][1] = C[L - 1][y][1];
                } else {
                    const float4 q = lds4(prev + (my_row + y + R) * LX + lane * 4);
                    v[y][0] = make_float2(q.x, q.y);
                    v[y][1] = make_float2(q.z, q.w);
                }
            }
            arrive<L, PHL, MODE>(v, prev, LX, lane * 4, done, mz);
        }
        if constexpr (L == K - 1) {
            emit(done, zp - R);
        } else {
            // my cells stay in registers for level L+1; the shared-memory plane
            // serves the neighbouring warps (the R rows at each end)
            float* lb = slev + (L * NB + (PH & 1)) * ROWS * LX;
#pragma unroll
            for (int y = 0; y < VY; ++y) {
                if (!S::CARRY || y < R || y >= VY - R)
                    *reinterpret_cast<float4*>(lb + (my_row + y + R) * LX + lane * 4) =
                        make_float4(done[y][0].x, done[y][0].y, done[y][1].x, done[y][1].y);
                if constexpr (S::CARRY) {
                    C[L][y][0] = done[y][0];
                    C[L][y][1] = done[y][1];
                }
            }
        }
    }

    // the levels of one phase, from the deepest down, so that level L reads
    // the carried cells of level L-1 before level L-1 replaces them; in the
    // head and tail of the stream a level runs only while its arrivals can
    // reach the requested output (ALL: a phase known to need every level)
    template <int L, int PH, int MODE, bool ALL>
    __device__ __forceinline__ void levels(int p, bool all) {
        if constexpr (ALL) {
            level_body<L, PH, MODE>(p);
        } else {
            const int zp = za + p - L * (R + 1);
            if (all || (zp >= lev_lo(L) && zp < lev_hi(L))) level_body<L, PH, MODE>(p);
        }
        if constexpr (L > 0) levels<L - 1, PH, MODE, ALL>(p, all);
    }

    // phase p = p0 + PH; false when an input copy did not land in time
    // the levels of phase p (PH = p mod 2R)
    template <int PH>
    __device__ __forceinline__ void phase_levels(int p) {
        // the arrivals of this phase span planes za + p - (K-1)(R+1) .. za + p;
        // a fixed plane among their targets (z' - R .. z') needs the cell path
        const bool all = p >= ps_lo && p < ps_hi;
        const bool fixed = za + p - (K - 1) * (R + 1) < 2 * R || za + p >= n0 - R;
        if constexpr (R == 1) {
            // short bodies: straight-line phases for the steady state, and
            // the checked ones for head, tail and fixed planes
            if (all && !fixed && wmode == kBndNone) levels<K - 1, PH, kBndNone, true>(p, true);
            else if (all && !fixed && wmode == kBndColumns) levels<K - 1, PH, kBndColumns, true>(p, true);
            else if (fixed || wmode != kBndNone) levels<K - 1, PH, kBndCells, false>(p, all);
            else levels<K - 1, PH, kBndNone, false>(p, all);
        } else {
            // long bodies (2R phases of them): one body per boundary mode,
            // which keeps the loop inside the instruction cache
            if (fixed || wmode == kBndCells) levels<K - 1, PH, kBndCells, false>(p, all);
            else if (wmode == kBndColumns) levels<K - 1, PH, kBndColumns, false>(p, all);
            else levels<K - 1, PH, kBndNone, false>(p, all);
        }
    }

    // phase p = p0 + PH: its input plane has landed (bounded wait), the
    // barrier, (zero-copy: the write-back of a host plane,) the copy of plane
    // p + PD, then the levels; false when an input copy did not land in time
    template <int PH>
    __device__ __forceinline__ bool phase(int p0) {
        const int p = p0 + PH;
        const int g = (gb + p) % NI;
        bool late = false;
        bool hp = false;
        if constexpr (ZC) hp = host_plane(za + p);
        const bool tma = !hp && za + p < zb;
        if (hp) cp_async_wait_group<PD - 1>();  // one group per phase: this phase's has landed
        else if (tma) late = !mbar_wait_bounded(bar0 + (uint32_t)g * 8u, (par >> g) & 1u);
        if (__syncthreads_or(late)) {
            pfail = p;
            return false;
        }
        if (tma) par ^= 1u << g;  // (flipped only once every thread saw the copy land)
        // the slot of phase p + PD last held phase p - 1, read before the barrier
        if constexpr (ZC) {
            if (hp) write_back(p);
            if (host_plane(za + p + PD)) stage_host(p + PD);
            else if (threadIdx.x == 0) {
                fence_proxy_async_smem();
                issue(p + PD);
            }
            cp_async_commit();
        } else if (threadIdx.x == 0) {
            fence_proxy_async_smem();
            issue(p + PD);
        }
        phase_levels<PH>(p);
        if constexpr (PH + 1 < W2) return phase<PH + 1>(p0);
        return true;
    }

    // one piece: output planes [zs, ze) of tile (tx, ty); false when an input
    // copy did not land in time
    __device__ __forceinline__ bool piece(int tx, int ty, int zs, int ze) {
        const int x0 = tx * S::TX, y0 = ty * S::TY;
        xs = x0 - S::HXA;
        ys = y0 - S::HY;
        gx0 = xs + lane * 4;
        xin = gx0 >= 0 && gx0 < nx;  // nx % 4 == 0: a vector is all in or all out
        bx0 = ES == 4 ? xs : (xs & ~7);  // 16-byte aligned box start
        col0 = (xs - bx0) + lane * 4;
        inyx = 0;
#pragma unroll
        for (int y = 0; y < VY; ++y)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int gy = ys + my_row + y, gx = gx0 + e;
                if (gy >= R && gy < ny - R && gx >= R && gx < nx - R) inyx |= 1u << (y * 4 + e);
            }
        // boundary mode of my warp: rows of the ring (or a lane holding both
        // ring sides) need per-cell masks; the ring's columns alone, a lane
        // predicate (R <= 4 columns, all inside the 4 cells of one lane)
        bool brow = false;
#pragma unroll
        for (int y = 0; y < VY; ++y) {
            const int gy = ys + my_row + y;
            brow |= (gy >= 0 && gy < R) || (gy >= ny - R && gy < ny);
        }
        xl = gx0 == 0;
        xr = gx0 == nx - 4;
        if (__any_sync(0xffffffffu, brow || (xl && xr))) wmode = kBndCells;
        else if (__any_sync(0xffffffffu, xl || xr)) wmode = kBndColumns;
        else wmode = kBndNone;
#pragma unroll
        for (int l = 0; l < K; ++l)
#pragma unroll
            for (int q = 0; q < W2; ++q)
#pragma unroll
                for (int y = 0; y < VY; ++y)
#pragma unroll
                    for (int h = 0; h < 2; ++h) A[l][q][y][h] = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < (K > 1 ? K - 1 : 1); ++l)
#pragma unroll
            for (int y = 0; y < VY; ++y)
#pragma unroll
                for (int h = 0; h < 2; ++h) C[l][y][h] = make_float2(0.f, 0.f);
        // stream over [za, zb): the outputs and the K*R planes each side
        const int in_lo = (int)a.in_lo, in_hi = (int)a.in_hi;
        za = zs - K * R > in_lo ? zs - K * R : in_lo;
        zb = ze + K * R < in_hi ? ze + K * R : in_hi;
        olo = need_lo = zs;
        ohi = need_hi = ze;
        // phases in which every level is active: level L handles arrival
        // za + p - L(R+1) in phase p
        ps_lo = 0;
        ps_hi = 1 << 30;
#pragma unroll
        for (int L = 0; L < K; ++L) {
            const int lo = lev_lo(L) - za + L * (R + 1), hi = lev_hi(L) - za + L * (R + 1);
            ps_lo = lo > ps_lo ? lo : ps_lo;
            ps_hi = hi < ps_hi ? hi : ps_hi;
        }
        // last arrival any level needs: level K-1 at plane need_hi + R - 1
        const int nph0 = (need_hi + R - 1 - za) + (K - 1) * (R + 1) + 1;
        const int nph = (nph0 + W2 - 1) / W2 * W2;
        // (the slots were last read through the generic proxy by the previous
        // piece, behind the barrier that ended it)
        if (threadIdx.x == 0) fence_proxy_async_smem();
        for (int q = 0; q < PD; ++q) {
            if constexpr (ZC) {
                if (host_plane(za + q)) stage_host(q);
                else if (threadIdx.x == 0) issue(q);
                cp_async_commit();
            } else if (threadIdx.x == 0) {
                issue(q);
            }
        }
        bool ok = true;
        for (int p0 = 0; p0 < nph && ok; p0 += W2) ok = phase<0>(p0);
        return ok;
    }

    __device__ __forceinline__ void run(unsigned char* smem) {
        bar0 = smem_u32(smem);
        sin = reinterpret_cast<const T*>(smem + S::kBarBytes);
        sin0 = bar0 + S::kBarBytes;
        slev = reinterpret_cast<float*>(smem + S::kBarBytes + NI * SLOT);
        lane = threadIdx.x & 31;
        warp = threadIdx.x >> 5;
        my_row = warp * VY;
        ny = (int)a.ny;
        nx = (int)a.nx;
        plane = a.ny * a.nx;
        n0 = (int)a.n0;
        out = static_cast<T*>(a.out);
        hin = static_cast<const T*>(a.host_in);
        hlo = ZC && hin ? (int)a.host_lo : 0;
        hhi = ZC && hin ? (int)a.host_hi : 0;
        gb = 0;
        par = 0;
        // this CTA's pieces.  Grid split: one tile and axis-0 segment.  Round
        // split (a.split = n segments per tile): the tiles x n units, segment-
        // major as the grid split orders them, are pieces 0 .. FG-1 (F whole
        // rounds of the G CTAs), and the U mod G units of the last, partial
        // round are each cut into floor(G / (U mod G)) pieces along axis 0
        // (pieces FG.., cut-major, so that pieces taken at the same time are
        // neighbouring tiles at the same planes).  The CTAs take the pieces
        // in order from the launch's counter (a.work_ctr), so that an SM that
        // finished a cheap piece takes the next one; without a counter CTA c
        // takes pieces c, c + G, c + 2G, ...  The constants of the
        // enumeration sit in shared memory (behind the mbarriers) and are
        // read again for every piece, so that they hold no registers while a
        // piece streams.
        volatile int* wk = reinterpret_cast<volatile int*>(smem + kWorkOff);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int i = 0; i < NI; ++i) mbar_init(bar0 + 8u * i, 1);
            fence_mbar_init();
            const int tiles_x = (nx + S::TX - 1) / S::TX;
            const int tiles = tiles_x * ((ny + S::TY - 1) / S::TY);
            const int nseg = a.split ? a.split : (int)gridDim.z;
            const int G = (int)gridDim.x, units = tiles * nseg;
            const int F = a.split ? units / G : 1;  // whole-unit rounds
            const int rem = a.split ? units - F * G : 0;
            const int jr = rem ? G / rem : 1;        // pieces per unit of the last round
            wk[0] = F * G;
            wk[1] = rem;
            wk[2] = jr;
            wk[3] = tiles_x;
            wk[4] = tiles;
            wk[5] = nseg;
            wk[6] = F * G + jr * rem;                 // pieces
        }
        __syncthreads();
        bool ok = true, ran = false;
        for (int i = 0;; ++i) {
            int v, k = 0, nk = 1;
            if (!a.split) {
                if (i > 0) break;
                v = (int)blockIdx.x + (int)blockIdx.y * wk[3] + (int)blockIdx.z * wk[4];
            } else {
                int u;
                if (a.work_ctr) {
                    if (threadIdx.x == 0) wk[7] = (int)atomicAdd(a.work_ctr, 1u);
                    __syncthreads();
                    u = wk[7];
                    __syncthreads();
                } else {
                    u = (int)blockIdx.x + i * (int)gridDim.x;
                }
                if (u >= wk[6]) break;
                const int FG = wk[0];
                if (u < FG) {
                    v = u;
                } else {
                    const int w = u - FG, rem = wk[1];
                    k = w / rem;
                    v = FG + w % rem;
                    nk = wk[2];
                }
            }
            const int tiles_x = wk[3], tiles = wk[4], nseg = wk[5];
            const int t = v % tiles, sg = v / tiles;
            const int64_t nout = a.out_hi - a.out_lo;
            const int s0 = (int)(nout * sg / nseg), s1 = (int)(nout * (sg + 1) / nseg);
            const int zs = (int)a.out_lo + s0 + (int)((int64_t)(s1 - s0) * k / nk);
            const int ze = (int)a.out_lo + s0 + (int)((int64_t)(s1 - s0) * (k + 1) / nk);
            if (ze <= zs) continue;
            if (ran) {
                // the next piece reuses the staging slots and level planes
                gb += zb - za;
                __syncthreads();
            }
            ok = piece(t % tiles_x, t / tiles_x, zs, ze);
            ran = true;
            if (!ok) break;
        }
        if (!ok) {
            // a copy did not land: report it and wait (bounded) for the
            // copies still in flight before the shared memory is released
            if (threadIdx.x == 0) {
                if (a.status) atomicOr(a.status, 1);
                // phases pfail .. pfail + PD - 1 were issued and not consumed
                unsigned pq = par;
                for (int q = pfail; q < pfail + PD && za + q < zb; ++q) {
                    if (ZC && host_plane(za + q)) continue;
                    const int g = (gb + q) % NI;
                    (void)mbar_wait_bounded(bar0 + (uint32_t)g * 8u, (pq >> g) & 1u);
                    pq ^= 1u << g;
                }
            }
            __syncthreads();
        }
        if constexpr (ZC) cp_async_wait_all();  // no cp.async copy outlives the CTA
        if (a.split && a.work_ctr && threadIdx.x == 0) {
            // the last CTA to finish (every other one has taken its last
            // piece) zeroes the counter for the next launch on this stream
            __threadfence();
            if (atomicAdd(a.work_ctr + 1, 1u) == gridDim.x - 1) {
                a.work_ctr[0] = 0u;
                a.work_ctr[1] = 0u;
                __threadfence();
            }
        }
    }
};

// ZC: the launch reads some input planes from the mapped host grid (zero-copy
// input); a separate instantiation, so that the launches of the copy-engine
// pipeline carry none of its code
template <typename T, int R, int K, bool ZC = false>
__global__ void __launch_bounds__(StarShape<R, K>::NT, StarShape<R, K>::MINB)
    star3d_tb_kernel(const StencilArgs a, const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(1024) unsigned char smem_tb[];
    StarTB<T, R, K, ZC> k(a, &tmap);
    k.run(smem_tb);
}

}  // namespace so2dr
