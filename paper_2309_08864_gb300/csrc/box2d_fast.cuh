// box2d_fast.cuh -- register-streaming temporal-blocking kernel for 2D box
// stencils ((2R+1)^2 points, radius R, K fused steps per launch), FP32
// arithmetic on FP32 / BF16 / FP16 storage.
//
// The on-chip temporal blocking of Sec. III / Sec. IV-A for the paper's
// box2d workloads (Table III), laid out for sm_103a:
//  * a CTA owns a strip of 1024 columns (256 threads x 4 columns) and streams
//    the rows of axis 0 through it; axis 0 may be split into segments
//    (gridDim.z) so that the grid fills the SMs;
//  * each input row is read from device memory once: cp.async copies
//    (zero-fill outside the grid) stage it PD rows ahead in shared memory,
//    so that enough bytes are in flight to cover the DRAM latency even at
//    depth 1; a thread reads its x window (its 4 columns and R on each side)
//    with three aligned vector loads from a padded shared-memory row;
//  * every fused level keeps 2R partial sums per cell in registers: when
//    the level below produces row y', the row's (2R+1)-tap products are added
//    into the targets y'-R..y'+R (one coefficient row each) and target y'-R
//    is complete.  The slot of a target is fixed by its row index modulo 2R
//    and the row loop is unrolled 2R times, so the ring never moves data;
//  * cells go in x pairs through packed FP32x2 FMAs; the pairs that start at
//    an odd column are packed once per arriving row and serve all 2R+1
//    targets;
//  * levels are pipelined across rows (level l consumes what level l-1
//    completed in the previous phase: one barrier per row), and each level
//    keeps R+2 rows in shared memory: the arrival, the row being written,
//    and the R older rows from which boundary cells take back their value;
//  * per cell the products are summed in one fixed order, row by row from
//    offset (-R, -R), the first one a plain multiply -- the order of the
//    generic kernel -- so every launch, tile and chunk rounds identically.
#pragma once

#include "stencil.cuh"
#include "tb_common.cuh"

namespace so2dr {

template <int R, int K> struct BoxShape {
    static constexpr int VX = 4;                       // columns per thread
    static constexpr int NT = 256;                     // threads per CTA
    static constexpr int LX = NT * VX;                 // staged columns per row
    static constexpr int HXA = ((R * K + 3) / 4) * 4;  // halo per side, whole vectors
    static constexpr int TX = LX - 2 * HXA;            // output columns per CTA
    static constexpr int PAD = 4;                      // spare elements each side of a row
    static constexpr int ROW = LX + 2 * PAD;
    static constexpr int NB = R + 2;                   // row slots per level
    static constexpr int PD = 4;                       // input rows staged ahead
    static constexpr int NBI = R + 1 + PD;             // input row slots
    template <int ES> static constexpr int smem() { return NBI * ROW * ES + NB * (K - 1) * ROW * 4; }
    // two CTAs per SM (at most 128 registers a thread), so that one CTA's
    // barrier waits are hidden by the other's work; radius >= 3 at R*K >= 8
    // would spill under that cap and keeps one
    static constexpr int MINB = (R >= 3 && R * K >= 8) ? 1 : 2;
    static_assert(MINB == 1 || 2 * (smem<4>() + 1024) <= 228 * 1024, "two CTAs must fit an SM's shared memory");
};

template <typename T, int R, int K>
struct FastBox {
    using S = BoxShape<R, K>;
    static constexpr int NT = S::NT, LX = S::LX, ROW = S::ROW, PAD = S::PAD, NB = S::NB, PD = S::PD,
                         NBI = S::NBI;
    static constexpr int W2 = 2 * R, WD = 2 * R + 1;
    static constexpr int NF = 12;  // window: columns -4..7 around my first column
    // accumulation loop order (same results): column offset outer for small
    // R*K, target outer for larger ones (measured on 16384^2: offset-outer
    // 14-28% faster up to R*K = 4, 2-15% slower from 8)
    static constexpr bool kOffsetOuter = R * K <= 4;

    const StencilArgs& a;
    T* sin;       // [NBI][ROW] staged input rows (row of phase p in slot p % NBI)
    float* slev;  // [K-1][NB][ROW] completed rows of levels 0..K-2
    int tid, n0, nx, olo, ohi, need_lo, need_hi, xs, gx0, za, zb, slot_next;
    int ps_lo, ps_hi;  // phases in which every level is active
    bool xin, warp_bnd;
    unsigned inx;  // bit e: my column e is an interior column
    const T* in;
    T* out;
    float2 A[K][W2][2];  // 2R partial sums per cell per level, in x pairs

    __device__ __forceinline__ explicit FastBox(const StencilArgs& args) : a(args) {}

    // one commit group per call (empty past the input, where the slot keeps
    // stale data that only phantom targets see), so that waiting for all but
    // the newest PD - 1 groups always means: this phase's row has landed
    __device__ __forceinline__ void stage_row(int z, int b) {
        if (z < zb) {
            cp_async_vec4(sin + b * ROW + PAD + 4 * tid, xin ? in + (int64_t)slot_next * nx + gx0 : in, xin);
            if (++slot_next == a.in_cap) slot_next = 0;
        }
        cp_async_commit();
    }

    // one arrival at level L (phase PH = (row - za) mod 2R): f holds the
    // arriving row's columns -4..7 around my first column
    template <int L, int PH>
    __device__ __forceinline__ void arrive(const float (&f)[NF], float2 (&done)[2]) {
        // pair starting at window index j (column j - 4 and the next)
        float2 P[NF - 1];
#pragma unroll
        for (int j = 4 - R; j <= 6 + R; ++j) P[j] = make_float2(f[j], f[j + 1]);
        // target q (q = 0..2R) is row y' - R + q, its slot (PH - R + q) mod 2R;
        // this arrival is its coefficient row 2R - q; target 2R (row y' + R)
        // starts in the slot target 0 leaves.  Every target adds its products
        // in ascending column order whichever loop is outer.
        if constexpr (kOffsetOuter) {
            // column offset outer: the 2(2R+1) accumulators of one step are
            // independent (faster while R*K <= 4 leaves the registers for it)
            float2 acc[W2 + 1][2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
                for (int q = 0; q < W2; ++q) acc[q][h] = A[L][pmod(PH - R + q, W2)][h];
                acc[W2][h] = __fmul2_rn(a.cf2[0], P[2 * h - R + 4]);
            }
#pragma unroll
            for (int dx = -R; dx <= R; ++dx)
#pragma unroll
                for (int q = 0; q <= W2; ++q)
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        if (q < W2 || dx > -R)
                            acc[q][h] = __ffma2_rn(a.cf2[(W2 - q) * WD + dx + R], P[2 * h + dx + 4], acc[q][h]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                done[h] = acc[0][h];
#pragma unroll
                for (int q = 1; q < W2; ++q) A[L][pmod(PH - R + q, W2)][h] = acc[q][h];
                A[L][pmod(PH - R, W2)][h] = acc[W2][h];
            }
        } else {
            // target outer: one accumulator chain at a time (fewer live registers)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
                for (int q = 0; q < W2; ++q) {
                    float2& acc = A[L][pmod(PH - R + q, W2)][h];
                    float2 s2 = acc;
#pragma unroll
                    for (int dx = -R; dx <= R; ++dx)
                        s2 = __ffma2_rn(a.cf2[(W2 - q) * WD + dx + R], P[2 * h + dx + 4], s2);
                    if (q == 0) done[h] = s2;
                    else acc = s2;
                }
                float2 s2 = __fmul2_rn(a.cf2[0], P[2 * h - R + 4]);
#pragma unroll
                for (int dx = -R + 1; dx <= R; ++dx) s2 = __ffma2_rn(a.cf2[dx + R], P[2 * h + dx + 4], s2);
                A[L][pmod(PH - R, W2)][h] = s2;
            }
        }
    }

    // boundary cells keep their value: on completion they take back the
    // value they had at their centre arrival, R phases ago (slot `cen`)
    template <typename ST>
    __device__ __forceinline__ void fixup(float2 (&done)[2], int zt, const ST* cen) {
        const bool zbnd = zt < R || zt >= n0 - R;
        if (!(zbnd || warp_bnd)) return;
        if (zbnd || inx != 0xFu) {
            const float4 q = lds4(cen + PAD + 4 * tid);
            if (zbnd || !(inx & 1u)) done[0].x = q.x;
            if (zbnd || !(inx & 2u)) done[0].y = q.y;
            if (zbnd || !(inx & 4u)) done[1].x = q.z;
            if (zbnd || !(inx & 8u)) done[1].y = q.w;
        }
    }

    __device__ __forceinline__ void emit(const float2 (&done)[2], int zt) {
        if (zt < olo || zt >= ohi) return;
        const int lx0 = 4 * tid;
        if (!(lx0 >= S::HXA && lx0 < S::HXA + S::TX && xin)) return;
        st4(out + (int64_t)(zt - (int)a.out_lo) * nx + gx0, make_float4(done[0].x, done[0].y, done[1].x, done[1].y));
    }

    template <typename ST>
    __device__ __forceinline__ void window(const ST* row, float (&f)[NF]) {
        const ST* p = row + PAD + 4 * tid - 4;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float4 q = lds4(p + 4 * i);
            f[4 * i] = q.x;
            f[4 * i + 1] = q.y;
            f[4 * i + 2] = q.z;
            f[4 * i + 3] = q.w;
        }
    }

    // level L of phase p (PH = p mod 2R): consumes input row za + p (L = 0)
    // or what level L-1 completed in phase p-1 (row za + p - L(R+1))
    // (ALL: a phase in which every level is active, run as straight-line code)
    template <int L, int PH, bool ALL>
    __device__ __forceinline__ void level(int p, const T* sbuf, int buf) {
        if constexpr (ALL) {
            level_body<L, PH>(p, sbuf, buf);
        } else {
            const int zp = za + p - L * (R + 1);
            const int lo = need_lo - (K - L) * R, hi = need_hi + (K - L) * R;
            if (!(zp < za || zp < lo || zp >= hi)) level_body<L, PH>(p, sbuf, buf);
        }
        if constexpr (L + 1 < K) level<L + 1, PH, ALL>(p, sbuf, buf);
    }

    template <int L, int PH>
    __device__ __forceinline__ void level_body(int p, const T* sbuf, int buf) {
        const int zp = za + p - L * (R + 1);
        float f[NF];
        float2 done[2];
        const int zt = zp - R;
        if constexpr (L == 0) {
            window(sbuf, f);
            arrive<0, PH>(f, done);
            fixup(done, zt, sin + ((p - R + NBI * R) % NBI) * ROW);
        } else {
            window(slev + ((L - 1) * NB + (p - 1 + NB) % NB) * ROW, f);
            arrive<L, pmod(PH - L * (R + 1), W2)>(f, done);
            fixup(done, zt, slev + ((L - 1) * NB + (p - 1 - R + NB * (R + 1)) % NB) * ROW);
        }
        if constexpr (L == K - 1) {
            emit(done, zt);
        } else {
            *reinterpret_cast<float4*>(slev + (L * NB + buf) * ROW + PAD + 4 * tid) =
                make_float4(done[0].x, done[0].y, done[1].x, done[1].y);
        }
    }

    template <int PH>
    __device__ __forceinline__ void phase(int p0) {
        const int p = p0 + PH;
        asm volatile("cp.async.wait_group %0;\n" ::"n"(PD - 1) : "memory");
        __syncthreads();
        // slot (p + PD) % NBI last held row p + PD - NBI = p - R - 1, whose
        // last reader (the level-0 fixup of phase p - 1) is behind the barrier
        stage_row(za + p + PD, (p + PD) % NBI);
        if (p >= ps_lo && p < ps_hi) level<0, PH, true>(p, sin + (p % NBI) * ROW, p % NB);
        else level<0, PH, false>(p, sin + (p % NBI) * ROW, p % NB);
        if constexpr (PH + 1 < W2) phase<PH + 1>(p0);
    }

    __device__ __forceinline__ void run(void* smem) {
        sin = reinterpret_cast<T*>(smem);
        slev = reinterpret_cast<float*>(smem) + (NBI * ROW * sizeof(T)) / 4;
        tid = threadIdx.x;
        nx = (int)a.nx;
        n0 = (int)a.n0;
        xs = (int)blockIdx.x * S::TX - S::HXA;
        gx0 = xs + 4 * tid;
        xin = gx0 >= 0 && gx0 < nx;  // nx % 4 == 0: a vector is all in or all out
        in = static_cast<const T*>(a.in);
        out = static_cast<T*>(a.out);
        inx = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (gx0 + e >= R && gx0 + e < nx - R) inx |= 1u << e;
        warp_bnd = __any_sync(0xffffffffu, inx != 0xFu);
        // the row pads feed only cells outside every level's valid columns;
        // zero them so that nothing there is undefined
        for (int i = tid; i < NBI * 2 * PAD; i += NT) {
            const int row = i / (2 * PAD), k = i % (2 * PAD);
            sin[row * ROW + (k < PAD ? k : LX + k)] = T(0.f);
        }
        for (int i = tid; i < (K - 1) * NB * 2 * PAD; i += NT) {
            const int row = i / (2 * PAD), k = i % (2 * PAD);
            slev[row * ROW + (k < PAD ? k : LX + k)] = 0.f;
        }
#pragma unroll
        for (int l = 0; l < K; ++l)
#pragma unroll
            for (int q = 0; q < W2; ++q)
#pragma unroll
                for (int h = 0; h < 2; ++h) A[l][q][h] = make_float2(0.f, 0.f);
        // axis-0 segment of this CTA: outputs [zs, ze), stream over [za, zb)
        const int nseg = gridDim.z;
        const int nout = (int)(a.out_hi - a.out_lo), in_lo = (int)a.in_lo, in_hi = (int)a.in_hi;
        const int zs = (int)a.out_lo + (int)((int64_t)nout * blockIdx.z / nseg);
        const int ze = (int)a.out_lo + (int)((int64_t)nout * (blockIdx.z + 1) / nseg);
        za = zs - K * R > in_lo ? zs - K * R : in_lo;
        zb = ze + K * R < in_hi ? ze + K * R : in_hi;
        olo = need_lo = zs;
        ohi = need_hi = ze;
        slot_next = (int)((a.in_slot0 + (za - in_lo)) % a.in_cap);
        // phases in which every level is active: level L handles arrival
        // za + p - L(R+1) in phase p, and needs arrivals from
        // max(za, need_lo - (K-L)R) to need_hi + (K-L)R
        ps_lo = 0;
        ps_hi = 1 << 30;
#pragma unroll
        for (int L = 0; L < K; ++L) {
            const int llo = need_lo - (K - L) * R;
            const int lo = (llo > za ? llo : za) - za + L * (R + 1);
            const int hi = need_hi + (K - L) * R - za + L * (R + 1);
            ps_lo = lo > ps_lo ? lo : ps_lo;
            ps_hi = hi < ps_hi ? hi : ps_hi;
        }
        // last arrival any level needs: level K-1 at row need_hi + R - 1
        const int nph0 = (need_hi + R - 1 - za) + (K - 1) * (R + 1) + 1;
        const int nph = (nph0 + W2 - 1) / W2 * W2;
        for (int i = 0; i < PD; ++i) stage_row(za + i, i);
        for (int p0 = 0; p0 < nph; p0 += W2) phase<0>(p0);
        cp_async_wait_all();
    }
};

template <typename T, int R, int K>
__global__ void __launch_bounds__(BoxShape<R, K>::NT, BoxShape<R, K>::MINB) box2d_fast_kernel(const StencilArgs a) {
    extern __shared__ float4 smem4[];
    FastBox<T, R, K> k(a);
    k.run(smem4);
}

}  // namespace so2dr
