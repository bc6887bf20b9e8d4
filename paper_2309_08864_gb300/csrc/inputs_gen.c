/*
 * inputs_gen.c -- seeded synthetic inputs shared by the tests, the smoke check
 * and the benchmark.  Holds no stencil arithmetic.
 *
 * Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014), used counter-style so that any cell can be
 * drawn on its own: the draw for linear index i of stream `seed` is
 *     x_i = mix64(seed * 2^40 + (i + 1) * 0x9E3779B97F4A7C15)
 * with the published SplitMix64 finaliser mix64.  A uniform double in [0, 1)
 * is (x_i >> 11) * 2^-53; it is mapped to [a, b) as a + (b - a) * u and, for
 * FP32 output, rounded to nearest-even.  Normal draws use Box-Muller on the
 * draws 2i and 2i+1 of the stream.
 *
 * The linear index is the row-major index of the cell in the FULL grid, so a
 * sub-box [lo, hi) gets exactly the values the full grid holds there.
 */
#include <math.h>
#include <stdint.h>

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline double unit_draw(uint64_t seed, uint64_t i) {
    uint64_t x = mix64((seed << 40) + (i + 1) * 0x9E3779B97F4A7C15ULL);
    return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

/* dims/lo/hi have 3 entries (2D grids pass n2 = 1, lo2 = 0, hi2 = 1).
 * dist 0: uniform [a, b); dist 1: normal with mean a and deviation b.
 * out_kind 0: double, 1: float. */
void so2dr_gen_box(uint64_t seed, const int64_t* dims, const int64_t* lo, const int64_t* hi,
                   int dist, double a, double b, int out_kind, void* out) {
    int64_t e0 = hi[0] - lo[0], e1 = hi[1] - lo[1], e2 = hi[2] - lo[2];
#pragma omp parallel for schedule(static)
    for (int64_t i0 = 0; i0 < e0; ++i0) {
        for (int64_t i1 = 0; i1 < e1; ++i1) {
            int64_t gbase = ((lo[0] + i0) * dims[1] + (lo[1] + i1)) * dims[2] + lo[2];
            int64_t obase = (i0 * e1 + i1) * e2;
            for (int64_t i2 = 0; i2 < e2; ++i2) {
                uint64_t g = (uint64_t)(gbase + i2);
                double v;
                if (dist == 0) {
                    v = a + (b - a) * unit_draw(seed, g);
                } else {
                    double u1 = unit_draw(seed, 2 * g), u2 = unit_draw(seed, 2 * g + 1);
                    double rad = sqrt(-2.0 * log(1.0 - u1));
                    v = a + b * rad * cos(6.283185307179586 * u2);
                }
                if (out_kind == 0) ((double*)out)[obase + i2] = v;
                else ((float*)out)[obase + i2] = (float)v;
            }
        }
    }
}
