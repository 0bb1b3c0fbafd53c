// kx_math.cuh -- table-driven FP64 log2 and exp for the per-point stage work.
//
// On this GPU the FP64 pipe runs at a small fraction of the FP32 rate, so the
// stage kernels' cost is the count of FP64 instructions on their dependent
// chains.  These two functions follow P. T. P. Tang's table-driven methods
// (ACM TOMS 15(2), 1989, for exp; ACM TOMS 16(4), 1990, for log): an exact
// argument reduction with integer exponent arithmetic, a table of 2^(j/64)
// or log2 F_k in double-double, and a short polynomial on a tiny interval.
// The tables are computed on the host in long double (kx_math_tables_init).
// Accuracy is absolute, which is what every caller needs: |error| <= ~2 ulp of
// the result's magnitude (checked against CUDA's log2/exp by kx_math_check).
#pragma once

#include <stdint.h>

// The including file (one translation unit) defines the tables before this
// header:
//   __device__ double4_32a g_kx_log2_tab[256];  k = top 8 bits of the significand,
//       F_k = 1 + k/256: (F_k, 1/F_k, log2 F_k high part, low part)
//   __device__ double2 g_kx_exp2_tab[64];   2^(j/64), high and low parts

// log2(x) = e + frac for normal x > 0: e the unbiased exponent, frac =
// log2(m) for the significand m in [1, 2) (frac in [0, 1], absolute error
// ~1e-17).  Callers pass x >= 1e-300 (normal, positive, finite).  tab: the
// table, or a copy of it in shared memory (the stage kernels take one before
// they wait for their predecessor, so the lookup is not an L2 round trip).
__device__ __forceinline__ void kx_log2_parts(double x, int &e, double &frac,
                                              const double4_32a *tab = g_kx_log2_tab) {
    const long long bits = __double_as_longlong(x);
    e = (int)((bits >> 52) & 0x7ff) - 1023;
    const long long mb = bits & 0x000fffffffffffffLL;
    const int k = (int)(mb >> 44);
    const double m = __longlong_as_double(mb | 0x3ff0000000000000LL);
    const double4_32a t = tab[k];
    // r = (m - F)/F: m - F is exact (Sterbenz), 0 <= r < 1/256 (r = 0 at m = F,
    // so log2 of a power of two is exact)
    const double r = (m - t.x) * t.y;
    // log2(1 + r) = (1/ln 2) sum_{j>=1} (-1)^(j+1) r^j / j, through r^7 (r^8/8 < 1e-20)
    const double c1 = 1.4426950408889634074, c2 = -0.72134752044448170368;
    const double c3 = 0.48089834696298780245, c4 = -0.36067376022224085184;
    const double c5 = 0.28853900817779268147, c6 = -0.24044917348149390123;
    const double c7 = 0.20609929155556620105;
    double p = fma(r, c7, c6);
    p = fma(r, p, c5);
    p = fma(r, p, c4);
    p = fma(r, p, c3);
    p = fma(r, p, c2);
    p = fma(r, p, c1);
    frac = t.z + fma(r, p, t.w);
}

__device__ __forceinline__ double kx_log2(double x) {
    int e;
    double fr;
    kx_log2_parts(x, e, fr);
    return (double)e + fr;
}

// exp(x): x = (N/64) ln 2 + r, N = rint(64 x / ln 2), |r| <= ln 2 / 128;
// exp(x) = 2^(N div 64) 2^((N mod 64)/64) exp(r), exp(r) - 1 by its Taylor
// series through r^6 (|r|^7/7! < 2e-20).  0 below -745.2, inf above 709.78.
__device__ __forceinline__ double kx_exp(double x) {
    if (!(x == x)) return x;
    if (x < -745.2) return 0.0;
    if (x > 709.78) return __longlong_as_double(0x7ff0000000000000LL);
    const double inv = 92.332482616893656768;       // 64 / ln 2
    const double l_hi = 0.01083042469326756;          // ln 2 / 64, 32 significant bits
    const double l_lo = 2.9815858269852933e-12;       // ln 2 / 64 - l_hi
    const double Nd = rint(x * inv);
    const int N = (int)Nd;
    const double r = fma(-Nd, l_lo, fma(-Nd, l_hi, x));
    double p = fma(r, 1.0 / 720.0, 1.0 / 120.0);
    p = fma(r, p, 1.0 / 24.0);
    p = fma(r, p, 1.0 / 6.0);
    p = fma(r, p, 0.5);
    p = fma(r * r, p, r);                              // exp(r) - 1
    const int j = N & 63, m = N >> 6;                  // arithmetic shift: floor(N / 64)
    const double2 t = g_kx_exp2_tab[j];
    const double y = t.x + fma(t.x, p, t.y);           // 2^(j/64) exp(r), in [0.99, 2)
    if (m >= -1021) return __longlong_as_double(__double_as_longlong(y) + ((long long)m << 52));
    // result below the normal range: scale in two steps
    return __longlong_as_double(__double_as_longlong(y) + ((long long)(m + 600) << 52)) *
           2.409919865102884e-181;                      // 2^-600
}
