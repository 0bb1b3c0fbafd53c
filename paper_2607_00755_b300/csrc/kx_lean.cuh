// kx_lean.cuh -- arithmetic for the per-instance stage kernels of the FP32
// path, whose time on this part is set by the FP64 pipe.  Each FP64
// instruction of a warp (add, multiply, fused multiply-add, compare, or a
// conversion to or from float) holds its sub-partition's FP64 unit for about
// 64 cycles, against about one cycle for an FP32 or integer instruction.  So:
//   * conversions between float and double and the tests of doubles that the
//     stage needs (sign, finiteness, order) work on the IEEE-754 bit patterns
//     with integer instructions;
//   * sums, products and the logarithm that only have to be good to about 44
//     bits use double-float arithmetic: a value is the unevaluated sum hi + lo
//     of two floats (Dekker's and Knuth's error-free transformations).
// The sums and products below use the _rn intrinsics, which the compiler never
// contracts into fused multiply-adds: the error-free transformations rely on
// each operation being rounded on its own.
#pragma once

#include <stdint.h>

// ---------------------------------------------------------------- bit tests
__device__ __forceinline__ unsigned long long kx_bits(double x) {
    return (unsigned long long)__double_as_longlong(x);
}
// |x| as a bit pattern: for non-negative doubles the patterns order like the values
__device__ __forceinline__ unsigned long long kx_abs_bits(double x) {
    return kx_bits(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ bool kx_nonfinite(double x) { return kx_abs_bits(x) >= 0x7ff0000000000000ull; }
// x < 0 for a finite x (-0.0 is not negative)
__device__ __forceinline__ bool kx_negative(double x) {
    return (long long)kx_bits(x) < 0 && kx_abs_bits(x) != 0ull;
}
// A signed 64-bit key that orders like the doubles (finite or infinite, not
// NaN); -0.0 and +0.0 share the key 0.
__device__ __forceinline__ long long kx_order_key(double x) {
    const long long b = (long long)kx_bits(x);
    return b < 0 ? -(b & 0x7fffffffffffffffll) : b;
}
__device__ __forceinline__ bool kx_dlt(double a, double b) { return kx_order_key(a) < kx_order_key(b); }
__device__ __forceinline__ bool kx_dge(double a, double b) { return kx_order_key(a) >= kx_order_key(b); }

// ---------------------------------------------------------------- conversions
// float -> double, exact for every float (zeros, subnormals, infinities, NaNs).
__device__ __forceinline__ double kx_f2d(float x) {
    const uint32_t u = __float_as_uint(x);
    const unsigned long long s = (unsigned long long)(u >> 31) << 63;
    const uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    unsigned long long r;
    if (e == 0xffu) {
        r = 0x7ff0000000000000ull | ((unsigned long long)m << 29);
    } else if (e != 0u) {
        r = ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
    } else if (m == 0u) {
        r = 0ull;
    } else {
        // subnormal: m 2^-149 with its leading bit at position p < 23
        const int p = 31 - __clz((int)m);
        r = ((unsigned long long)(p - 149 + 1023) << 52) |
            (((unsigned long long)m << (52 - p)) & 0x000fffffffffffffull);
    }
    return __longlong_as_double((long long)(s | r));
}

// x 2^s rounded to the nearest float (ties to even), for results in the float
// normal range; results below 2^-126 (and double subnormals) become a zero of
// x's sign, results above the largest float an infinity; NaN stays NaN.
// (s only moves the exponent, so the scaling itself is exact.)
__device__ __forceinline__ float kx_d2f_pow2(double x, int s) {
    const unsigned long long b = kx_bits(x);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const unsigned long long mag = b & 0x7fffffffffffffffull;
    const unsigned long long frac = mag & 0x000fffffffffffffull;
    const int ex = (int)(mag >> 52);
    if (ex == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (frac ? 0x400000u : 0u));
    if (ex == 0) return __uint_as_float(sign);
    const int fe = ex - 1023 + s;
    if (fe < -126) return __uint_as_float(sign);
    if (fe > 127) return __uint_as_float(sign | 0x7f800000u);
    // round the 52 fraction bits to 23 (nearest, ties to even); a carry out of
    // the fraction raises the exponent, up to the infinity pattern
    const unsigned long long rr = (frac + 0x0fffffffull + ((frac >> 29) & 1ull)) >> 29;
    return __uint_as_float(sign | (((uint32_t)(fe + 127) << 23) + (uint32_t)rr));
}
__device__ __forceinline__ float kx_d2f(double x) { return kx_d2f_pow2(x, 0); }

// x 2^s: exponent arithmetic on the bit pattern for a normal x whose result
// stays normal; other inputs (zeros, subnormals, over- or underflow) take
// CUDA's ldexp.
__device__ __forceinline__ double kx_ldexp_bits(double x, int s) {
    const unsigned long long b = kx_bits(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex > 0 && ex < 0x7ff && ex + s > 0 && ex + s < 0x7ff)
        return __longlong_as_double((long long)(b + ((unsigned long long)(long long)s << 52)));
    return ldexp(x, s);
}

// ---------------------------------------------------------------- double-float
struct kx_df {
    float hi, lo;
};

// Knuth's TwoSum: s + e == a + b exactly (any order of magnitude)
__device__ __forceinline__ void kx_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}
// Dekker's Fast2Sum (|a| >= |b| or a == 0): s + e == a + b exactly
__device__ __forceinline__ kx_df kx_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return kx_df{s, __fsub_rn(b, __fsub_rn(s, a))};
}
// a + b, about 44 significant bits
__device__ __forceinline__ kx_df kx_df_add(kx_df a, kx_df b) {
    float s, e;
    kx_two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return kx_fast_two_sum(s, e);
}
__device__ __forceinline__ kx_df kx_df_neg(kx_df a) { return kx_df{-a.hi, -a.lo}; }
// a b: the product of the high parts exactly (fused multiply-add), the cross terms rounded
__device__ __forceinline__ kx_df kx_df_mul(kx_df a, kx_df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return kx_fast_two_sum(p, e);
}
// the nearest float to hi + lo
__device__ __forceinline__ float kx_df_round(kx_df a) { return __fadd_rn(a.hi, a.lo); }
// hi + lo as a double (exact: the two floats' significands fit in 53 bits when
// |lo| <= ulp(hi), as the normalised results above are); one FP64 add
__device__ __forceinline__ double kx_df_to_double(kx_df a) { return kx_f2d(a.hi) + kx_f2d(a.lo); }
// The double-float nearest x (FP64 arithmetic: for values made outside the
// stage's critical path, e.g. before its wait for the predecessor kernel)
__device__ __forceinline__ kx_df kx_df_of(double x) {
    const float hi = (float)x;
    return kx_df{hi, (float)(x - (double)hi)};
}

// ---------------------------------------------------------------- log2
// 1/ln 2 as a double-float (hi = RN_float(1/ln 2), lo = RN_float(1/ln 2 - hi))
#define KX_INVLN2_HI 0x1.715476p+0f
#define KX_INVLN2_LO 0x1.4ae0c0p-26f

// log2 x = e + fr for a positive normal double x (the caller floors x): e its
// binary exponent, fr = log2 m of its significand m in [1, 2) as a
// double-float.  With F_k = 1 + k/256 (k the top 8 fraction bits),
// log2 m = log2 F_k + log2(1 + r), r = (m - F_k)/F_k in [0, 2^-8), and
// log2(1 + r) = (r - r^2/2 + r^3/3 - r^4/4 + r^5/5) / ln 2 + O(r^6) (the r^6 term
// is below 1e-15): the first two terms in double-float, the rest (below 3e-8)
// in float.  The absolute error of fr is below about 2e-14.
// tab[k] = (1/F_k as hi, lo; log2 F_k as hi, lo).
__device__ __forceinline__ void kx_log2_df(double x, int &e, kx_df &fr, const float4 *tab) {
    const unsigned long long b = kx_bits(x);
    e = (int)((b >> 52) & 0x7ff) - 1023;
    const unsigned long long mb = b & 0x000fffffffffffffull;
    const int k = (int)(mb >> 44);
    // m - F_k = (mb mod 2^44) 2^-52 = u 2^-31 + w 2^-52 with u < 2^23, w < 2^21:
    // each is 1 + v 2^-23 - 1 (exact) scaled by a power of two
    const uint32_t u = (uint32_t)((mb >> 21) & 0x7fffffull), w = (uint32_t)(mb & 0x1fffffull);
    const float dh = __fmul_rn(__fsub_rn(__uint_as_float(0x3f800000u | u), 1.f), 0x1p-8f);
    const float dl = __fmul_rn(__fsub_rn(__uint_as_float(0x3f800000u | w), 1.f), 0x1p-29f);
    const float4 t = tab[k];
    const kx_df r = kx_df_mul(kx_df{dh, dl}, kx_df{t.x, t.y});
    const kx_df c1 = {KX_INVLN2_HI, KX_INVLN2_LO};
    const kx_df c1r = kx_df_mul(c1, r);
    // c1 r^2 / 2 (the halving is exact)
    const kx_df q = kx_df_mul(c1r, r);
    const kx_df q2 = {__fmul_rn(q.hi, 0.5f), __fmul_rn(q.lo, 0.5f)};
    const float r1 = r.hi;
    const float tail = __fmul_rn(__fmul_rn(__fmul_rn(r1, r1), r1),
                                 fmaf(r1, fmaf(r1, 0x1.2776c6p-2f, -0x1.715476p-2f), 0x1.ec709ep-2f));
    kx_df p = kx_df_add(c1r, kx_df_neg(q2));
    p = kx_df_add(p, kx_df{tail, 0.f});
    fr = kx_df_add(kx_df{t.z, t.w}, p);
}
