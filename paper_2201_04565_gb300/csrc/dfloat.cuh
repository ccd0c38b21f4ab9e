// dfloat.cuh -- integer-pipe conversions and double-float arithmetic.
//
// On GB300 the FP64 pipe (and every conversion to or from a 64-bit type) runs
// at about 1/70 of the FP32 rate, so the spring arithmetic of the F32 and DF
// modes avoids it:
//   - positions (FP64) are converted to 64-bit fixed point value * 2^S with
//     integer bit operations (exact when |x| >= 2^(52-S), truncated to 2^-S
//     otherwise), so spring vectors are exact integer differences;
//   - fixed-point values are turned into floats, or into unevaluated sums
//     hi + lo of two floats ("double-float", 48 significant bits), with
//     integer bit operations;
//   - double-float sums and products use the error-free transformations of
//     Dekker (1971) and Knuth (TAOCP vol. 2): TwoSum, Fast2Sum, and TwoProd
//     via a fused multiply-add.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lsm_internal.h"

namespace lsm {

// x * 2^S as a signed 64-bit integer, truncated toward zero. Requires
// |x| < 2^(62-S); *over is set when that bound is violated (or x is not
// finite).
__device__ __forceinline__ long long dbl_to_fix(double x, int S, bool &over)
{
    // x 2^S = m53 2^(e - 1075 + S); with the 53-bit significand moved to the
    // top of a 64-bit word (m = m53 2^11) that is m >> (1086 - e - S), one
    // logical right shift (zero or subnormal x: a shift of 64 or more, 0)
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    const unsigned long long m = ((unsigned long long)b << 11) | 0x8000000000000000ULL;
    const int rs = 1086 - e - S;
    over |= rs < 2;  // |x| >= 2^(62-S) (also catches inf / nan)
    const unsigned long long f = rs >= 64 ? 0ull : (m >> (rs < 2 ? 2 : rs));
    return b < 0 ? -(long long)f : (long long)f;
}

// Float with the top 24 significant bits of u * 2^-S (u > 0), truncated;
// *rem receives the bits below them (u - value * 2^S).
__device__ __forceinline__ float ufix_top24(unsigned long long u, int S, unsigned long long &rem)
{
    const int t = 63 - __clzll((long long)u);  // index of the top bit
    unsigned long long m24;
    if (t >= 23) {
        m24 = u >> (t - 23);
        rem = u - (m24 << (t - 23));
    } else {
        m24 = u << (23 - t);
        rem = 0;
    }
    const int ex = t - S + 127;  // biased exponent of the result
    const unsigned bits = ((unsigned)ex << 23) | ((unsigned)m24 & 0x7FFFFFu);
    return ex > 0 ? __uint_as_float(bits) : 0.0f;
}

// v * 2^-S as a float (truncated to 24 bits).
__device__ __forceinline__ float fix_to_float(long long v, int S)
{
    if (v == 0) return 0.0f;
    unsigned long long rem;
    const unsigned long long u = (unsigned long long)(v < 0 ? -v : v);
    const float f = ufix_top24(u, S, rem);
    return v < 0 ? -f : f;
}

__device__ __forceinline__ ff fast_two_sum(float a, float b);

// v * 2^-S as a double-float (top 48 significant bits, truncated).
__device__ __forceinline__ ff fix_to_ff(long long v, int S)
{
    if (v == 0) return ff{0.0f, 0.0f};
    unsigned long long rem, rem2;
    const unsigned long long u = (unsigned long long)(v < 0 ? -v : v);
    const float h = ufix_top24(u, S, rem);
    const float l = rem ? ufix_top24(rem, S, rem2) : 0.0f;
    const ff r = fast_two_sum(h, l);
    return v < 0 ? ff{-r.hi, -r.lo} : r;
}

// v * 2^-S as a float via two 32-bit int->float conversions (fast path on
// sm_103a, unlike the 64-bit ones). p24 = 2^(24-S), p0 = 2^-S. Exact split:
// v = hi * 2^24 + lo with 0 <= lo < 2^24; one rounding in the final fma.
__device__ __forceinline__ float fix_to_float_i2f(long long v, float p24, float p0)
{
    const int hi = (int)(v >> 24);
    const int lo = (int)(v & 0xFFFFFFLL);
    return __fmaf_rn(__int2float_rn(hi), p24, __fmul_rn(__int2float_rn(lo), p0));
}

// Exact float -> double with integer operations (subnormals flush to zero).
__device__ __forceinline__ double f2d_bits(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xFFu;
    unsigned long long bits = (unsigned long long)(u >> 31) << 63;
    if (e == 0xFFu)
        bits |= (0x7FFull << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
    else if (e != 0)
        bits |= ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)bits);
}

// f2d_bits for the forces the integration takes, in fewer integer
// operations: the same double for every finite float (subnormals flush to a
// signed zero); an infinity or NaN, which only a step from positions already
// out of range can produce, gives a finite value of magnitude at least 2^128,
// so that the next step's fixed-point conversion reports the state as out of
// range (LSM_ENONFINITE).
__device__ __forceinline__ double f2d_force(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned ax = u & 0x7FFFFFFFu, sign = u & 0x80000000u;
    const bool tiny = ax < 0x00800000u;                                    // zero or subnormal
    const unsigned hi = tiny ? sign : (((ax >> 3) + (896u << 20)) | sign);  // exponent rebiased by 1023 - 127
    const unsigned lo = tiny ? 0u : (u << 29);
    return __hiloint2double((int)hi, (int)lo);
}

// f2d_force for a force held in units of 2^k: the float's value times 2^k
// as a double, the power of two folded into the exponent rebias
// (bias = (896 + k) << 20; 896 << 20 is f2d_force), so the unit costs
// nothing; zero and subnormals give a signed zero, non-finite values a
// finite value of at least 2^(128 + k), as in f2d_force.
__device__ __forceinline__ double f2d_force_scaled(float f, unsigned bias)
{
    const unsigned u = __float_as_uint(f);
    const unsigned ax = u & 0x7FFFFFFFu, sign = u & 0x80000000u;
    const bool tiny = ax < 0x00800000u;
    const unsigned hi = tiny ? sign : (((ax >> 3) + bias) | sign);
    const unsigned lo = tiny ? 0u : (u << 29);
    return __hiloint2double((int)hi, (int)lo);
}

// Double -> float with integer operations, truncating the significand
// (|x| below the float range gives a signed zero, above it infinity).
__device__ __forceinline__ float d2f_bits(double d)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu);
    const int fe = e - 1023 + 127;
    if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (((hi & 0xFFFFFu) | lo) ? 0x400000u : 0u));
    if (fe <= 0) return __uint_as_float(sign);
    if (fe >= 255) return __uint_as_float(sign | 0x7F800000u);
    return __uint_as_float(sign | ((unsigned)fe << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}

// isfinite for a double, from its exponent bits.
__device__ __forceinline__ bool dbl_finite_bits(double d)
{
    return ((unsigned)(__double_as_longlong(d) >> 32) & 0x7FF00000u) != 0x7FF00000u;
}

// Reciprocal square root estimate of a positive normal float: the hardware
// approximation (about 2^-22.9 relative; subnormal inputs flush to zero),
// which every caller refines by Newton steps.
__device__ __forceinline__ float rsqrt_approx(float a)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a));
    return y;
}

// -- error-free transformations and double-float arithmetic ----------------

__device__ __forceinline__ ff two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff{s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b)  // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return ff{p, __fmaf_rn(a, b, -p)};
}

// Accurate double-float addition (both parts through TwoSum).
__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    ff s = two_sum(a.hi, b.hi);
    const ff t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    ff p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// a * b without the final renormalisation: (p, e) with p = fl(a.hi b.hi)
// and |e| within a few units of 2^-24 |p|, a valid unevaluated sum for
// the callers that only multiply or add it further (the neglected a.lo b.lo
// is below 2^-46 relative, as in ff_mul).
__device__ __forceinline__ ff ff_mul_un(ff a, ff b)
{
    ff p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    return p;
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b)
{
    ff p = two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// a / b with one Newton correction of the single-precision quotient.
__device__ __forceinline__ ff ff_div(ff a, ff b)
{
    const float rb = __frcp_rn(b.hi);
    const float q1 = __fmul_rn(a.hi, rb);
    const ff r = ff_sub(a, ff_mul_f(b, q1));
    const float q2 = __fmul_rn(r.hi, rb);
    ff q = fast_two_sum(q1, q2);
    const ff r2 = ff_sub(a, ff_mul(b, q));
    return fast_two_sum(q.hi, __fadd_rn(q.lo, __fmul_rn(r2.hi, rb)));
}

// sqrt(a), a > 0, from the single-precision reciprocal square root and one
// double-float Newton correction.
__device__ __forceinline__ ff ff_sqrt(ff a)
{
    const float y = rsqrtf(a.hi);
    const float x = __fmul_rn(a.hi, y);
    const ff xx = two_prod(x, x);
    const ff d = ff_sub(a, xx);
    return fast_two_sum(x, __fmul_rn(d.hi, __fmul_rn(0.5f, y)));
}

// v * 2^-S as a double-float from two 24-bit chunks, v = h 2^24 + l with
// h = floor(v / 2^24) and 0 <= l < 2^24. For |v| < 2^48 both chunks convert
// exactly and do not overlap, so Fast2Sum returns RN(v 2^-S) and the exact
// remainder. Up to |v| < 2^55 the result is v rounded to about 2^-24
// relative (h rounds); beyond, h wraps. The callers choose S so that every
// spring that can still be intact (length up to its critical length) has
// |v| < 2^48, and a vector that rounds here is longer than every critical
// length, so the break test decides it the same way.
__device__ __forceinline__ ff fix_to_ff_i2f2(long long v, float p24, float p0)
{
    const int h = (int)__funnelshift_r((unsigned)v, (unsigned)(v >> 32), 24);  // v >> 24
    const float a = __fmul_rn(__int2float_rn(h), p24);
    const float b = __fmul_rn(__int2float_rn((int)((unsigned)v & 0xFFFFFFu)), p0);
    return fast_two_sum(a, b);
}

// The same value in units of 2^(24-S): v / 2^24 = h + l 2^-24, the high
// chunk converted without a scale factor and the low one scaled by the exact
// power 2^-24, joined by Fast2Sum. Every result equals fix_to_ff_i2f2's times
// 2^(S-24) exactly (scaling by a power of two commutes with the rounding),
// one multiplication fewer; the DF kernels keep their spring tables, forces
// and sample sums in this unit (see f2d_force_scaled).
__device__ __forceinline__ ff fix_to_ff_u24(long long v)
{
    const int h = (int)__funnelshift_r((unsigned)v, (unsigned)(v >> 32), 24);  // v >> 24
    const float a = __int2float_rn(h);
    const float b = __fmul_rn(__int2float_rn((int)((unsigned)v & 0xFFFFFFu)), 0x1p-24f);
    return fast_two_sum(a, b);
}

// a^2 for a double-float a.
__device__ __forceinline__ ff ff_sqr(ff a)
{
    ff p = two_prod(a.hi, a.hi);
    p.lo = __fmaf_rn(__fadd_rn(a.hi, a.hi), a.lo, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// 1 / sqrt(a), a > 0: the float estimate, one float Newton step, then one
// Newton step in double-float, y1 = y0 + y0 (1 - a y0^2) / 2 (relative error
// about 2^-46; the residual 1 - a y0^2 is formed exactly up to the final
// rounding because a y0^2 is within a few float ulps of 1).
__device__ __forceinline__ ff ff_rsqrt(ff a)
{
    float y0 = rsqrtf(a.hi);
    y0 = __fmul_rn(y0, __fmaf_rn(-0.5f * a.hi, __fmul_rn(y0, y0), 1.5f));
    const ff t = ff_mul(a, two_prod(y0, y0));
    const float rho = __fsub_rn(__fsub_rn(1.0f, t.hi), t.lo);
    return fast_two_sum(y0, __fmul_rn(__fmul_rn(0.5f, y0), rho));
}

// a^2 + b^2 for double-floats a, b: exact float squares of the high parts
// (TwoProd), one TwoSum, and the small terms in float (about 2^-46 relative).
__device__ __forceinline__ ff ff_norm2(ff a, ff b)
{
    const float p1 = __fmul_rn(a.hi, a.hi), e1 = __fmaf_rn(a.hi, a.hi, -p1);
    const float p2 = __fmul_rn(b.hi, b.hi), e2 = __fmaf_rn(b.hi, b.hi, -p2);
    const ff s = two_sum(p1, p2);
    float l = __fmaf_rn(__fadd_rn(a.hi, a.hi), a.lo, __fadd_rn(e1, e2));
    l = __fmaf_rn(__fadd_rn(b.hi, b.hi), b.lo, l);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, l));
}

// ff_norm2 without the final renormalisation: (hi, lo) with hi + lo = a^2 +
// b^2 to about 2^-46 relative, hi within a few float ulps of the sum (the
// callers only compare it with a bound or take its reciprocal square root).
__device__ __forceinline__ ff ff_norm2_un(ff a, ff b)
{
    const float p1 = __fmul_rn(a.hi, a.hi), e1 = __fmaf_rn(a.hi, a.hi, -p1);
    const float p2 = __fmul_rn(b.hi, b.hi), e2 = __fmaf_rn(b.hi, b.hi, -p2);
    const ff s = two_sum(p1, p2);
    float l = __fmaf_rn(__fadd_rn(a.hi, a.hi), a.lo, __fadd_rn(e1, e2));
    l = __fmaf_rn(__fadd_rn(b.hi, b.hi), b.lo, l);
    return ff{s.hi, __fadd_rn(s.lo, l)};
}

// a^2 + b^2 + c^2 in the same form as ff_norm2_un: exact float squares of
// the high parts (TwoProd), two TwoSums, the small terms in float.
__device__ __forceinline__ ff ff_norm3_un(ff a, ff b, ff c)
{
    const float p1 = __fmul_rn(a.hi, a.hi), e1 = __fmaf_rn(a.hi, a.hi, -p1);
    const float p2 = __fmul_rn(b.hi, b.hi), e2 = __fmaf_rn(b.hi, b.hi, -p2);
    const float p3 = __fmul_rn(c.hi, c.hi), e3 = __fmaf_rn(c.hi, c.hi, -p3);
    const ff s = two_sum(p1, p2);
    const ff t = two_sum(s.hi, p3);
    float l = __fmaf_rn(__fadd_rn(a.hi, a.hi), a.lo, __fadd_rn(__fadd_rn(e1, e2), e3));
    l = __fmaf_rn(__fadd_rn(b.hi, b.hi), b.lo, l);
    l = __fmaf_rn(__fadd_rn(c.hi, c.hi), c.lo, l);
    return ff{t.hi, __fadd_rn(__fadd_rn(t.lo, s.lo), l)};
}

// a > b for an unnormalised a and a double-float b: the sign of X + Y with
// X = fl(a.hi - b.hi), Y = fl(a.lo - b.lo), taken as the exact comparison
// X > -Y (the rounded sum fl(X + Y) has the sign of X + Y, so this is the
// same decision in one operation fewer). Near a tie a.hi - b.hi is exact
// (Sterbenz: the two lie within a factor 2), so the decision is resolved to
// the low parts' precision, about 2^-46 relative; far from a tie the high
// parts decide.
__device__ __forceinline__ bool ff_gt_un(ff a, ff b)
{
    return __fsub_rn(a.hi, b.hi) > __fsub_rn(b.lo, a.lo);
}

// The spring factor g = 1 - r0 / r from r^2 (double-float) and r0, with
// y = 1/r to about 2^-45: the hardware reciprocal square root estimate y0
// (relative error below 2^-22.9), the residual rho = 1 - r^2 y0^2, and one
// double-float Newton step, r0 / r = r0 y0 (1 + rho / 2), whose neglected
// term 3/8 rho^2 stays near 2^-45.2. With y0^2 = q + qe exactly (TwoProd),
// rho is three fused multiply-adds: 1 - r2.hi q is formed exactly before
// its one rounding (r2.hi q lies within about 2^-21.9 of 1), then the terms
// r2.hi qe and r2.lo q of order 2^-24 follow (r2.lo qe, below 2^-47, is
// dropped). The product r0.hi y0 = p is exact (TwoProd), so 1 - r0 y0 is
// exact up to the small terms summed in float. 1 - p.hi needs no TwoSum:
// Fast2Sum(1, -p.hi) is exact for every 0 < p.hi < 2^24, by Dekker's
// condition for p.hi <= 1, and above 1 because 1 - p.hi is then a multiple
// of ulp(p.hi) below 2^24 ulp(p.hi), so the subtraction is exact and the
// error term 0. *y receives 1/r.
__device__ __forceinline__ ff ff_spring_g(ff r2, ff r0, ff *y)
{
    const float y0 = rsqrt_approx(r2.hi);
    const ff q = two_prod(y0, y0);
    const float rho =
        __fmaf_rn(-r2.lo, q.hi, __fmaf_rn(-r2.hi, q.lo, __fmaf_rn(-r2.hi, q.hi, 1.0f)));
    const ff p = two_prod(r0.hi, y0);
    float t2 = __fmaf_rn(-r0.lo, y0, -p.lo);
    t2 = __fmaf_rn(-0.5f * p.hi, rho, t2);
    const ff s = fast_two_sum(1.0f, -p.hi);
    if (y) *y = fast_two_sum(y0, __fmul_rn(__fmul_rn(0.5f, y0), rho));
    return fast_two_sum(s.hi, __fadd_rn(s.lo, t2));
}

// 1 - a for a double-float a (exact TwoSum on the high part).
__device__ __forceinline__ ff ff_one_minus(ff a)
{
    ff s = two_sum(1.0f, -a.hi);
    return fast_two_sum(s.hi, __fsub_rn(s.lo, a.lo));
}

// Double-float addition with one TwoSum on the high parts (Dekker's form):
// absolute error within a few units of 2^-46 (|a| + |b|), enough for sums
// whose accuracy is judged against the largest term.
__device__ __forceinline__ ff ff_add_sloppy(ff a, ff b)
{
    const ff s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

// a + b for a float b.
__device__ __forceinline__ ff ff_add_f(ff a, float b)
{
    const ff s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

// a / b with a single correction of the float quotient (about 2^-44 relative).
__device__ __forceinline__ ff ff_div_fast(ff a, ff b)
{
    const float rb = __frcp_rn(b.hi);
    const float q0 = __fmul_rn(a.hi, rb);
    const ff r = ff_add_sloppy(a, ff_neg(ff_mul_f(b, q0)));
    return fast_two_sum(q0, __fmul_rn(r.hi, rb));
}

__device__ __forceinline__ bool ff_gt(ff a, ff b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

__device__ __forceinline__ double ff_to_double(ff a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }

}  // namespace lsm
