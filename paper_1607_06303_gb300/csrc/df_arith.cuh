// df_arith.cuh -- double-float (fp32 hi + lo) arithmetic and exact
// float64 <-> fp32 conversions by bit manipulation.
//
// GB300 issues float64 instructions, including float64 <-> fp32
// conversions, at about 1/64 of its fp32 rate.  Kernels whose float64 work
// is the bound run it instead on the fp32 pipes as double-float pairs
// (Dekker's exact product by FMA, Knuth's two-sum; about 2^-47 relative per
// operation), and move values between the two formats with integer
// operations only.
#pragma once

namespace signtri {

// x = hi + lo with hi its leading 24 significand bits and lo the next 29
// (rounded to 24), from x's bits.  Values outside fp32's exponent range
// (below 2^-126, from 2^128) give 0 and infinity.
__device__ __forceinline__ void split_df(double x, float &hi, float &lo)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7ff) - 1023;          // unbiased exponent
    if (e < -126 || e > 127) {
        hi = (e > 127) ? __int_as_float(((unsigned)(bits >> 32) & 0x80000000u) | 0x7f800000u) : 0.f;
        lo = 0.f;
        return;
    }
    const unsigned sign = (unsigned)(bits >> 32) & 0x80000000u;
    const unsigned long long mant = bits & 0xfffffffffffffull;  // 52 fraction bits
    hi = __int_as_float((int)(sign | ((unsigned)(e + 127) << 23) | (unsigned)(mant >> 29)));
    const unsigned mlo = (unsigned)(mant & 0x1fffffffull);       // the rest: mlo 2^(e - 52)
    float l = __uint2float_rn(mlo);
    const int el = e - 52;                                      // >= -178
    l = (el >= -126) ? __fmul_rn(l, __int_as_float((el + 127) << 23))
                     : __fmul_rn(__fmul_rn(l, __int_as_float((el + 127 + 64) << 23)), __int_as_float((127 - 64) << 23));
    lo = sign ? -l : l;
}

// x truncated to fp32 (its leading 24 significand bits; 0 below 2^-126,
// infinity from 2^128), from its bits
__device__ __forceinline__ float f64_to_f32_trunc(double x)
{
    float hi, lo;
    split_df(x, hi, lo);
    return hi;
}

// |x| as the bits of a non-negative float64: they order like the values,
// so maxima can be taken as integers
__device__ __forceinline__ unsigned long long abs_bits(double x)
{
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// The exponent e of frexp for a non-negative float64 given by its bits
// (m = f 2^e, f in [0.5, 1)); subnormals give -1022, zero gives 0
__device__ __forceinline__ int frexp_exp_of_bits(unsigned long long b)
{
    const int ef = (int)(b >> 52);
    return ef ? ef - 1022 : (b ? -1022 : 0);
}

// The float64 value of an fp32 x, assembled from its bits (exact).  Zeros
// and fp32 subnormals give 0; infinities and NaNs stay so.
__device__ __forceinline__ double f32_to_f64_bits(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0) return 0.0;
    const unsigned long long de = (e == 0xffu) ? 0x7ffull : (unsigned long long)(e - 127 + 1023);
    const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) | (de << 52) |
                                 ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}

// hi + lo in float64: one float64 addition of bit-converted operands
__device__ __forceinline__ double df_to_double(float hi, float lo)
{
    return __dadd_rn(f32_to_f64_bits(hi), f32_to_f64_bits(lo));
}

// (h, l) <- normalised pair of s + e (Dekker's fast two-sum, |s| >= |e|)
__device__ __forceinline__ void df_fast_norm(float s, float e, float &h, float &l)
{
    h = __fadd_rn(s, e);
    l = __fsub_rn(e, __fsub_rn(h, s));
}

// (h, l) = a * b, double-float (a_l b_l dropped)
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &h, float &l)
{
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    df_fast_norm(p, e, h, l);
}

// (h, l) = a + b, double-float (two-sum of the high parts)
__device__ __forceinline__ void df_add2(float ah, float al, float bh, float bl, float &h, float &l)
{
    const float s = __fadd_rn(ah, bh);
    const float bb = __fsub_rn(s, ah);
    const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
    df_fast_norm(s, __fadd_rn(err, __fadd_rn(al, bl)), h, l);
}

// (h, l) = c u + s v: one coordinate of a plane rotation, double-float
__device__ __forceinline__ void df_rot(float ch, float cl, float uh, float ul, float sh, float sl, float vh, float vl,
                                       float &h, float &l)
{
    float ph, pl, qh, ql;
    df_mul(ch, cl, uh, ul, ph, pl);
    df_mul(sh, sl, vh, vl, qh, ql);
    df_add2(ph, pl, qh, ql, h, l);
}

}  // namespace signtri
