// Double-FP32 ("double-float") arithmetic on the FP32 units, for FP64-accuracy results on
// GB300, whose FP64 units retire about 2 FMA per SM per clock (64 times fewer than FP32).
//
// A value is an unevaluated sum hi + lo of two floats.  FP64 operands are split exactly with
// integer instructions (hi = the 24 leading significand bits, lo = the next 29 bits rounded to
// 24, i.e. 47 bits kept); products are error-free with FMA (TwoProduct, Ogita-Rump-Oishi
// 2005), sums with Knuth's TwoSum; results are rounded to FP64 once.  Magnitudes below 2^-126
// are flushed to zero and below 2^-74 lose their lo part (a relative error of 2^-24 on values
// that small, far below the FP64 rounding of the unit-scale results they enter).
#pragma once

#include <cuda_runtime.h>

struct ff {
    float hi, lo;
};

static __device__ __noinline__ ff ff_split_slow(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
    const int e = (int)((h32 >> 20) & 0x7FFu);
    const unsigned sign = h32 & 0x80000000u;
    ff r;
    if (e < 897) { r.hi = 0.f; r.lo = 0.f; return r; }
    if (e > 1150) { r.hi = __int_as_float((int)(sign | 0x7F800000u)); r.lo = 0.f; return r; }
    r.hi = __int_as_float((int)(sign | ((unsigned)(e - 896) << 23) | ((h32 & 0xFFFFFu) << 3) | (l32 >> 29)));
    if (e < 949) { r.lo = 0.f; return r; }
    const float scale = __int_as_float((e - 948) << 23);  // 2^(e - 1075)
    const float lo = __fmul_rn(__uint2float_rn(l32 & 0x1FFFFFFFu), scale);
    r.lo = __int_as_float(__float_as_int(lo) | (int)sign);
    return r;
}

// Same split on the common path, in about a dozen integer instructions: with t the high word
// minus the exponent rebias (float exponent field ef in bits 20..27 when in range),
// hi = sign | ((t:l32) >> 29) (one funnel shift gives exponent and the 23 leading fraction
// bits), lo = (the 29 remaining fraction bits) * 2^(ef - 179).  Magnitudes outside
// [2^-74, 2^128) take the exact slow path above.
__device__ __forceinline__ ff ff_split(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
    const unsigned sign = h32 & 0x80000000u;
    const unsigned t = (h32 & 0x7FFFFFFFu) - (896u << 20);
    const unsigned ef = t >> 20;
    if (ef - 53u > 201u) return ff_split_slow(x);
    ff r;
    r.hi = __int_as_float((int)(__funnelshift_r(l32, t, 29) | sign));
    const float scale = __int_as_float((int)((ef - 52u) << 23));
    const float lo = __fmul_rn(__uint2float_rn(l32 & 0x1FFFFFFFu), scale);
    r.lo = __int_as_float(__float_as_int(lo) | (int)sign);
    return r;
}

// a*b ~ p + e exactly up to the dropped lo*lo term.
__device__ __forceinline__ void ff_two_prod(ff a, ff b, float &p, float &e) {
    p = __fmul_rn(a.hi, b.hi);
    e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
}

// a * z for a float z (exact product of a.hi and z, plus a.lo * z).
__device__ __forceinline__ void ff_prod_f(ff a, float z, float &p, float &e) {
    p = __fmul_rn(a.hi, z);
    e = __fmaf_rn(a.hi, z, -p);
    e = __fmaf_rn(a.lo, z, e);
}

// (s, c) += x with the rounding error of s + x folded into c (TwoSum).
__device__ __forceinline__ void ff_acc_add(float &s, float &c, float x) {
    const float t = __fadd_rn(s, x);
    const float z = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(x, z));
    s = t;
    c = __fadd_rn(c, err);
}

__device__ __forceinline__ void ff_acc_prod(float &s, float &c, float p, float e) {
    ff_acc_add(s, c, p);
    c = __fadd_rn(c, e);
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float z = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, z)), __fsub_rn(b.hi, z));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    ff r;
    r.hi = __fadd_rn(s, e);
    r.lo = __fsub_rn(e, __fsub_rn(r.hi, s));
    return r;
}

__device__ __forceinline__ ff ff_norm(float s, float c) {
    ff r;
    r.hi = __fadd_rn(s, c);
    r.lo = __fsub_rn(c, __fsub_rn(r.hi, s));
    return r;
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }

__device__ __forceinline__ double ff_to_double(ff v) { return (double)v.hi + (double)v.lo; }
