// Double-float ("FP32 pair") arithmetic for the mixed path (no paper
// counterpart: the paper computes in FP64).
//
// GB300 executes FP32 about 62x faster than FP64 (74.5 vs 1.19 TFLOP/s
// measured), so the mixed path keeps its accuracy-critical quantities -- the
// lifted right-hand side F, the refined iterate U and the residual
// F - A U -- as unevaluated sums hi + lo of two FP32 numbers (about 44-48
// significant bits) and computes them with error-free transformations:
//   two_sum (Knuth): s + e = a + b exactly;
//   two_prod (FMA): p + e = a * b exactly.
// The compiler must not reassociate these (no fast-math flags anywhere).
#pragma once

#include <cuda_runtime.h>

struct dfloat {
    float hi, lo;
};

__device__ __forceinline__ void df_two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ void df_fast_two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    e = b - (s - a);
}

__device__ __forceinline__ dfloat df_make(float a, float b) {
    dfloat r;
    df_two_sum(a, b, r.hi, r.lo);
    return r;
}

// x + y, error about 2^-44 (|x| + |y|)
__device__ __forceinline__ dfloat df_add(dfloat x, dfloat y) {
    float s, e;
    df_two_sum(x.hi, y.hi, s, e);
    e += x.lo + y.lo;
    dfloat r;
    df_fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

// x + y with full cancellation accuracy (both hi and lo parts two-summed)
__device__ __forceinline__ dfloat df_add_accurate(dfloat x, dfloat y) {
    float s, e, t, f;
    df_two_sum(x.hi, y.hi, s, e);
    df_two_sum(x.lo, y.lo, t, f);
    e += t;
    df_fast_two_sum(s, e, s, e);
    e += f;
    dfloat r;
    df_fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

// c * v for a double-float coefficient c and a double-float value v
__device__ __forceinline__ dfloat df_mul(dfloat c, dfloat v) {
    const float p = c.hi * v.hi;
    float e = fmaf(c.hi, v.hi, -p);
    e = fmaf(c.hi, v.lo, e);
    e = fmaf(c.lo, v.hi, e);
    dfloat r;
    df_fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ dfloat df_neg(dfloat x) {
    dfloat r;
    r.hi = -x.hi;
    r.lo = -x.lo;
    return r;
}

// Rounds an FP64 value to a pair: hi = fl32(x), lo = fl32(x - hi).
__device__ __forceinline__ dfloat df_from_double(double x) {
    dfloat r;
    r.hi = __double2float_rn(x);
    r.lo = __double2float_rn(x - (double)r.hi);
    return r;
}

__device__ __forceinline__ double df_to_double(dfloat x) { return (double)x.hi + (double)x.lo; }

// Splits an FP64 value into hi + lo FP32 parts without FP64 arithmetic: hi keeps
// the top 24 significant bits (integer operations), lo is the remaining 29 bits
// converted to FP32 (rounded to 24 bits) and scaled by 2^(e - 52) with two exact
// multiplications, so |x - (hi + lo)| <= 2^-48 |x| (lo may lose bits to FP32's
// subnormal range when |x| < 2^-74).  |x| outside FP32's normal range gives 0;
// inputs are finite.
__device__ __forceinline__ dfloat df_split_bits(double x) {
    const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
    const int e = (int)((hw >> 20) & 0x7FFu) - 1023;
    dfloat r;
    r.hi = 0.f;
    r.lo = 0.f;
    if (e < -126 || e > 127) return r;
    const unsigned sign = hw & 0x80000000u;
    const unsigned ebits = (unsigned)(e + 127) << 23;           // 2^e as FP32
    r.hi = __uint_as_float(sign | ebits | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
    const float rem = __uint2float_rn(lw & 0x1FFFFFFFu) * 0x1p-52f;
    r.lo = __uint_as_float(__float_as_uint(rem * __uint_as_float(ebits)) | sign);
    return r;
}

__device__ __forceinline__ dfloat df_of(float x) {
    dfloat r;
    r.hi = x;
    r.lo = 0.f;
    return r;
}
__device__ __forceinline__ dfloat df_of(double x) { return df_split_bits(x); }
