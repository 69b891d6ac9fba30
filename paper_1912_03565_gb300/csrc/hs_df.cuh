// Double-float ("FP32 pair") arithmetic for the mixed path.
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

// Splits an FP64 value into hi + lo FP32 parts with integer operations only
// (no FP64 instruction): hi keeps the top 24 significant bits, lo the next 24
// (truncated), so |x - (hi + lo)| <= 2^-47 |x|.  Values below 2^-126 in
// magnitude (FP32's normal range) become 0; inputs are finite.
__device__ __forceinline__ dfloat df_split_bits(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7FF) - 1023;
    const unsigned long long m = b & 0xFFFFFFFFFFFFFULL;
    dfloat r;
    r.hi = 0.f;
    r.lo = 0.f;
    if (e < -126 || e > 127) return r;
    r.hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)(m >> 29));
    const unsigned rem = (unsigned)(m & 0x1FFFFFFFULL);  // low 29 bits
    if (rem == 0) return r;
    const int p = 31 - __clz(rem);                       // msb position, 0..28
    const int el = e - 52 + p;                           // exponent of the lo part
    if (el < -126) return r;
    const unsigned frac = (p >= 23) ? ((rem >> (p - 23)) & 0x7FFFFFu) : ((rem << (23 - p)) & 0x7FFFFFu);
    r.lo = __uint_as_float(sign | ((unsigned)(el + 127) << 23) | frac);
    return r;
}

__device__ __forceinline__ dfloat df_of(float x) {
    dfloat r;
    r.hi = x;
    r.lo = 0.f;
    return r;
}
__device__ __forceinline__ dfloat df_of(double x) { return df_split_bits(x); }
