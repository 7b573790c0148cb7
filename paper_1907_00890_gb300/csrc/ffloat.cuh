// Float-float ("FP32-pair") arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi)/2, about 48 significant bits (relative precision ~1e-14) on the FP32 pipe, which on this
// GPU issues about 60 times as many operations per second as the FP64 pipe.  Error-free transformations:
// two-sum (Knuth) for additions, an FMA residual for products (p = a*b exactly equals fl(a*b) + fma(a,b,-p)),
// a Dekker-style correction for quotients.  Additions use the "sloppy" form (one two-sum of the high parts
// plus the low parts), whose error is bounded relative to |a| + |b| -- the bound an FFT's error analysis
// needs.  No operation here may be contracted or re-associated by the compiler beyond what is written:
// the error terms are computed with explicit fmaf and plain additions.
#pragma once

#include <cuda_runtime.h>

namespace vofp {

struct __align__(8) ff {
  float hi, lo;
  __host__ __device__ __forceinline__ ff() {}
  __host__ __device__ __forceinline__ ff(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ __forceinline__ ff(double d) {
    hi = (float)d;
    lo = (float)(d - (double)hi);
  }
  __host__ __device__ __forceinline__ ff(int i) : hi((float)i), lo(0.0f) {}
  __host__ __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

struct __align__(16) cff {
  ff x, y;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff(s, e);
}

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {  // requires |a| >= |b|
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return ff(s, e);
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return ff_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }

__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }

__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}

__device__ __forceinline__ ff operator/(ff a, ff b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const ff r = a - b * ff(q1, 0.0f);
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return ff_fast_two_sum(q1, q2);
}

__device__ __forceinline__ ff& operator+=(ff& a, ff b) {
  a = a + b;
  return a;
}
__device__ __forceinline__ ff& operator-=(ff& a, ff b) {
  a = a - b;
  return a;
}
__device__ __forceinline__ ff& operator*=(ff& a, ff b) {
  a = a * b;
  return a;
}
__device__ __forceinline__ ff& operator/=(ff& a, ff b) {
  a = a / b;
  return a;
}

// Exact widening of a reduced-precision value to a pair, and its leading FP32 part.
__host__ __device__ __forceinline__ ff ff_of(float x) { return ff(x, 0.0f); }
__host__ __device__ __forceinline__ ff ff_of(ff x) { return x; }
__host__ __device__ __forceinline__ float lead(float x) { return x; }
__host__ __device__ __forceinline__ float lead(ff x) { return x.hi; }
__host__ __device__ __forceinline__ ff ff_of(double x) { return ff(x); }
__host__ __device__ __forceinline__ float lead(double x) { return (float)x; }

// ---- conversions on the integer pipe ----------------------------------------------------------------------
// On this GPU a conversion between FP64 and FP32 issues on the FP64 unit (same rate and latency as an FP64
// multiply-add), so the reduced-precision passes split and join doubles with integer operations instead.
// Magnitudes below the FP32 normal range are flushed to zero; above it they become infinities.

// FP32 value of the 24 leading significand bits of a double (truncated, not rounded).
__device__ __forceinline__ float f32_lead_bits(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi32 = (unsigned)(b >> 32);
  const unsigned sign = hi32 & 0x80000000u;
  const int e = (int)((hi32 >> 20) & 0x7ffu);
  const int ef = e - 1023 + 127;
  const unsigned m23 = (unsigned)(b >> 29) & 0x7fffffu;
  unsigned r = sign | ((unsigned)ef << 23) | m23;
  if (ef <= 0) r = sign;                                              // zero, subnormal range
  if (ef >= 255) r = sign | 0x7f800000u | (e == 0x7ff && (b << 12) ? 1u : 0u);  // overflow, inf, nan
  return __uint_as_float(r);
}

// Split a double into a normalised FP32 pair: hi = its 24 leading significand bits, lo = the next 24 of the
// remaining 29 (relative error of the pair below 2^-47).
__device__ __forceinline__ ff ff_split(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi32 = (unsigned)(b >> 32);
  const unsigned sign = hi32 & 0x80000000u;
  const int e = (int)((hi32 >> 20) & 0x7ffu);
  const float hi = f32_lead_bits(d);
  const unsigned rem = (unsigned)b & 0x1fffffffu;  // the 29 significand bits below hi
  // rem * 2^(e - 1075): its leading one at bit p
  const int p = 31 - __clz(rem | 1u);
  const int elo = p + e - 1075 + 127;
  const unsigned ml = (p >= 23 ? (rem >> (p - 23)) : (rem << (23 - p))) & 0x7fffffu;
  unsigned lb = sign | ((unsigned)elo << 23) | ml;
  if (rem == 0u || elo <= 0 || e - 1023 + 127 <= 0 || e - 1023 + 127 >= 255) lb = 0u;
  return ff_fast_two_sum(hi, __uint_as_float(lb));
}

// Exact widening of a normal FP32 value to FP64 (zero and subnormals give zero; inf and nan pass).
__device__ __forceinline__ double f64_of_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned ef = (u >> 23) & 0xffu;
  const unsigned long long m = (unsigned long long)(u & 0x7fffffu) << 29;
  unsigned long long r = sign | ((unsigned long long)(ef + 1023u - 127u) << 52) | m;
  if (ef == 0u) r = sign;
  if (ef == 255u) r = sign | 0x7ff0000000000000ull | m;
  return __longlong_as_double((long long)r);
}

// 1 / x for a normal x within the FP32 range: an FP32 reciprocal of its leading bits as the seed (integer-pipe
// split and join), then two Newton steps y <- y + y (1 - x y) in FP64 (quadratic convergence: 2^-23 -> 2^-46 ->
// below FP64 rounding), four FP64 multiply-adds against an FP64 division's longer sequence on this GPU.
__device__ __forceinline__ double recip_newton(double x) {
  double y = f64_of_bits(__frcp_rn(f32_lead_bits(x)));
  y = fma(y, fma(-x, y, 1.0), y);
  return fma(y, fma(-x, y, 1.0), y);
}

// The same with one Newton step: relative error about 2^-46 (1.4e-14), two FP64 multiply-adds.
__device__ __forceinline__ double recip_newton1(double x) {
  const double y = f64_of_bits(__frcp_rn(f32_lead_bits(x)));
  return fma(y, fma(-x, y, 1.0), y);
}

// Reduced-precision value <-> double with the conversions above (one FP64 addition for a pair).
__device__ __forceinline__ float red_of(double d, float*) { return f32_lead_bits(d); }
__device__ __forceinline__ ff red_of(double d, ff*) { return ff_split(d); }
__device__ __forceinline__ double red_of(double d, double*) { return d; }
__device__ __forceinline__ double wide_of(float x) { return f64_of_bits(x); }
__device__ __forceinline__ double wide_of(ff x) { return f64_of_bits(x.hi) + f64_of_bits(x.lo); }
__device__ __forceinline__ double wide_of(double x) { return x; }

}  // namespace vofp
