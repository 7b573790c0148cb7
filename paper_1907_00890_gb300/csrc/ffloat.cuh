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

}  // namespace vofp
