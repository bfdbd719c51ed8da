// Double-float ("dd") arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi)/2, giving a 48-bit significand (unit round-off 2^-48 ~ 3.6e-15).
// Built on the error-free transformations of Knuth (TwoSum), Dekker (FastTwoSum) and the FMA
// form of TwoProduct; every FP32 operation is written with a _rn intrinsic so the compiler
// can neither contract nor reassociate it (that would break the error-free steps).
//
// GB300 runs FP32 at about 60x its FP64 rate, so FP64-accuracy work that would be bound by
// the FP64 pipe runs several times faster as dd on the FP32 pipes.
#pragma once
#include <cuda_runtime.h>

namespace otgb {

struct dd {
  float hi, lo;
  dd() = default;
  __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  // constants: the nearest float and the nearest float to the remainder (folded at compile
  // time for literal arguments)
  __host__ __device__ constexpr explicit dd(double v)
      : hi((float)v), lo((float)(v - (double)(float)v)) {}
};

__device__ __forceinline__ dd dd_make(float hi, float lo) { return dd(hi, lo); }

// split an FP64 value: hi = nearest float, lo = nearest float to the (exact) remainder
__device__ __forceinline__ dd dd_from_double(double a) {
  const float h = __double2float_rn(a);
  return dd{h, __double2float_rn(a - (double)h)};
}
__device__ __forceinline__ double dd_to_double(dd a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ dd two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dd{s, e};
}
// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ dd fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dd{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dd dd_add(dd a, dd b) {
  const dd s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
__device__ __forceinline__ dd dd_add_f(dd a, float b) {
  const dd s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ dd dd_mul_f(dd a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return fast_two_sum(p, e);
}
// a * 2^k (exact)
__device__ __forceinline__ dd dd_scale2(dd a, float pow2) {
  return dd{__fmul_rn(a.hi, pow2), __fmul_rn(a.lo, pow2)};
}
// a * b + c
__device__ __forceinline__ dd dd_fma(dd a, dd b, dd c) { return dd_add(dd_mul(a, b), c); }

__device__ __forceinline__ bool dd_gt(dd a, dd b) {
  return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}

// operators, so that the templated transforms can run on dd
__device__ __forceinline__ dd operator+(dd a, dd b) { return dd_add(a, b); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return dd_sub(a, b); }
__device__ __forceinline__ dd operator-(dd a) { return dd_neg(a); }
__device__ __forceinline__ dd operator*(dd a, dd b) { return dd_mul(a, b); }
// multiplication by a sign +-1 (exact)
__device__ __forceinline__ dd operator*(int s, dd a) { return s >= 0 ? a : dd_neg(a); }
__device__ __forceinline__ dd& operator+=(dd& a, dd b) { return a = dd_add(a, b); }

// complex dd
struct ddc {
  dd x, y;
};

}  // namespace otgb
