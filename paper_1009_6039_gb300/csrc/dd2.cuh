// Two double-float numbers in the lanes of packed FP32 register pairs (f32x2.cuh): high words
// (hi_a, hi_b) and low words (lo_a, lo_b).  Every step of dd.cuh's error-free transformations
// (TwoSum, FastTwoSum, the FMA TwoProduct) runs once for both numbers as a packed
// round-to-nearest instruction, in dd.cuh's order, so each lane is bit for bit dd.cuh's
// result from the same inputs.
#pragma once
#include "f32x2.cuh"

namespace otgb {
namespace pair {

__device__ __forceinline__ u64 neg2(u64 a) { return mul2(a, pk(-1.f, -1.f)); }

// two double-float numbers, one per lane
struct D2 {
  u64 h, l;
};
__device__ __forceinline__ D2 two_sum2(u64 a, u64 b) {
  const u64 s = add2(a, b);
  const u64 bb = sub2(s, a);
  return D2{s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}
__device__ __forceinline__ D2 fast_two_sum2(u64 a, u64 b) {
  const u64 s = add2(a, b);
  return D2{s, sub2(b, sub2(s, a))};
}
__device__ __forceinline__ D2 d2_add(D2 a, D2 b) {
  const D2 s = two_sum2(a.h, b.h);
  return fast_two_sum2(s.h, add2(s.l, add2(a.l, b.l)));
}
__device__ __forceinline__ D2 d2_neg(D2 a) { return D2{neg2(a.h), neg2(a.l)}; }
__device__ __forceinline__ D2 d2_sub(D2 a, D2 b) { return d2_add(a, d2_neg(b)); }
__device__ __forceinline__ D2 d2_mul(D2 a, D2 b) {
  const u64 p = mul2(a.h, b.h);
  u64 e = fma2(a.h, b.h, neg2(p));
  e = fma2(a.h, b.l, e);
  e = fma2(a.l, b.h, e);
  return fast_two_sum2(p, e);
}

}  // namespace pair
}  // namespace otgb
