// Packed FP32 pairs for the transform passes that hold two columns (or rows) side by side
// (the f32x2 instructions of f32x2.cuh): complex pairs (PC: the real parts of two
// complex numbers in one register pair, the imaginary parts in another), their butterflies
// and Stockham stages of 4 elements per thread, and the 16-byte-element shared-memory swizzle
// i ^ ((i >> 2) & 7), under which every stage's reads and writes of a quarter warp fall in
// distinct bank groups (checked for the radix-4 / radix-2 stages of lengths 256 .. 2048).
#pragma once
#include "f32x2.cuh"
#include "spectral.cuh"

namespace otgb {
namespace pair {

// two complex numbers, one per column: re = (a.x, b.x), im = (a.y, b.y)
struct __align__(16) PC {
  u64 re, im;
};

__device__ __forceinline__ int swz(int i) { return i ^ ((i >> 2) & 7); }

// v * w (SIGN < 0) or v * conj(w) (SIGN > 0); wx = (w.x, w.x), wy = (w.y, w.y), nwy = -wy
template <int SIGN>
__device__ __forceinline__ PC cmulp(PC v, u64 wx, u64 wy, u64 nwy) {
  PC r;
  if (SIGN < 0) {
    r.re = fma2(v.im, nwy, mul2(v.re, wx));
    r.im = fma2(v.re, wy, mul2(v.im, wx));
  } else {
    r.re = fma2(v.im, wy, mul2(v.re, wx));
    r.im = fma2(v.re, nwy, mul2(v.im, wx));
  }
  return r;
}

template <int R, int SIGN> struct BflyP;
template <int SIGN> struct BflyP<2, SIGN> {
  __device__ __forceinline__ static void run(PC* v) {
    const PC a = v[0], b = v[1];
    v[0].re = add2(a.re, b.re);
    v[0].im = add2(a.im, b.im);
    v[1].re = sub2(a.re, b.re);
    v[1].im = sub2(a.im, b.im);
  }
};
template <int SIGN> struct BflyP<4, SIGN> {
  __device__ __forceinline__ static void run(PC* v) {
    const u64 t0r = add2(v[0].re, v[2].re), t0i = add2(v[0].im, v[2].im);
    const u64 t1r = sub2(v[0].re, v[2].re), t1i = sub2(v[0].im, v[2].im);
    const u64 t2r = add2(v[1].re, v[3].re), t2i = add2(v[1].im, v[3].im);
    const u64 dr = sub2(v[1].re, v[3].re), di = sub2(v[1].im, v[3].im);
    v[0].re = add2(t0r, t2r);
    v[0].im = add2(t0i, t2i);
    v[2].re = sub2(t0r, t2r);
    v[2].im = sub2(t0i, t2i);
    // t3 = SIGN i d: v1 = t1 + t3, v3 = t1 - t3
    if (SIGN > 0) {
      v[1].re = sub2(t1r, di);
      v[1].im = add2(t1i, dr);
      v[3].re = add2(t1r, di);
      v[3].im = sub2(t1i, dr);
    } else {
      v[1].re = add2(t1r, di);
      v[1].im = sub2(t1i, dr);
      v[3].re = sub2(t1r, di);
      v[3].im = add2(t1i, dr);
    }
  }
};

template <int REM>
__host__ __device__ constexpr int pstage_count() {
  if constexpr (REM > 1)
    return 1 + pstage_count<REM / (REM % 4 == 0 ? 4 : 2)>();
  else
    return 0;
}

// One stage of radix R (span Ns) on NP transform pairs of length L, 4 elements per thread;
// tw: the stage-ordered twiddles as (w.x, w.x, w.y, w.y) words.  Out of place (one barrier)
// or in place (INPLACE: the stores wait for every thread's loads).
template <int R, int SIGN, int L, int Ns, int NP, bool INPLACE = false>
__device__ __forceinline__ void pstage(PC* const (&in)[NP], PC* const (&out)[NP], int t,
                                       const ulonglong2* __restrict__ tw) {
  constexpr int E = 4, TPT = L / E, LR = L / R;
  constexpr int a = Ns == 1 ? 0 : __builtin_ctz(Ns);
  PC v[NP][E];
#pragma unroll
  for (int b = 0; b < E / R; ++b) {
    const int j = t + b * TPT;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int src = swz(j + r * LR);
#pragma unroll
      for (int q = 0; q < NP; ++q) v[q][b * R + r] = in[q][src];
    }
  }
  if (INPLACE) __syncthreads();
#pragma unroll
  for (int b = 0; b < E / R; ++b) {
    const int j = t + b * TPT;
    const int qd = j >> a;
    const int k = j & (Ns - 1);
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const ulonglong2 w = tw[(Ns - 1) + (r - 1) * Ns + k];
        const u64 nwy = sub2(0ull, w.y);  // (0, 0) - (w.y, w.y)
#pragma unroll
        for (int q = 0; q < NP; ++q)
          v[q][b * R + r] = cmulp<SIGN>(v[q][b * R + r], w.x, w.y, nwy);
      }
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) BflyP<R, SIGN>::run(&v[q][b * R]);
    const int d = qd * (Ns * R) + k;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int dst = swz(d + r * Ns);
#pragma unroll
      for (int q = 0; q < NP; ++q) out[q][dst] = v[q][b * R + r];
    }
  }
  __syncthreads();
}

// the transform: stages alternating between a and b, starting from a; the result ends in a
// for an even number of stages, in b for an odd one
template <int SIGN, int L, int Ns, int REM, int NP, bool FROM_A>
__device__ __forceinline__ void pfft_rec(PC* const (&a)[NP], PC* const (&b)[NP], int t,
                                         const ulonglong2* __restrict__ tw) {
  if constexpr (REM > 1) {
    constexpr int R = REM % 4 == 0 ? 4 : 2;
    if constexpr (FROM_A)
      pstage<R, SIGN, L, Ns, NP>(a, b, t, tw);
    else
      pstage<R, SIGN, L, Ns, NP>(b, a, t, tw);
    pfft_rec<SIGN, L, Ns * R, REM / R, NP, !FROM_A>(a, b, t, tw);
  }
}

// the same transform in place
template <int SIGN, int L, int Ns, int REM, int NP>
__device__ __forceinline__ void pfft_inplace(PC* const (&a)[NP], int t,
                                             const ulonglong2* __restrict__ tw) {
  if constexpr (REM > 1) {
    constexpr int R = REM % 4 == 0 ? 4 : 2;
    pstage<R, SIGN, L, Ns, NP, true>(a, a, t, tw);
    pfft_inplace<SIGN, L, Ns * R, REM / R, NP>(a, t, tw);
  }
}

// the stage twiddles of the 4-element transforms of length L, broadcast to both lanes
template <int L>
__device__ __forceinline__ void load_tw4(ulonglong2* tw4, const float2* __restrict__ twb, int t,
                                         int nthreads) {
  const float2* __restrict__ st = twb + (size_t)stage_table_slot<4>() * L;
  for (int i = t; i < L; i += nthreads) {
    const float2 w = st[i];
    tw4[i] = make_ulonglong2(pk(w.x, w.x), pk(w.y, w.y));
  }
}


}  // namespace pair
}  // namespace otgb
