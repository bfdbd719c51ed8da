// Spectral kernels of Strain's method (Sec. 4.2): batched 2-D real FFTs of the packed
// half spectrum with the symbol multiplies and the coefficient apply fused in.
//
// A 1-D transform of length L is done by one group of L/E threads on a shared-memory
// buffer: a Stockham auto-sort FFT whose stages have radix 8/4/2 (L = 2^a, E = 8) or a
// first radix-3 stage followed by radix 4/2 (L = 3 * 2^a, E = 12).  Each thread holds the
// E elements of its E/R butterflies in registers between the shared-memory read and write
// of a stage.  Twiddles come from a table exp(-2 pi i t / L) built once per plan.
//
// Matvec (the dominant step, Sec. 4.2):
//   row_r2c          sigma (N x M real)  -> X (N x M/2 complex, packed)
//   col COL_MATVEC   X -> sigma-hat (column FFT) -> S = rho-bar sigma-hat / (N M)
//                    -> Q0 = S, Q1 = (2 pi i k2) S, Q2 = -(2 pi k2)^2 S -> inverse column FFTs
//   row_c2r COMBINE  five row inverse transforms (d_xx Q0, d_x Q0, d_x Q1, Q1, Q2) weighted
//                    by a11, b1, 2 a12, b2, a22 and summed: w = L Lbar^{-1} sigma.
#pragma once
#include <deque>
#include <mutex>
#include <vector>

#include "otgb_internal.cuh"

namespace otgb {

#define OTGB_TWO_PI 6.283185307179586476925286766559
#define OTGB_SQRT_HALF 0.70710678118654752440084436210485
#define OTGB_SQRT3_HALF 0.86602540378443864676372317075294

template <typename T> __device__ __forceinline__ C2<T> mk2(T x, T y) {
  C2<T> r;
  r.x = x;
  r.y = y;
  return r;
}
template <typename T> __device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) {
  return mk2<T>(a.x + b.x, a.y + b.y);
}
template <typename T> __device__ __forceinline__ C2<T> csub(C2<T> a, C2<T> b) {
  return mk2<T>(a.x - b.x, a.y - b.y);
}
template <typename T> __device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  return mk2<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ C2<T> cconj(C2<T> a) {
  return mk2<T>(a.x, -a.y);
}
template <typename T> __device__ __forceinline__ C2<T> cscale(C2<T> a, T s) {
  return mk2<T>(a.x * s, a.y * s);
}
// multiply by SIGN * i
template <typename T, int SIGN> __device__ __forceinline__ C2<T> mul_si(C2<T> a) {
  return SIGN > 0 ? mk2<T>(-a.y, a.x) : mk2<T>(a.y, -a.x);
}

// In-register DFTs of size R with exponent sign SIGN (-1 forward, +1 inverse).
template <typename T, int R, int SIGN> struct Bfly;

template <typename T, int SIGN> struct Bfly<T, 2, SIGN> {
  __device__ __forceinline__ static void run(C2<T>* v) {
    C2<T> a = v[0], b = v[1];
    v[0] = cadd<T>(a, b);
    v[1] = csub<T>(a, b);
  }
};

template <typename T, int SIGN> struct Bfly<T, 3, SIGN> {
  __device__ __forceinline__ static void run(C2<T>* v) {
    C2<T> a = v[0], s = cadd<T>(v[1], v[2]), d = csub<T>(v[1], v[2]);
    C2<T> t = mk2<T>(a.x - (T)0.5 * s.x, a.y - (T)0.5 * s.y);
    C2<T> u = cscale<T>(mul_si<T, SIGN>(d), (T)OTGB_SQRT3_HALF);
    v[0] = cadd<T>(a, s);
    v[1] = cadd<T>(t, u);
    v[2] = csub<T>(t, u);
  }
};

template <typename T, int SIGN> struct Bfly<T, 4, SIGN> {
  __device__ __forceinline__ static void run(C2<T>* v) {
    C2<T> t0 = cadd<T>(v[0], v[2]), t1 = csub<T>(v[0], v[2]);
    C2<T> t2 = cadd<T>(v[1], v[3]), t3 = mul_si<T, SIGN>(csub<T>(v[1], v[3]));
    v[0] = cadd<T>(t0, t2);
    v[2] = csub<T>(t0, t2);
    v[1] = cadd<T>(t1, t3);
    v[3] = csub<T>(t1, t3);
  }
};

// FP32: a complex number is a register pair, so complex additions and subtractions are
// single packed instructions (add/sub.rn.f32x2: per lane the same IEEE operation as the
// scalar forms, so the results are bit for bit those of the scalar butterflies); the
// multiplication by +-i mixes the lanes and stays scalar.
__device__ __forceinline__ float2 padd2(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "add.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 psub2(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}

template <int SIGN> struct Bfly<float, 2, SIGN> {
  __device__ __forceinline__ static void run(float2* v) {
    const float2 a = v[0], b = v[1];
    v[0] = padd2(a, b);
    v[1] = psub2(a, b);
  }
};

template <int SIGN> struct Bfly<float, 4, SIGN> {
  __device__ __forceinline__ static void run(float2* v) {
    const float2 t0 = padd2(v[0], v[2]), t1 = psub2(v[0], v[2]);
    const float2 t2 = padd2(v[1], v[3]), d = psub2(v[1], v[3]);
    v[0] = padd2(t0, t2);
    v[2] = psub2(t0, t2);
    // t3 = SIGN i d; v1 = t1 + t3, v3 = t1 - t3
    if (SIGN > 0) {
      v[1] = make_float2(t1.x - d.y, t1.y + d.x);
      v[3] = make_float2(t1.x + d.y, t1.y - d.x);
    } else {
      v[1] = make_float2(t1.x + d.y, t1.y - d.x);
      v[3] = make_float2(t1.x - d.y, t1.y + d.x);
    }
  }
};

template <typename T, int SIGN> struct Bfly<T, 8, SIGN> {
  __device__ __forceinline__ static void run(C2<T>* v) {
    C2<T> e[4] = {v[0], v[2], v[4], v[6]};
    C2<T> o[4] = {v[1], v[3], v[5], v[7]};
    Bfly<T, 4, SIGN>::run(e);
    Bfly<T, 4, SIGN>::run(o);
    // o[k] *= exp(SIGN 2 pi i k / 8)
    const T h = (T)OTGB_SQRT_HALF;
    C2<T> o1 = o[1], o3 = o[3];
    o[1] = mk2<T>(h * (o1.x - SIGN * o1.y), h * (o1.y + SIGN * o1.x));
    o[2] = mul_si<T, SIGN>(o[2]);
    o[3] = mk2<T>(h * (-o3.x - SIGN * o3.y), h * (-o3.y + SIGN * o3.x));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = cadd<T>(e[k], o[k]);
      v[k + 4] = csub<T>(e[k], o[k]);
    }
  }
};

// Shared-memory stride of one transform buffer of length L: between the stages of a
// transform the data sit in a padded layout (one element of padding per 16, spad) so that
// the strided stage writes spread over the banks; the transform's input and output use the
// plain layout 0..L-1.
__host__ __device__ constexpr int FB(int L) { return L + (L >> 4) + 1; }
__device__ __forceinline__ int spad(int i, bool on) { return on ? i + (i >> 4) : i; }

// Stage-ordered twiddle tables.  A base table of length L (exp(-2 pi i t / L), t < L) is
// followed by one stage table per thread width E = 4, 8, 12 (L entries each; only the width
// the length allows is filled): the stage with span Ns and radix R holds exp(-2 pi i k r /
// (Ns R)) for r = 1..R-1, k = 0..Ns-1 at (Ns - 1) + (r - 1) Ns + k (the stages before it hold
// sum Ns'(R' - 1) = Ns - 1 entries).  The threads of a warp take consecutive k, so a stage's
// twiddle loads are contiguous instead of the strided k r L / (Ns R) of the base table.
template <int E> __host__ __device__ constexpr int stage_table_slot() {
  return E == 4 ? 1 : (E == 8 ? 2 : 3);
}

// One Stockham stage of radix R on a transform of length L held in buf (all threads of
// the block must call it; inactive threads only take part in the barriers).  pin / pout:
// the stage reads / writes the padded layout.  st: the stage table of this width.
template <typename T, int E, int R, int SIGN>
__device__ __forceinline__ void stockham_stage(C2<T>* buf, int L, int Ns, int t, bool active,
                                               const C2<T>* __restrict__ st, bool pin,
                                               bool pout) {
  const int TPT = L / E;
  const int LR = L / R;
  C2<T> v[E];
  if (active) {
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
      const int j = t + b * TPT;
#pragma unroll
      for (int r = 0; r < R; ++r) v[b * R + r] = buf[spad(j + r * LR, pin)];
    }
  }
  __syncthreads();
  if (active) {
    // Ns = 2^a or 3 * 2^a: j / Ns by a shift (and a division by the constant 3)
    const int a = __ffs(Ns) - 1;
    const bool pow2 = (Ns >> a) == 1;
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
      const int j = t + b * TPT;
      const int qd = pow2 ? (j >> a) : ((j >> a) / 3);
      const int k = j - qd * Ns;
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C2<T> w = st[(Ns - 1) + (r - 1) * Ns + k];
          if (SIGN > 0) w.y = -w.y;
          v[b * R + r] = cmul<T>(v[b * R + r], w);
        }
      }
      Bfly<T, R, SIGN>::run(&v[b * R]);
      const int d = qd * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[spad(d + r * Ns, pout)] = v[b * R + r];
    }
  }
  __syncthreads();
}

// NB independent transforms of the same length interleaved in the same threads: each stage
// loads a twiddle once for all NB buffers, and the NB butterflies give the scheduler
// independent work (the passes are latency-bound at the sizes of interest).
template <typename T, int E, int R, int SIGN, int NB>
__device__ __forceinline__ void stockham_stage_multi(C2<T>* const (&bufs)[NB], int L, int Ns,
                                                     int t, bool active,
                                                     const C2<T>* __restrict__ st, bool pin,
                                                     bool pout) {
  const int TPT = L / E;
  const int LR = L / R;
  C2<T> v[NB][E];
  if (active) {
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
      const int j = t + b * TPT;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int src = spad(j + r * LR, pin);
#pragma unroll
        for (int q = 0; q < NB; ++q) v[q][b * R + r] = bufs[q][src];
      }
    }
  }
  __syncthreads();
  if (active) {
    const int a = __ffs(Ns) - 1;
    const bool pow2 = (Ns >> a) == 1;
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
      const int j = t + b * TPT;
      const int qd = pow2 ? (j >> a) : ((j >> a) / 3);
      const int k = j - qd * Ns;
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C2<T> w = st[(Ns - 1) + (r - 1) * Ns + k];
          if (SIGN > 0) w.y = -w.y;
#pragma unroll
          for (int q = 0; q < NB; ++q) v[q][b * R + r] = cmul<T>(v[q][b * R + r], w);
        }
      }
#pragma unroll
      for (int q = 0; q < NB; ++q) Bfly<T, R, SIGN>::run(&v[q][b * R]);
      const int d = qd * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int dst = spad(d + r * Ns, pout);
#pragma unroll
        for (int q = 0; q < NB; ++q) bufs[q][dst] = v[q][b * R + r];
      }
    }
  }
  __syncthreads();
}

template <typename T, int E, int SIGN, int NB>
__device__ __forceinline__ void fft_smem_multi_rt(C2<T>* const (&bufs)[NB], int L, int t,
                                                  bool active, const C2<T>* __restrict__ twb) {
  const C2<T>* __restrict__ tw = twb + (size_t)stage_table_slot<E>() * L;
  int Ns = 1;
  int rem = L;
  if (E % 3 == 0) {
    stockham_stage_multi<T, E, 3, SIGN, NB>(bufs, L, Ns, t, active, tw, false, rem / 3 > 1);
    Ns *= 3;
    rem /= 3;
  }
  while (rem > 1) {
    const bool pin = Ns > 1;
    if (E % 8 == 0 && rem % 8 == 0) {
      stockham_stage_multi<T, E, 8, SIGN, NB>(bufs, L, Ns, t, active, tw, pin, rem / 8 > 1);
      Ns *= 8;
      rem /= 8;
    } else if (rem % 4 == 0) {
      stockham_stage_multi<T, E, 4, SIGN, NB>(bufs, L, Ns, t, active, tw, pin, rem / 4 > 1);
      Ns *= 4;
      rem /= 4;
    } else {
      stockham_stage_multi<T, E, 2, SIGN, NB>(bufs, L, Ns, t, active, tw, pin, rem / 2 > 1);
      Ns *= 2;
      rem /= 2;
    }
  }
}

// Full unnormalised transform X_k = sum_n x_n exp(SIGN 2 pi i k n / L), in place in buf.
// Radix sequence: [3,] then 8s (E = 8) or 4s (E = 12), then the remaining 4 or 2.
template <typename T, int E, int SIGN>
__device__ __forceinline__ void fft_smem_rt(C2<T>* buf, int L, int t, bool active,
                                            const C2<T>* __restrict__ twb) {
  const C2<T>* __restrict__ tw = twb + (size_t)stage_table_slot<E>() * L;
  int Ns = 1;
  int rem = L;
  if (E % 3 == 0) {
    stockham_stage<T, E, 3, SIGN>(buf, L, Ns, t, active, tw, false, rem / 3 > 1);
    Ns *= 3;
    rem /= 3;
  }
  while (rem > 1) {
    const bool pin = Ns > 1;
    if (E % 8 == 0 && rem % 8 == 0) {
      stockham_stage<T, E, 8, SIGN>(buf, L, Ns, t, active, tw, pin, rem / 8 > 1);
      Ns *= 8;
      rem /= 8;
    } else if (rem % 4 == 0) {
      stockham_stage<T, E, 4, SIGN>(buf, L, Ns, t, active, tw, pin, rem / 4 > 1);
      Ns *= 4;
      rem /= 4;
    } else {
      stockham_stage<T, E, 2, SIGN>(buf, L, Ns, t, active, tw, pin, rem / 2 > 1);
      Ns *= 2;
      rem /= 2;
    }
  }
}

// The same transforms with the length fixed at compile time (power-of-two L): the stage
// sequence (radix 8 or 4 while the remainder allows, then 4 or 2), the spans, the thread
// counts and the shared-memory indices fold into constants, which removes most of the
// integer work of a stage.  The arithmetic and its order are those of the run-time version,
// so the results are bit for bit the same.
template <typename T, int E, int R, int SIGN, int L, int Ns, bool PIN, bool POUT, int NB,
          bool INPLACE>
__device__ __forceinline__ void stockham_stage_c(C2<T>* const (&in)[NB], C2<T>* const (&out)[NB],
                                                 int t, bool active,
                                                 const C2<T>* __restrict__ st) {
  constexpr int TPT = L / E;
  constexpr int LR = L / R;
  constexpr int a = Ns == 1 ? 0 : __builtin_ctz(Ns);
  C2<T> v[NB][E];
  if (active) {
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
      const int j = t + b * TPT;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int src = spad(j + r * LR, PIN);
#pragma unroll
        for (int q = 0; q < NB; ++q) v[q][b * R + r] = in[q][src];
      }
    }
  }
  // in place, the stores must wait for every thread's loads; from one buffer into the
  // other, the stage needs only the barrier at its end
  if (INPLACE) __syncthreads();
  if (active) {
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
      const int j = t + b * TPT;
      const int qd = j >> a;
      const int k = j & (Ns - 1);
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C2<T> w = st[(Ns - 1) + (r - 1) * Ns + k];
          if (SIGN > 0) w.y = -w.y;
#pragma unroll
          for (int q = 0; q < NB; ++q) v[q][b * R + r] = cmul<T>(v[q][b * R + r], w);
        }
      }
#pragma unroll
      for (int q = 0; q < NB; ++q) Bfly<T, R, SIGN>::run(&v[q][b * R]);
      const int d = qd * (Ns * R) + k;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int dst = spad(d + r * Ns, POUT);
#pragma unroll
        for (int q = 0; q < NB; ++q) out[q][dst] = v[q][b * R + r];
      }
    }
  }
  __syncthreads();
}

// radix of the stage with remainder REM (E elements per thread): 8 or 4 while the remainder
// allows, then 4 or 2 -- the sequence of the run-time transforms
template <int E, int REM>
__host__ __device__ constexpr int stage_radix() {
  return (E % 8 == 0 && REM % 8 == 0) ? 8 : (REM % 4 == 0 ? 4 : 2);
}
template <int E, int REM>
__host__ __device__ constexpr int stage_count() {
  if constexpr (REM > 1)
    return 1 + stage_count<E, REM / stage_radix<E, REM>()>();
  else
    return 0;
}

template <typename T, int E, int SIGN, int L, int Ns, int REM, int NB>
__device__ __forceinline__ void fft_smem_c(C2<T>* const (&bufs)[NB], int t, bool active,
                                           const C2<T>* __restrict__ tw) {
  if constexpr (REM > 1) {
    constexpr int R = stage_radix<E, REM>();
    stockham_stage_c<T, E, R, SIGN, L, Ns, (Ns > 1), (REM / R > 1), NB, true>(bufs, bufs, t,
                                                                             active, tw);
    fft_smem_c<T, E, SIGN, L, Ns * R, REM / R, NB>(bufs, t, active, tw);
  }
}

// Ping-pong form: the stages alternate between bufs and the scratch buffers (one barrier a
// stage); with an odd number of stages the first runs in place, so that the result ends in
// bufs.  Same arithmetic and order as above.
template <typename T, int E, int SIGN, int L, int Ns, int REM, int NB, bool FROM_A>
__device__ __forceinline__ void fft_smem_pp_rec(C2<T>* const (&a)[NB], C2<T>* const (&b)[NB],
                                                int t, bool active,
                                                const C2<T>* __restrict__ tw) {
  if constexpr (REM > 1) {
    constexpr int R = stage_radix<E, REM>();
    if constexpr (FROM_A)
      stockham_stage_c<T, E, R, SIGN, L, Ns, (Ns > 1), (REM / R > 1), NB, false>(a, b, t,
                                                                                active, tw);
    else
      stockham_stage_c<T, E, R, SIGN, L, Ns, (Ns > 1), (REM / R > 1), NB, false>(b, a, t,
                                                                                active, tw);
    fft_smem_pp_rec<T, E, SIGN, L, Ns * R, REM / R, NB, !FROM_A>(a, b, t, active, tw);
  }
}

template <typename T, int E, int SIGN, int L, int NB>
__device__ __forceinline__ void fft_smem_c_pp(C2<T>* const (&a)[NB], C2<T>* const (&b)[NB],
                                              int t, bool active,
                                              const C2<T>* __restrict__ tw) {
  if constexpr (stage_count<E, L>() % 2 == 1) {
    constexpr int R0 = stage_radix<E, L>();
    stockham_stage_c<T, E, R0, SIGN, L, 1, false, (L / R0 > 1), NB, true>(a, a, t, active, tw);
    fft_smem_pp_rec<T, E, SIGN, L, R0, L / R0, NB, true>(a, b, t, active, tw);
  } else {
    fft_smem_pp_rec<T, E, SIGN, L, 1, L, NB, true>(a, b, t, active, tw);
  }
}

// with scratch buffers (as many as bufs, each of FB(L) elements): the ping-pong transforms
// for the 4-element kernels at power-of-two lengths 256 .. 2048, else the in-place ones
template <typename T, int E, int SIGN, int NB>
__device__ __forceinline__ void fft_smem_multi_pp(C2<T>* const (&bufs)[NB],
                                                  C2<T>* const (&scratch)[NB], int L, int t,
                                                  bool active, const C2<T>* __restrict__ twb) {
  if constexpr (E == 4) {
    const C2<T>* __restrict__ tw = twb + (size_t)stage_table_slot<E>() * L;
    switch (L) {
      case 256: fft_smem_c_pp<T, E, SIGN, 256, NB>(bufs, scratch, t, active, tw); return;
      case 512: fft_smem_c_pp<T, E, SIGN, 512, NB>(bufs, scratch, t, active, tw); return;
      case 1024: fft_smem_c_pp<T, E, SIGN, 1024, NB>(bufs, scratch, t, active, tw); return;
      case 2048: fft_smem_c_pp<T, E, SIGN, 2048, NB>(bufs, scratch, t, active, tw); return;
      default: break;
    }
  }
  fft_smem_multi_rt<T, E, SIGN, NB>(bufs, L, t, active, twb);
}

// dispatch on the length: the compile-time transforms for the 4-element-per-thread kernels
// at the power-of-two lengths 256 .. 2048, the run-time ones otherwise
template <typename T, int E, int SIGN, int NB>
__device__ __forceinline__ void fft_smem_multi(C2<T>* const (&bufs)[NB], int L, int t,
                                               bool active, const C2<T>* __restrict__ twb) {
  if constexpr (E == 4) {
    const C2<T>* __restrict__ tw = twb + (size_t)stage_table_slot<E>() * L;
    switch (L) {
      case 256: fft_smem_c<T, E, SIGN, 256, 1, 256, NB>(bufs, t, active, tw); return;
      case 512: fft_smem_c<T, E, SIGN, 512, 1, 512, NB>(bufs, t, active, tw); return;
      case 1024: fft_smem_c<T, E, SIGN, 1024, 1, 1024, NB>(bufs, t, active, tw); return;
      case 2048: fft_smem_c<T, E, SIGN, 2048, 1, 2048, NB>(bufs, t, active, tw); return;
      default: break;
    }
  }
  fft_smem_multi_rt<T, E, SIGN, NB>(bufs, L, t, active, twb);
}

template <typename T, int E, int SIGN>
__device__ __forceinline__ void fft_smem(C2<T>* buf, int L, int t, bool active,
                                         const C2<T>* __restrict__ twb) {
  if constexpr (E == 4) {
    if (L >= 256 && L <= 2048 && (L & (L - 1)) == 0) {
      C2<T>* const bufs[1] = {buf};
      fft_smem_multi<T, E, SIGN, 1>(bufs, L, t, active, twb);
      return;
    }
  }
  fft_smem_rt<T, E, SIGN>(buf, L, t, active, twb);
}

// ---------------------------------------------------------------------------------------
// Warp-synchronous transforms for power-of-two lengths L <= 2048 (FP32 passes).  A thread
// holds W = 32 elements; the L/32 threads of one transform are at most one warp for
// L <= 1024 (synchronised with __syncwarp) and two warps for L = 2048 (a named barrier per
// transform pair).  Stages: radix 32, then the remaining factor (32, 16, 8, 4 or 2),
// each one shared-memory round trip.  Shared memory is padded by one element per 32 so
// the stride-32 patterns of the stages hit distinct banks.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int pad32(int i) { return i + (i >> 5); }

// Twiddle load that the compiler may not hoist out of loops (a hoisted set of butterfly
// twiddles would occupy ~80 registers across the output loop of the column pass).
template <typename T> __device__ __forceinline__ C2<T> ldtw(const C2<T>* p);
template <> __device__ __forceinline__ float2 ldtw<float>(const float2* p) {
  float2 r;
  asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "l"(p));
  return r;
}
template <> __device__ __forceinline__ double2 ldtw<double>(const double2* p) {
  double2 r;
  asm volatile("ld.global.nc.v2.f64 {%0, %1}, [%2];" : "=d"(r.x), "=d"(r.y) : "l"(p));
  return r;
}

// radix-16 DFT as 4 x 4 with internal twiddles W16^t = tw[t * step16]
template <typename T, int SIGN> struct Bfly16 {
  __device__ __forceinline__ static void run(C2<T>* v, const C2<T>* __restrict__ tw,
                                             int step16) {
    C2<T> a[4][4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
      C2<T> x[4] = {v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]};
      Bfly<T, 4, SIGN>::run(x);
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1) {
        if (n1 * k1 == 0) {
          a[n1][k1] = x[k1];
        } else {
          C2<T> w = ldtw<T>(tw + (n1 * k1) * step16);
          if (SIGN > 0) w.y = -w.y;
          a[n1][k1] = cmul<T>(x[k1], w);
        }
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      C2<T> x[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
      Bfly<T, 4, SIGN>::run(x);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = x[k2];
    }
  }
};

// radix-32 DFT as 8 x 4: X[k1 + 4 k2] = sum_n1 W8^{n1 k2} W32^{n1 k1} (DFT4 of v[n1 + 8m])
template <typename T, int SIGN> struct Bfly32 {
  __device__ __forceinline__ static void run(C2<T>* v, const C2<T>* __restrict__ tw,
                                             int step32) {
    C2<T> a[8][4];
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) {
      C2<T> x[4] = {v[n1], v[n1 + 8], v[n1 + 16], v[n1 + 24]};
      Bfly<T, 4, SIGN>::run(x);
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1) {
        if (n1 * k1 == 0) {
          a[n1][k1] = x[k1];
        } else {
          C2<T> w = ldtw<T>(tw + (n1 * k1) * step32);
          if (SIGN > 0) w.y = -w.y;
          a[n1][k1] = cmul<T>(x[k1], w);
        }
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      C2<T> x[8];
#pragma unroll
      for (int n1 = 0; n1 < 8; ++n1) x[n1] = a[n1][k1];
      Bfly<T, 8, SIGN>::run(x);
#pragma unroll
      for (int k2 = 0; k2 < 8; ++k2) v[k1 + 4 * k2] = x[k2];
    }
  }
};

// synchronisation of the threads of one transform (TPT = L/32 threads, aligned groups)
__device__ __forceinline__ void wsync(int TPT) {
  if (TPT <= 32) {
    __syncwarp();
  } else {
    // two warps per transform (L = 2048): named barrier 1 + pair index
    const int id = 1 + (threadIdx.x >> 6);
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(64) : "memory");
  }
}

// One stage of radix R (W = 32 elements per thread, W/R butterflies) on padded buf.
template <typename T, int R, int SIGN>
__device__ __forceinline__ void wstage(C2<T>* buf, int L, int Ns, int t, bool active,
                                       const C2<T>* __restrict__ tw) {
  constexpr int W = 32;
  const int TPT = L / W;
  const int LR = L / R;
  C2<T> v[W];
  if (active) {
#pragma unroll
    for (int b = 0; b < W / R; ++b) {
      const int j = t + b * TPT;
#pragma unroll
      for (int r = 0; r < R; ++r) v[b * R + r] = buf[pad32(j + r * LR)];
    }
  }
  wsync(TPT);
  if (active) {
    const int tstep = L / (Ns * R);
    const int a = __ffs(Ns) - 1;
#pragma unroll
    for (int b = 0; b < W / R; ++b) {
      const int j = t + b * TPT;
      const int qd = j >> a;
      const int k = j - (qd << a);
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C2<T> w = ldtw<T>(tw + k * r * tstep);
          if (SIGN > 0) w.y = -w.y;
          v[b * R + r] = cmul<T>(v[b * R + r], w);
        }
      }
      if (R == 32)
        Bfly32<T, SIGN>::run(&v[b * R], tw, L / 32);
      else if (R == 16)
        Bfly16<T, SIGN>::run(&v[b * R], tw, L / 16);
      else
        Bfly<T, (R == 8 ? 8 : (R == 4 ? 4 : 2)), SIGN>::run(&v[b * R]);
      const int d = qd * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[pad32(d + r * Ns)] = v[b * R + r];
    }
  }
  wsync(TPT);
}

// Full transform of a power-of-two length 32 <= L <= 2048, in place in padded buf.
template <typename T, int SIGN>
__device__ __forceinline__ void fft_warp(C2<T>* buf, int L, int t, bool active,
                                         const C2<T>* __restrict__ tw) {
  wstage<T, 32, SIGN>(buf, L, 1, t, active, tw);
  int rem = L / 32, Ns = 32;
  if (rem >= 32) {
    wstage<T, 32, SIGN>(buf, L, Ns, t, active, tw);
    rem /= 32;
    Ns *= 32;
  }
  if (rem == 16) wstage<T, 16, SIGN>(buf, L, Ns, t, active, tw);
  else if (rem == 8) wstage<T, 8, SIGN>(buf, L, Ns, t, active, tw);
  else if (rem == 4) wstage<T, 4, SIGN>(buf, L, Ns, t, active, tw);
  else if (rem == 2) wstage<T, 2, SIGN>(buf, L, Ns, t, active, tw);
}

__host__ __device__ inline bool warp_fft_ok(int L) {
  return L >= 32 && L <= 2048 && (L & (L - 1)) == 0;
}

// signed frequency of index n of length L, with a Nyquist flag
// Eigenvalue of the 4th-order second-difference stencil (-1, 16, -30, 16, -1) / (12 h^2)
// on L points at the frequency with cosine c:  L^2 (-2 cos 2t + 32 cos t - 30) / 12
// = L^2 (1 - c)(c - 7) / 3.
template <typename T>
__device__ __forceinline__ T fd_lap(T c, int L) {
  return ((T)1 - c) * (c - (T)7) / (T)3 * (T)L * (T)L;
}
// The same eigenvalue in FP32 from a twiddle w = (cos t, -+sin t), with 1 - cos t formed as
// sin^2 t / (1 + cos t) where cos t > 0: no cancellation at the lowest frequencies, which
// carry most of a Poisson solution (1 - cos t from an FP32 cosine would lose ~5 digits at
// t = 2 pi / 1024).
__device__ __forceinline__ float fd_lap_w(float2 w, int L) {
  const float omc = w.x > 0.f ? w.y * w.y / (1.f + w.x) : 1.f - w.x;
  return omc * (w.x - 7.f) / 3.f * (float)L * (float)L;
}
template <typename T>
__device__ __forceinline__ T inv_or_zero(T x) {
  return x == (T)0 ? (T)0 : (T)1 / x;
}
// Gaussian low-pass exp(-((k1 / (M/4))^2 + (k2 / (N/4))^2) / 2) of COL_POISSON_LP (1 else)
template <typename T, int MODE>
__device__ __forceinline__ T lowpass(int k1, int k2, int M, int N) {
  if (MODE != COL_POISSON_LP) return (T)1;
  const double a = (double)k1 / (0.25 * M), b = (double)k2 / (0.25 * N);
  return (T)exp(-0.5 * (a * a + b * b));
}
template <int MODE>
__device__ __forceinline__ float lowpass_f(int k1, int k2, int M, int N) {
  if (MODE != COL_POISSON_LP) return 1.f;
  const float a = (float)k1 / (0.25f * (float)M), b = (float)k2 / (0.25f * (float)N);
  return expf(-0.5f * (a * a + b * b));
}
__device__ __forceinline__ int sfreq(int n, int L, bool* nyq) {
  *nyq = (2 * n == L);
  return (2 * n <= L) ? n : n - L;
}

// Derivative symbols come from per-plan tables (SpecTables::symx, symy): entry k holds
// (s1, s2) with i s1 the first-derivative symbol (0 at Nyquist) and s2 the second-
// derivative symbol of frequency index k along x (k <= M/2) or y (k < N): the paper's
// spectral symbols 2 pi k and -(2 pi k)^2 (Sec. 4.2), or those of the 4th-order stencils.
//
// rho-bar(k) = 1 / (abar11 d11 + 2 abar12 d1 d2 + abar22 d22 + bbar1 d1 + bbar2 d2), 0 where
// the denominator is 0; sx = (s1, s2) of k1, sy of k2.
template <typename T>
__device__ __forceinline__ C2<T> rho_bar(const T ab[5], C2<T> sx, C2<T> sy) {
  T dr = ab[0] * sx.y - (T)2 * ab[1] * sx.x * sy.x + ab[2] * sy.y;
  T di = ab[3] * sx.x + ab[4] * sy.x;
  T den = dr * dr + di * di;
  if (den == (T)0) return mk2<T>((T)0, (T)0);
  return mk2<T>(dr / den, -di / den);
}

// ---------------------------------------------------------------------------------------
// Row real-to-complex transform (forward), packed output.
// ---------------------------------------------------------------------------------------
template <typename T> struct MaxThreads {
  static constexpr int value = sizeof(T) == 8 ? 256 : 512;
};

// The real-to-complex split of one row: buf holds the length-L complex transform Z of the
// row's M = 2L real values packed as z_n = x_2n + i x_(2n+1); out receives the half
// spectrum X_0..X_(L-1) (X_0 and the Nyquist value X_L packed as (X_0, X_L), both real).
template <typename T>
__device__ __forceinline__ void r2c_split_store(const C2<T>* buf, C2<T>* __restrict__ out, int L,
                                                int t, int TPT, const C2<T>* __restrict__ twM) {
  for (int k = t; k <= L / 2; k += TPT) {
    if (k == 0) {
      C2<T> z = buf[0];
      out[0] = mk2<T>(z.x + z.y, z.x - z.y);
    } else {
      C2<T> zk = buf[k], zm = buf[L - k];
      // E = (Zk + conj Zm)/2, O = -i (Zk - conj Zm)/2, X_k = E + W_M^k O,
      // X_{L-k} = conj(E - W_M^k O)
      C2<T> Ev = mk2<T>((T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y));
      C2<T> Ov = mk2<T>((T)0.5 * (zk.y + zm.y), (T)-0.5 * (zk.x - zm.x));
      C2<T> wo = cmul<T>(twM[k], Ov);
      out[k] = cadd<T>(Ev, wo);
      if (2 * k != L) out[L - k] = cconj<T>(csub<T>(Ev, wo));
    }
  }
}

template <typename T, int E>
__global__ void __launch_bounds__(MaxThreads<T>::value) k_row_r2c(const T* __restrict__ xbase, size_t x_stride,
                          const int* __restrict__ jptr, const double* __restrict__ scale,
                          C2<T>* __restrict__ spec, int N, int M,
                          const C2<T>* __restrict__ twL, const C2<T>* __restrict__ twM,
                          const int* __restrict__ skip, Bat bat, const DevScalars* msc) {
  xbase = badv(xbase, bat);
  jptr = badv(jptr, bat);
  scale = badv(scale, bat);
  spec = badv(spec, bat);
  skip = badv(skip, bat);
  msc = badv(msc, bat);
  if ((skip && *skip) || (msc && bskip(msc, bat))) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* sm = reinterpret_cast<C2<T>*>(smem_raw);
  const int L = M / 2;
  const int TPT = L / E;
  const int q = threadIdx.x / TPT, t = threadIdx.x % TPT;
  const int RB = blockDim.x / TPT;
  const int row = blockIdx.x * RB + q;
  const bool active = row < N;
  C2<T>* buf = sm + q * FB(L);
  int jv = jptr ? *jptr : 0;
  const T* x = xbase + (size_t)jv * x_stride;
  const T sc = scale ? (T)scale[jv] : (T)1;
  if (active) {
    const C2<T>* xr = reinterpret_cast<const C2<T>*>(x + (size_t)row * M);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int n = t + e * TPT;
      C2<T> z = xr[n];
      buf[n] = mk2<T>(z.x * sc, z.y * sc);
    }
  }
  __syncthreads();
  fft_smem<T, E, -1>(buf, L, t, active, twL);
  if (active) r2c_split_store<T>(buf, spec + (size_t)row * L, L, t, TPT, twM);
}

// ---------------------------------------------------------------------------------------
// Column transforms with the spectral multiplies of Strain's method.
// ---------------------------------------------------------------------------------------
// Q (columns per block) is a power of two
// columns col0 .. col0 + Q - 1 of an N x Lc spectrum <-> shared memory, column q at
// sm + q * cs
template <typename T, int E>
__device__ __forceinline__ void col_load(const C2<T>* __restrict__ src, C2<T>* sm, int N,
                                         int Lc, int Q, int col0, int cs) {
  const int lq = __ffs(Q) - 1;
  for (int idx = threadIdx.x; idx < Q * N; idx += blockDim.x) {
    const int n = idx >> lq, q = idx & (Q - 1);
    const int col = col0 + q;
    if (col < Lc) sm[q * cs + n] = src[(size_t)n * Lc + col];
  }
}

template <typename T, int E>
__device__ __forceinline__ void col_store(C2<T>* __restrict__ dst, const C2<T>* sm, int N,
                                          int Lc, int Q, int col0, int cs) {
  const int lq = __ffs(Q) - 1;
  for (int idx = threadIdx.x; idx < Q * N; idx += blockDim.x) {
    const int n = idx >> lq, q = idx & (Q - 1);
    const int col = col0 + q;
    if (col < Lc) dst[(size_t)n * Lc + col] = sm[q * cs + n];
  }
}

// the FP32 matvec column pass with 4 elements per thread runs its three inverse transforms
// interleaved (3 buffers per column); with 8 or 12 the registers would spill
template <typename T, int E, int MODE>
__host__ __device__ constexpr int col_nbuf() {
  return (MODE == COL_MATVEC && sizeof(T) == 4 && E == 4) ? 3 : 1;
}

// (the FP32 pass with 4 elements per thread is held to 64 registers, so that two blocks of
// 512 threads fit on an SM: 256 blocks at 1024^2 then run in one wave)
template <typename T, int E, int MODE>
__global__ void __launch_bounds__(MaxThreads<T>::value, (E == 4 && sizeof(T) == 4) ? 2 : 1)
    k_col(const C2<T>* __restrict__ spec, C2<T>* __restrict__ out0,
                      C2<T>* __restrict__ out1, C2<T>* __restrict__ out2, int N, int M, int Q,
                      double inv_nm,
                      const C2<T>* __restrict__ twN, const C2<T>* __restrict__ twM,
                      const DevScalars* __restrict__ sc, const int* __restrict__ skip,
                      const C2<T>* __restrict__ symx, const C2<T>* __restrict__ symy, Bat bat) {
  spec = badv(spec, bat);
  out0 = badv(out0, bat);
  out1 = badv(out1, bat);
  out2 = badv(out2, bat);
  sc = badv(sc, bat);
  skip = badv(skip, bat);
  if ((skip && *skip) || (sc && bskip(sc, bat))) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* sm = reinterpret_cast<C2<T>*>(smem_raw);
  const int Lc = M / 2;
  const int TPT = N / E;
  const int q = threadIdx.x / TPT, t = threadIdx.x % TPT;
  const int col0 = blockIdx.x * Q;
  const int col = col0 + q;
  const bool active = (q < Q) && (col < Lc);
  constexpr int NBUF = col_nbuf<T, E, MODE>();
  const int cs = NBUF * FB(N);
  C2<T>* buf = sm + q * cs;

  // the interleaved FP32 matvec pass keeps its stage twiddle table in shared memory (after
  // the columns' buffers): every stage reads R - 1 twiddles per butterfly, and from global
  // memory those loads sat on the stage chain's critical path
  const C2<T>* twS = twN;
  if (NBUF == 3) {
    C2<T>* tws = sm + Q * cs;
    const C2<T>* src = twN + (size_t)stage_table_slot<E>() * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tws[i] = src[i];
    twS = tws - (size_t)stage_table_slot<E>() * N;  // the fft routines add the slot back
  }
  col_load<T, E>(spec, sm, N, Lc, Q, col0, cs);
  __syncthreads();
  if (MODE == COL_INV) {
    fft_smem<T, E, +1>(buf, N, t, active, twN);
    col_store<T, E>(out0, sm, N, Lc, Q, col0, cs);
    return;
  }
  fft_smem<T, E, -1>(buf, N, t, active, twS);
  if (MODE == COL_FWD) {
    col_store<T, E>(out0, sm, N, Lc, Q, col0, cs);
    return;
  }
  T ab[5];
#pragma unroll
  for (int a = 0; a < 5; ++a)
    ab[a] = sc ? (T)(MODE == COL_LBARINV ? sc->abar_n[a] : sc->abar[a]) : (T)0;
  const T inv = (T)inv_nm;
  C2<T> s[E], s0[E];
  if (active) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = t + e * TPT;
      bool nyq2;
      const int k2 = sfreq(k, N, &nyq2);
      C2<T> z = buf[k];
      C2<T> r;
      if (col == 0) {
        // unpack the two real columns k1 = 0 and k1 = M/2 carried as X0 + i XL
        C2<T> p = buf[(N - k) % N];
        C2<T> A = mk2<T>((T)0.5 * (z.x + p.x), (T)0.5 * (z.y - p.y));
        C2<T> B = mk2<T>((T)0.5 * (z.y + p.y), (T)-0.5 * (z.x - p.x));
        if (MODE == COL_POISSON || MODE == COL_POISSON_LP) {
          const T ly = fd_lap<T>(twN[k].x, N);
          A = cscale<T>(A, inv_or_zero<T>(ly) * lowpass<T, MODE>(0, k2, M, N));
          B = cscale<T>(B, inv_or_zero<T>(fd_lap<T>((T)-1, M) + ly) *
                               lowpass<T, MODE>(M / 2, k2, M, N));
        } else {
          A = cmul<T>(rho_bar<T>(ab, symx[0], symy[k]), A);
          B = cmul<T>(rho_bar<T>(ab, symx[M / 2], symy[k]), B);
          // the matvec's Q0 carries its Nyquist channel premultiplied by d11(M/2) =
          // -(2 pi M/2)^2, so that the two channels sharing the complex column have
          // comparable magnitudes; formed here from the unpacked channels (recovering one
          // channel from the packed sum would cost eps times the other's magnitude)
          if (MODE == COL_MATVEC) {
            const C2<T> Bn = cscale<T>(B, symx[M / 2].y);
            s0[e] = cscale<T>(mk2<T>(A.x - Bn.y, A.y + Bn.x), inv);
          }
        }
        r = mk2<T>(A.x - B.y, A.y + B.x);  // A + i B
      } else {
        if (MODE == COL_POISSON || MODE == COL_POISSON_LP) {
          r = cscale<T>(z, inv_or_zero<T>(fd_lap<T>(twM[col].x, M) + fd_lap<T>(twN[k].x, N)) *
                               lowpass<T, MODE>(col, k2, M, N));
        } else {
          r = cmul<T>(rho_bar<T>(ab, symx[col], symy[k]), z);
        }
      }
      s[e] = cscale<T>(r, inv);
    }
  }
  __syncthreads();
  if (NBUF == 3) {
    // Q0 = S (Nyquist channel premultiplied), Q1 = (i s1(k2)) S, Q2 = s2(k2) S into the
    // three buffers, then the three inverse transforms interleaved (in place: ping-pong
    // stages cost this kernel more in registers, capped at 64 for two blocks per SM, than
    // they save in barriers)
    if (active) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int k = t + e * TPT;
        const C2<T> v = s[e];
        const C2<T> sy = symy[k];
        buf[k] = col == 0 ? s0[e] : v;
        buf[FB(N) + k] = mk2<T>(-sy.x * v.y, sy.x * v.x);
        buf[2 * FB(N) + k] = cscale<T>(v, sy.y);
      }
    }
    __syncthreads();
    C2<T>* const bufs[3] = {buf, buf + FB(N), buf + 2 * FB(N)};
    fft_smem_multi<T, E, +1, 3>(bufs, N, t, active, twS);
    col_store<T, E>(out0, sm, N, Lc, Q, col0, cs);
    col_store<T, E>(out1, sm + FB(N), N, Lc, Q, col0, cs);
    col_store<T, E>(out2, sm + 2 * FB(N), N, Lc, Q, col0, cs);
    return;
  }
  const int nout = (MODE == COL_MATVEC) ? 3 : 1;
#pragma unroll 1
  for (int p = 0; p < nout; ++p) {
    if (active) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int k = t + e * TPT;
        C2<T> v = (MODE == COL_MATVEC && p == 0 && col == 0) ? s0[e] : s[e];
        if (p == 1) {  // (i s1(k2)) S, zero at Nyquist
          const T s1 = symy[k].x;
          v = mk2<T>(-s1 * v.y, s1 * v.x);
        } else if (p == 2) {  // s2(k2) S
          v = cscale<T>(v, symy[k].y);
        }
        buf[k] = v;
      }
    }
    __syncthreads();
    fft_smem<T, E, +1>(buf, N, t, active, twN);
    col_store<T, E>(p == 0 ? out0 : (p == 1 ? out1 : out2), sm, N, Lc, Q, col0, cs);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Row complex-to-real inverse transforms (raw: sum over the full Hermitian spectrum).
// ---------------------------------------------------------------------------------------
// row symbol kinds: 0 = 1, 1 = d/dx (i s1 of k1), 2 = d2/dx2 (s2 of k1) from the symbol
// table symx (kind 2 expects a matvec Q0, whose packed Nyquist channel is premultiplied)
template <typename T>
__device__ __forceinline__ C2<T> row_symbol_apply(C2<T> X, int k, int kind,
                                                  const C2<T>* __restrict__ symx) {
  if (kind == 0) return X;
  if (k == 0) {
    // packed (X0, XL): k1 = 0 and k1 = M/2 (Nyquist).  For d2/dx2 the Nyquist channel of
    // Q0 already carries the factor s2(M/2): the column pass applies it before its
    // inverse transform (see k_col), so that the two channels sharing one complex column
    // have comparable magnitudes.
    if (kind == 1) return mk2<T>((T)0, (T)0);
    return mk2<T>((T)0, X.y);
  }
  const C2<T> sx = symx[k];
  if (kind == 1) return mk2<T>(-sx.x * X.y, sx.x * X.x);
  return cscale<T>(X, sx.y);
}

// the FP32 row combine with 4 elements per thread runs its five transforms interleaved
// (5 buffers per row, and 5 scratch buffers for the ping-pong stages)
template <typename T, int E, int MODE>
__host__ __device__ constexpr int row_nbuf() {
  return (MODE == ROWINV_COMBINE && sizeof(T) == 4 && E == 4) ? 10 : 1;
}

// complex-to-real pre-processing on a packed row in buf (in place):
// Z_k = (X_k + conj X_{L-k}) + i (X_k - conj X_{L-k}) conj(W_M^k)
template <typename T>
__device__ __forceinline__ void c2r_preprocess(C2<T>* buf, int L, int t, int TPT, bool active,
                                               const C2<T>* __restrict__ twM) {
  if (active) {
    for (int k = t; k <= L / 2; k += TPT) {
      if (k == 0) {
        C2<T> x = buf[0];
        buf[0] = mk2<T>(x.x + x.y, x.x - x.y);
      } else {
        C2<T> xk = buf[k], xm = buf[L - k];
        C2<T> Ev = mk2<T>(xk.x + xm.x, xk.y - xm.y);
        C2<T> dv = mk2<T>(xk.x - xm.x, xk.y + xm.y);
        C2<T> Ov = cmul<T>(dv, cconj<T>(twM[k]));
        buf[k] = mk2<T>(Ev.x - Ov.y, Ev.y + Ov.x);
        if (2 * k != L) buf[L - k] = mk2<T>(Ev.x + Ov.y, -Ev.y + Ov.x);
      }
    }
  }
  __syncthreads();
}

// the same for NB rows at once (one pass, one barrier)
template <typename T, int NB>
__device__ __forceinline__ void c2r_preprocess_multi(C2<T>* const (&bufs)[NB], int L, int t,
                                                     int TPT, bool active,
                                                     const C2<T>* __restrict__ twM) {
  if (active) {
    for (int k = t; k <= L / 2; k += TPT) {
      if (k == 0) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const C2<T> x = bufs[b][0];
          bufs[b][0] = mk2<T>(x.x + x.y, x.x - x.y);
        }
      } else {
        const C2<T> w = cconj<T>(twM[k]);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const C2<T> xk = bufs[b][k], xm = bufs[b][L - k];
          const C2<T> Ev = mk2<T>(xk.x + xm.x, xk.y - xm.y);
          const C2<T> dv = mk2<T>(xk.x - xm.x, xk.y + xm.y);
          const C2<T> Ov = cmul<T>(dv, w);
          bufs[b][k] = mk2<T>(Ev.x - Ov.y, Ev.y + Ov.x);
          if (2 * k != L) bufs[b][L - k] = mk2<T>(Ev.x + Ov.y, -Ev.y + Ov.x);
        }
      }
    }
  }
  __syncthreads();
}

template <typename T, int E, int MODE>
__global__ void __launch_bounds__(MaxThreads<T>::value) k_row_c2r(const C2<T>* __restrict__ q0, const C2<T>* __restrict__ q1,
                          const C2<T>* __restrict__ q2, const T* __restrict__ coef,
                          T* __restrict__ out, const double* __restrict__ u_in,
                          double* __restrict__ u_out, double step, double out_scale, int N,
                          int M, const C2<T>* __restrict__ twL, const C2<T>* __restrict__ twM,
                          const int* __restrict__ skip, const DevScalars* __restrict__ sc,
                          const C2<T>* __restrict__ symx, Bat bat) {
  q0 = badv(q0, bat);
  q1 = badv(q1, bat);
  q2 = badv(q2, bat);
  coef = badv(coef, bat);
  out = badv(out, bat);
  u_in = badv(u_in, bat);
  u_out = badv(u_out, bat);
  skip = badv(skip, bat);
  sc = badv(sc, bat);
  if ((skip && *skip) || (sc && bskip(sc, bat))) return;
  if (MODE == ROWINV_UPDATE && sc) {
    // device-resident control: step s and the current/candidate buffers come from sc
    step = sc->step_s;
    if (sc->upar & 1) {
      double* t = const_cast<double*>(u_in);
      u_in = u_out;
      u_out = t;
    }
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* sm = reinterpret_cast<C2<T>*>(smem_raw);
  const int L = M / 2;
  const int TPT = L / E;
  const int q = threadIdx.x / TPT, t = threadIdx.x % TPT;
  const int RB = blockDim.x / TPT;
  const int row = blockIdx.x * RB + q;
  const bool active = row < N;
  constexpr int NBUF = row_nbuf<T, E, MODE>();
  C2<T>* buf = sm + q * NBUF * FB(L);
  const size_t P = (size_t)N * M;
  C2<T> acc[E];
#pragma unroll
  for (int e = 0; e < E; ++e) acc[e] = mk2<T>((T)0, (T)0);

  if (NBUF == 10) {
    // the five terms' transforms interleaved: d_xx Q0, d_x Q0, d_x Q1, Q1, Q2 in buffers 0..4
    if (active) {
      const size_t o = (size_t)row * L;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int k = t + e * TPT;
        const C2<T> x0 = q0[o + k], x1 = q1[o + k];
        buf[k] = row_symbol_apply<T>(x0, k, 2, symx);
        buf[FB(L) + k] = row_symbol_apply<T>(x0, k, 1, symx);
        buf[2 * FB(L) + k] = row_symbol_apply<T>(x1, k, 1, symx);
        buf[3 * FB(L) + k] = x1;
        buf[4 * FB(L) + k] = q2[o + k];
      }
    }
    __syncthreads();
    C2<T>* const bufs[5] = {buf, buf + FB(L), buf + 2 * FB(L), buf + 3 * FB(L),
                            buf + 4 * FB(L)};
    C2<T>* const scr[5] = {buf + 5 * FB(L), buf + 6 * FB(L), buf + 7 * FB(L),
                           buf + 8 * FB(L), buf + 9 * FB(L)};
    c2r_preprocess_multi<T, 5>(bufs, L, t, TPT, active, twM);
    fft_smem_multi_pp<T, E, +1, 5>(bufs, scr, L, t, active, twL);
    if (!active) return;
    const size_t o = (size_t)row * M;
    const C2<T>* c0 = reinterpret_cast<const C2<T>*>(coef + o);
    const C2<T>* c1 = reinterpret_cast<const C2<T>*>(coef + P + o);
    const C2<T>* c2 = reinterpret_cast<const C2<T>*>(coef + 2 * P + o);
    const C2<T>* c3 = reinterpret_cast<const C2<T>*>(coef + 3 * P + o);
    const C2<T>* c4 = reinterpret_cast<const C2<T>*>(coef + 4 * P + o);
    C2<T>* ov = reinterpret_cast<C2<T>*>(out + o);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int n = t + e * TPT;
      const C2<T> y0 = buf[n], y1 = buf[FB(L) + n], y2 = buf[2 * FB(L) + n],
                  y3 = buf[3 * FB(L) + n], y4 = buf[4 * FB(L) + n];
      const C2<T> a11 = c0[n], a12 = c1[n], a22 = c2[n], b1 = c3[n], b2 = c4[n];
      C2<T> r;
      r.x = a11.x * y0.x + b1.x * y1.x + (T)2 * a12.x * y2.x + b2.x * y3.x + a22.x * y4.x;
      r.y = a11.y * y0.y + b1.y * y1.y + (T)2 * a12.y * y2.y + b2.y * y3.y + a22.y * y4.y;
      ov[n] = r;
    }
    return;
  }

  const int nterm = (MODE == ROWINV_COMBINE) ? 5 : 1;
#pragma unroll 1
  for (int p = 0; p < nterm; ++p) {
    // term p: source plane, row symbol, coefficient plane, multiplicity
    const C2<T>* src = q0;
    int kind = 0, cidx = 0;
    T mult = (T)1;
    if (MODE == ROWINV_COMBINE) {
      if (p == 0) { src = q0; kind = 2; cidx = 0; }              // a11 * d_xx Lbar^-1 s
      else if (p == 1) { src = q0; kind = 1; cidx = 3; }         // b1  * d_x  Lbar^-1 s
      else if (p == 2) { src = q1; kind = 1; cidx = 1; mult = (T)2; }  // 2 a12 * d_xy
      else if (p == 3) { src = q1; kind = 0; cidx = 4; }         // b2  * d_y
      else { src = q2; kind = 0; cidx = 2; }                     // a22 * d_yy
    }
    if (active) {
      const C2<T>* sr = src + (size_t)row * L;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int k = t + e * TPT;
        buf[k] = row_symbol_apply<T>(sr[k], k, kind, symx);
      }
    }
    __syncthreads();
    c2r_preprocess<T>(buf, L, t, TPT, active, twM);
    fft_smem<T, E, +1>(buf, L, t, active, twL);
    if (active) {
      if (MODE == ROWINV_COMBINE) {
        const C2<T>* cr = reinterpret_cast<const C2<T>*>(coef + (size_t)cidx * P +
                                                         (size_t)row * M);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int n = t + e * TPT;
          C2<T> z = buf[n], a = cr[n];
          acc[e].x += mult * a.x * z.x;
          acc[e].y += mult * a.y * z.y;
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = buf[t + e * TPT];
      }
    }
    __syncthreads();
  }
  if (!active) return;
  if (MODE == ROWINV_UPDATE) {
    const double2* ui = reinterpret_cast<const double2*>(u_in + (size_t)row * M);
    double2* uo = reinterpret_cast<double2*>(u_out + (size_t)row * M);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int n = t + e * TPT;
      double2 a = ui[n];
      a.x += step * (double)acc[e].x;
      a.y += step * (double)acc[e].y;
      uo[n] = a;
    }
  } else {
    C2<T>* o = reinterpret_cast<C2<T>*>(out + (size_t)row * M);
    const T os = (T)out_scale;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int n = t + e * TPT;
      o[n] = (MODE == ROWINV_PLAIN) ? cscale<T>(acc[e], os) : acc[e];
    }
  }
}

// ---------------------------------------------------------------------------------------
// Concurrent-transform variants of the two dominant passes (FP32).  At 1024^2 a pass with
// one transform group per column/row launches fewer blocks than the GPU has SMs and is
// latency-bound, so these run the independent transforms of a column/row at the same
// time in separate thread groups with their own shared-memory buffers.
// ---------------------------------------------------------------------------------------
#define OTGB_PAR_THREADS 768

// Column pass of the matvec: forward column FFT (group 0), S = rho-bar sigma-hat / (N M),
// then the inverse column FFTs of S, (2 pi i k2) S and -(2 pi k2)^2 S in groups 0, 1, 2.
template <typename T, int E>
__global__ void __launch_bounds__(OTGB_PAR_THREADS)
    k_col_matvec_par(const C2<T>* __restrict__ spec, C2<T>* __restrict__ out0,
                     C2<T>* __restrict__ out1, C2<T>* __restrict__ out2, int N, int M, int Q,
                     double inv_nm,
                     const C2<T>* __restrict__ twN, const DevScalars* __restrict__ sc,
                     const int* __restrict__ skip, const C2<T>* __restrict__ symx,
                     const C2<T>* __restrict__ symy) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* sm = reinterpret_cast<C2<T>*>(smem_raw);
  const int Lc = M / 2, TPT = N / E, G = Q * TPT;
  const int grp = threadIdx.x / G, rem = threadIdx.x - grp * G;
  const int q = rem / TPT, t = rem - q * TPT;
  const int col0 = blockIdx.x * Q, col = col0 + q;
  const bool active = col < Lc;
  const int stride = Q * FB(N);  // one group's buffers
  C2<T>* buf = sm + grp * stride + q * FB(N);
  C2<T>* b0 = sm + q * FB(N);
  const int lq = __ffs(Q) - 1;
  for (int idx = threadIdx.x; idx < Q * N; idx += blockDim.x) {
    const int n = idx >> lq, qq = idx & (Q - 1);
    if (col0 + qq < Lc) sm[qq * FB(N) + n] = spec[(size_t)n * Lc + col0 + qq];
  }
  __syncthreads();
  fft_smem<T, E, -1>(b0, N, t, active && grp == 0, twN);
  T ab[5];
#pragma unroll
  for (int a = 0; a < 5; ++a) ab[a] = (T)sc->abar[a];
  const T inv = (T)inv_nm;
  // Q1 and Q2 go to their own buffers at once; Q0 (written over the spectrum that the
  // partner reads of column 0 still need) is held in registers until after the barrier.
  // Column 0's Q0 carries the Nyquist channel premultiplied by d11(M/2) = -(2 pi M/2)^2
  // so that the two channels sharing the complex column have comparable magnitudes.
  C2<T> s0[E];
  const bool lead = active && grp == 0;
  if (lead) {
    const T d11n = symx[M / 2].y;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = t + e * TPT;
      const C2<T> sy = symy[k];
      C2<T> z = b0[k], v;
      if (col == 0) {
        C2<T> pz = b0[(N - k) % N];
        C2<T> A = mk2<T>((T)0.5 * (z.x + pz.x), (T)0.5 * (z.y - pz.y));
        C2<T> B = mk2<T>((T)0.5 * (z.y + pz.y), (T)-0.5 * (z.x - pz.x));
        A = cscale<T>(cmul<T>(rho_bar<T>(ab, symx[0], symy[k]), A), inv);
        B = cscale<T>(cmul<T>(rho_bar<T>(ab, symx[M / 2], symy[k]), B), inv);
        v = mk2<T>(A.x - B.y, A.y + B.x);
        const C2<T> Bn = cscale<T>(B, d11n);
        s0[e] = mk2<T>(A.x - Bn.y, A.y + Bn.x);
      } else {
        v = cscale<T>(cmul<T>(rho_bar<T>(ab, symx[col], symy[k]), z), inv);
        s0[e] = v;
      }
      b0[stride + k] = mk2<T>(-sy.x * v.y, sy.x * v.x);
      b0[2 * stride + k] = cscale<T>(v, sy.y);
    }
  }
  __syncthreads();
  if (lead) {
#pragma unroll
    for (int e = 0; e < E; ++e) b0[t + e * TPT] = s0[e];
  }
  __syncthreads();
  fft_smem<T, E, +1>(buf, N, t, active, twN);
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    C2<T>* dst = g == 0 ? out0 : (g == 1 ? out1 : out2);
    for (int idx = threadIdx.x; idx < Q * N; idx += blockDim.x) {
      const int n = idx >> lq, qq = idx & (Q - 1);
      if (col0 + qq < Lc) dst[(size_t)n * Lc + col0 + qq] = sm[g * stride + qq * FB(N) + n];
    }
  }
}

// Row pass of the matvec: the five complex-to-real transforms of a row (d_xx Q0, d_x Q0,
// d_x Q1, Q1, Q2) in groups 0..4, then w = a11 . + b1 . + 2 a12 . + b2 . + a22 .
template <typename T, int E>
__global__ void __launch_bounds__(OTGB_PAR_THREADS)
    k_row_combine_par(const C2<T>* __restrict__ q0, const C2<T>* __restrict__ q1,
                      const C2<T>* __restrict__ q2, const T* __restrict__ coef,
                      T* __restrict__ out, int N, int M, int RB, const C2<T>* __restrict__ twL,
                      const C2<T>* __restrict__ twM, const int* __restrict__ skip,
                      const C2<T>* __restrict__ symx) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* sm = reinterpret_cast<C2<T>*>(smem_raw);
  const int L = M / 2, TPT = L / E, G = RB * TPT;
  const int grp = threadIdx.x / G, rem = threadIdx.x - grp * G;
  const int q = rem / TPT, t = rem - q * TPT;
  const int row0 = blockIdx.x * RB, row = row0 + q;
  const bool active = row < N;
  const int stride = RB * FB(L);
  C2<T>* buf = sm + grp * stride + q * FB(L);
  const int la = __ffs(L) - 1;
  const bool lp2 = (L >> la) == 1;
  for (int idx = threadIdx.x; idx < RB * L; idx += blockDim.x) {
    const int qq = lp2 ? (idx >> la) : ((idx >> la) / 3), k = idx - qq * L;
    if (row0 + qq < N) {
      const size_t o = (size_t)(row0 + qq) * L + k;
      const C2<T> x0 = q0[o], x1 = q1[o], x2 = q2[o];
      C2<T>* b = sm + qq * FB(L) + k;
      b[0] = row_symbol_apply<T>(x0, k, 2, symx);
      b[stride] = row_symbol_apply<T>(x0, k, 1, symx);
      b[2 * stride] = row_symbol_apply<T>(x1, k, 1, symx);
      b[3 * stride] = x1;
      b[4 * stride] = x2;
    }
  }
  __syncthreads();
  c2r_preprocess<T>(buf, L, t, TPT, active, twM);
  fft_smem<T, E, +1>(buf, L, t, active, twL);
  const size_t P = (size_t)N * M;
  for (int idx = threadIdx.x; idx < RB * L; idx += blockDim.x) {
    const int qq = lp2 ? (idx >> la) : ((idx >> la) / 3), n = idx - qq * L;
    const int r = row0 + qq;
    if (r < N) {
      const size_t o = (size_t)r * M;
      const C2<T>* c0 = reinterpret_cast<const C2<T>*>(coef + o);
      const C2<T>* c1 = reinterpret_cast<const C2<T>*>(coef + P + o);
      const C2<T>* c2 = reinterpret_cast<const C2<T>*>(coef + 2 * P + o);
      const C2<T>* c3 = reinterpret_cast<const C2<T>*>(coef + 3 * P + o);
      const C2<T>* c4 = reinterpret_cast<const C2<T>*>(coef + 4 * P + o);
      const C2<T>* b = sm + qq * FB(L) + n;
      const C2<T> y0 = b[0], y1 = b[stride], y2 = b[2 * stride], y3 = b[3 * stride],
                  y4 = b[4 * stride];
      const C2<T> a11 = c0[n], a12 = c1[n], a22 = c2[n], b1 = c3[n], b2 = c4[n];
      C2<T> acc;
      acc.x = a11.x * y0.x + b1.x * y1.x + (T)2 * a12.x * y2.x + b2.x * y3.x + a22.x * y4.x;
      acc.y = a11.y * y0.y + b1.y * y1.y + (T)2 * a12.y * y2.y + b2.y * y3.y + a22.y * y4.y;
      reinterpret_cast<C2<T>*>(out + o)[n] = acc;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Column pass of theta = Lbar^{-1} sigma for the mixed mode: the forward column FFT and the
// rho-bar multiply in FP32 (their round-off is damped by rho-bar ~ 1/k^2), the inverse
// column FFT in FP64 into an FP64 Q0 for the FP64 row pass that forms the update.  FP32
// round-off in those last passes would be white noise in theta, which the fourth-order
// stencils amplify by ~M^2 at the grid scale.
// ---------------------------------------------------------------------------------------
template <int E>
__global__ void __launch_bounds__(256)
    k_col_lbarinv_mixed(const float2* __restrict__ spec, double2* __restrict__ out, int N,
                        int M, int Q, double inv_nm, const float2* __restrict__ twN32,
                        const double2* __restrict__ twN64, const DevScalars* __restrict__ sc,
                        const float2* __restrict__ symx, const float2* __restrict__ symy) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* sm = reinterpret_cast<double2*>(smem_raw);
  const int Lc = M / 2, TPT = N / E;
  const int q = threadIdx.x / TPT, t = threadIdx.x - q * TPT;
  const int col0 = blockIdx.x * Q, col = col0 + q;
  const bool active = (q < Q) && (col < Lc);
  double2* db = sm + q * FB(N);
  float2* fb = reinterpret_cast<float2*>(db);  // FP32 phase uses the first half
  const int lq = __ffs(Q) - 1;
  for (int idx = threadIdx.x; idx < Q * N; idx += blockDim.x) {
    const int n = idx >> lq, qq = idx & (Q - 1);
    if (col0 + qq < Lc)
      reinterpret_cast<float2*>(sm + qq * FB(N))[n] = spec[(size_t)n * Lc + col0 + qq];
  }
  __syncthreads();
  fft_smem<float, E, -1>(fb, N, t, active, twN32);
  float ab[5];
#pragma unroll
  for (int a = 0; a < 5; ++a) ab[a] = (float)sc->abar_n[a];
  const float inv = (float)inv_nm;
  double2 s[E];
  if (active) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = t + e * TPT;
      float2 z = fb[k], r;
      if (col == 0) {
        float2 pz = fb[(N - k) % N];
        float2 A = mk2<float>(0.5f * (z.x + pz.x), 0.5f * (z.y - pz.y));
        float2 B = mk2<float>(0.5f * (z.y + pz.y), -0.5f * (z.x - pz.x));
        A = cmul<float>(rho_bar<float>(ab, symx[0], symy[k]), A);
        B = cmul<float>(rho_bar<float>(ab, symx[M / 2], symy[k]), B);
        r = mk2<float>(A.x - B.y, A.y + B.x);
      } else {
        r = cmul<float>(rho_bar<float>(ab, symx[col], symy[k]), z);
      }
      s[e] = mk2<double>((double)(r.x * inv), (double)(r.y * inv));
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int e = 0; e < E; ++e) db[t + e * TPT] = s[e];
  }
  __syncthreads();
  fft_smem<double, E, +1>(db, N, t, active, twN64);
  for (int idx = threadIdx.x; idx < Q * N; idx += blockDim.x) {
    const int n = idx >> lq, qq = idx & (Q - 1);
    if (col0 + qq < Lc) out[(size_t)n * Lc + col0 + qq] = sm[qq * FB(N) + n];
  }
}

// Same pass with the inverse column transform in double-float (dd.cuh): the FP64-accuracy
// part of theta on the FP32 pipes.  MODE COL_POISSON / COL_POISSON_LP divides by the
// eigenvalues of the fourth-order FD Laplacian instead (zero mode -> 0; _LP times the
// Gaussian low-pass): the Poisson solves of the learned warm start in mixed precision.
template <int E, int MODE>
__global__ void __launch_bounds__(256)
    k_col_lbarinv_dd(const float2* __restrict__ spec, ddc* __restrict__ out, int N, int M,
                     int Q, double inv_nm, const float2* __restrict__ twN32,
                     const float2* __restrict__ twM32, const ddc* __restrict__ twNdd,
                     const DevScalars* __restrict__ sc, const float2* __restrict__ symx,
                     const float2* __restrict__ symy, Bat bat) {
  spec = badv(spec, bat);
  out = badv(out, bat);
  sc = badv(sc, bat);
  if (sc && bskip(sc, bat)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ddc* sm = reinterpret_cast<ddc*>(smem_raw);
  const int Lc = M / 2, TPT = N / E;
  const int q = threadIdx.x / TPT, t = threadIdx.x - q * TPT;
  const int col0 = blockIdx.x * Q, col = col0 + q;
  const bool active = (q < Q) && (col < Lc);
  ddc* db = sm + q * FB(N);
  float2* fb = reinterpret_cast<float2*>(db);  // FP32 phase uses the first quarter
  const int lq = __ffs(Q) - 1;
  for (int idx = threadIdx.x; idx < Q * N; idx += blockDim.x) {
    const int n = idx >> lq, qq = idx & (Q - 1);
    if (col0 + qq < Lc)
      reinterpret_cast<float2*>(sm + qq * FB(N))[n] = spec[(size_t)n * Lc + col0 + qq];
  }
  __syncthreads();
  fft_smem<float, E, -1>(fb, N, t, active, twN32);
  float ab[5];
#pragma unroll
  for (int a = 0; a < 5; ++a) ab[a] = MODE == COL_LBARINV ? (float)sc->abar_n[a] : 0.f;
  const float inv = (float)inv_nm;
  float2 s[E];
  if (active) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int k = t + e * TPT;
      float2 z = fb[k], r;
      if (col == 0) {
        float2 pz = fb[(N - k) % N];
        float2 A = mk2<float>(0.5f * (z.x + pz.x), 0.5f * (z.y - pz.y));
        float2 B = mk2<float>(0.5f * (z.y + pz.y), -0.5f * (z.x - pz.x));
        if (MODE == COL_LBARINV) {
          A = cmul<float>(rho_bar<float>(ab, symx[0], symy[k]), A);
          B = cmul<float>(rho_bar<float>(ab, symx[M / 2], symy[k]), B);
        } else {
          bool nyq2;
          const int k2 = sfreq(k, N, &nyq2);
          const float ly = fd_lap_w(twN32[k], N);
          const float lxn = -16.f / 3.f * (float)M * (float)M;  // k1 = M/2 (cos t = -1)
          A = cscale<float>(A, inv_or_zero<float>(ly) * lowpass_f<MODE>(0, k2, M, N));
          B = cscale<float>(B, inv_or_zero<float>(lxn + ly) * lowpass_f<MODE>(M / 2, k2, M, N));
        }
        r = mk2<float>(A.x - B.y, A.y + B.x);
      } else if (MODE == COL_LBARINV) {
        r = cmul<float>(rho_bar<float>(ab, symx[col], symy[k]), z);
      } else {
        bool nyq2;
        const int k2 = sfreq(k, N, &nyq2);
        r = cscale<float>(z, inv_or_zero<float>(fd_lap_w(twM32[col], M) + fd_lap_w(twN32[k], N)) *
                                 lowpass_f<MODE>(col, k2, M, N));
      }
      s[e] = mk2<float>(r.x * inv, r.y * inv);
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      ddc v;
      v.x = dd(s[e].x, 0.0f);
      v.y = dd(s[e].y, 0.0f);
      db[t + e * TPT] = v;
    }
  }
  __syncthreads();
  fft_smem<dd, E, +1>(db, N, t, active, twNdd);
  for (int idx = threadIdx.x; idx < Q * N; idx += blockDim.x) {
    const int n = idx >> lq, qq = idx & (Q - 1);
    if (col0 + qq < Lc) out[(size_t)n * Lc + col0 + qq] = sm[qq * FB(N) + n];
  }
}

// theta rows (complex-to-real) in double-float, then u_out = u_in + step theta in FP64
// (u_in == nullptr: u_out = step theta)
template <int E>
__global__ void __launch_bounds__(256)
    k_row_c2r_update_dd(const ddc* __restrict__ q, const double* __restrict__ u_in,
                        double* __restrict__ u_out, double step, int N, int M,
                        const ddc* __restrict__ twL, const ddc* __restrict__ twM,
                        const DevScalars* __restrict__ sc, Bat bat) {
  q = badv(q, bat);
  u_in = badv(u_in, bat);
  u_out = badv(u_out, bat);
  sc = badv(sc, bat);
  if (sc && bskip(sc, bat)) return;
  if (sc) {
    step = sc->step_s;
    if (sc->upar & 1) {
      double* tmp = const_cast<double*>(u_in);
      u_in = u_out;
      u_out = tmp;
    }
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ddc* sm = reinterpret_cast<ddc*>(smem_raw);
  const int L = M / 2, TPT = L / E;
  const int qq = threadIdx.x / TPT, t = threadIdx.x % TPT;
  const int RB = blockDim.x / TPT;
  const int row = blockIdx.x * RB + qq;
  const bool active = row < N;
  ddc* buf = sm + qq * FB(L);
  if (active) {
    const ddc* sr = q + (size_t)row * L;
#pragma unroll
    for (int e = 0; e < E; ++e) buf[t + e * TPT] = sr[t + e * TPT];
  }
  __syncthreads();
  c2r_preprocess<dd>(buf, L, t, TPT, active, twM);
  fft_smem<dd, E, +1>(buf, L, t, active, twL);
  if (!active) return;
  const double2* ui = u_in ? reinterpret_cast<const double2*>(u_in + (size_t)row * M) : nullptr;
  double2* uo = reinterpret_cast<double2*>(u_out + (size_t)row * M);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int n = t + e * TPT;
    const ddc z = buf[n];
    double2 a = ui ? ui[n] : make_double2(0.0, 0.0);
    a.x += step * dd_to_double(z.x);
    a.y += step * dd_to_double(z.y);
    uo[n] = a;
  }
}

// ---------------------------------------------------------------------------------------
// Warp-FFT versions of the three matvec passes (FP32, power-of-two lengths).  Each thread
// holds 32 elements of one transform; the threads of a transform are one warp (or part of
// one) for lengths up to 1024, so its stages synchronise with __syncwarp.
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
    k_row_r2c_w(const T* __restrict__ xbase, size_t x_stride, const int* __restrict__ jptr,
                const double* __restrict__ scale, C2<T>* __restrict__ spec, int N, int M,
                int RB, const C2<T>* __restrict__ twL, const C2<T>* __restrict__ twM,
                const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* sm = reinterpret_cast<C2<T>*>(smem_raw);
  const int L = M / 2, TPT = L / 32, LP = L + L / 32;
  const int q = threadIdx.x / TPT, t = threadIdx.x - q * TPT;
  const int row = blockIdx.x * RB + q;
  const bool active = row < N;
  C2<T>* buf = sm + q * LP;
  const int jv = jptr ? *jptr : 0;
  const T* x = xbase + (size_t)jv * x_stride;
  const T sc = scale ? (T)scale[jv] : (T)1;
  if (active) {
    const C2<T>* xr = reinterpret_cast<const C2<T>*>(x + (size_t)row * M);
#pragma unroll 8
    for (int e = 0; e < 32; ++e) {
      const int n = t + e * TPT;
      const C2<T> z = xr[n];
      buf[pad32(n)] = mk2<T>(z.x * sc, z.y * sc);
    }
  }
  wsync(TPT);
  fft_warp<T, -1>(buf, L, t, active, twL);
  if (active) {
    C2<T>* out = spec + (size_t)row * L;
    for (int k = t; k <= L / 2; k += TPT) {
      if (k == 0) {
        const C2<T> z = buf[0];
        out[0] = mk2<T>(z.x + z.y, z.x - z.y);
      } else {
        const C2<T> zk = buf[pad32(k)], zm = buf[pad32(L - k)];
        const C2<T> Ev = mk2<T>((T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y));
        const C2<T> Ov = mk2<T>((T)0.5 * (zk.y + zm.y), (T)-0.5 * (zk.x - zm.x));
        const C2<T> wo = cmul<T>(twM[k], Ov);
        out[k] = cadd<T>(Ev, wo);
        if (2 * k != L) out[L - k] = cconj<T>(csub<T>(Ev, wo));
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(384)
    k_col_matvec_w(const C2<T>* __restrict__ spec, C2<T>* __restrict__ out0,
                   C2<T>* __restrict__ out1, C2<T>* __restrict__ out2, int N, int M, int Q,
                   double inv_nm, const C2<T>* __restrict__ twN,
                   const DevScalars* __restrict__ sc, const int* __restrict__ skip,
                   const C2<T>* __restrict__ symx, const C2<T>* __restrict__ symy) {
  // threads: 3 groups (outputs Q0, Q1, Q2) x Q columns x N/32 threads per transform;
  // buffers [group][column][N + N/32]; group 0's buffer first holds the forward transform
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* sm = reinterpret_cast<C2<T>*>(smem_raw);
  const int Lc = M / 2, TPT = N / 32, NP = N + N / 32, G = Q * TPT;
  const int grp = threadIdx.x / G, rem = threadIdx.x - grp * G;
  const int q = rem / TPT, t = rem - q * TPT;
  const int col0 = blockIdx.x * Q, col = col0 + q;
  const bool active = col < Lc;
  const int stride = Q * NP;
  C2<T>* b0 = sm + q * NP;
  C2<T>* buf = b0 + grp * stride;
  const int lq = __ffs(Q) - 1;
  for (int idx = threadIdx.x; idx < Q * N; idx += blockDim.x) {
    const int n = idx >> lq, qq = idx & (Q - 1);
    if (col0 + qq < Lc) sm[qq * NP + pad32(n)] = spec[(size_t)n * Lc + col0 + qq];
  }
  __syncthreads();
  fft_warp<T, -1>(b0, N, t, active && grp == 0, twN);
  __syncthreads();
  T ab[5];
#pragma unroll
  for (int a = 0; a < 5; ++a) ab[a] = (T)sc->abar[a];
  const T inv = (T)inv_nm;
  const T d11n = symx[M / 2].y;
  // every group forms S = rho-bar sigma-hat / (N M) and its own symbol; groups 1 and 2
  // write at once, group 0 (which overwrites the spectrum) after the barrier.  Column 0 of
  // Q0 carries its Nyquist channel times d11(M/2), so that the two channels sharing the
  // complex column have comparable magnitudes through the inverse transform.
  C2<T> s0[32];
  if (active) {
#pragma unroll
    for (int e = 0; e < 32; ++e) {
      const int k = t + e * TPT;
      const C2<T> sy = symy[k];
      const C2<T> z = b0[pad32(k)];
      C2<T> v;
      if (col == 0) {
        const C2<T> pz = b0[pad32((N - k) & (N - 1))];
        C2<T> A = mk2<T>((T)0.5 * (z.x + pz.x), (T)0.5 * (z.y - pz.y));
        C2<T> B = mk2<T>((T)0.5 * (z.y + pz.y), (T)-0.5 * (z.x - pz.x));
        A = cscale<T>(cmul<T>(rho_bar<T>(ab, symx[0], symy[k]), A), inv);
        B = cscale<T>(cmul<T>(rho_bar<T>(ab, symx[M / 2], symy[k]), B), inv);
        if (grp == 0) B = cscale<T>(B, d11n);
        v = mk2<T>(A.x - B.y, A.y + B.x);
      } else {
        v = cscale<T>(cmul<T>(rho_bar<T>(ab, symx[col], symy[k]), z), inv);
      }
      if (grp == 1) v = mk2<T>(-sy.x * v.y, sy.x * v.x);
      else if (grp == 2) v = cscale<T>(v, sy.y);
      if (grp == 0) s0[e] = v;
      else buf[pad32(k)] = v;
    }
  }
  __syncthreads();
  if (active && grp == 0) {
#pragma unroll
    for (int e = 0; e < 32; ++e) buf[pad32(t + e * TPT)] = s0[e];
  }
  __syncthreads();
  fft_warp<T, +1>(buf, N, t, active, twN);
  __syncthreads();
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    C2<T>* dst = g == 0 ? out0 : (g == 1 ? out1 : out2);
    for (int idx = threadIdx.x; idx < Q * N; idx += blockDim.x) {
      const int n = idx >> lq, qq = idx & (Q - 1);
      if (col0 + qq < Lc) dst[(size_t)n * Lc + col0 + qq] = sm[g * stride + qq * NP + pad32(n)];
    }
  }
}

// c2r pre-processing on a padded row buffer (threads of one transform)
template <typename T>
__device__ __forceinline__ void c2r_pre_w(C2<T>* buf, int L, int t, int TPT, bool active,
                                          const C2<T>* __restrict__ twM) {
  if (active) {
    for (int k = t; k <= L / 2; k += TPT) {
      if (k == 0) {
        const C2<T> x = buf[0];
        buf[0] = mk2<T>(x.x + x.y, x.x - x.y);
      } else {
        const C2<T> xk = buf[pad32(k)], xm = buf[pad32(L - k)];
        const C2<T> Ev = mk2<T>(xk.x + xm.x, xk.y - xm.y);
        const C2<T> dv = mk2<T>(xk.x - xm.x, xk.y + xm.y);
        const C2<T> Ov = cmul<T>(dv, cconj<T>(twM[k]));
        buf[pad32(k)] = mk2<T>(Ev.x - Ov.y, Ev.y + Ov.x);
        if (2 * k != L) buf[pad32(L - k)] = mk2<T>(Ev.x + Ov.y, -Ev.y + Ov.x);
      }
    }
  }
  wsync(TPT);
}

template <typename T>
__global__ void __launch_bounds__(320)
    k_row_combine_w(const C2<T>* __restrict__ q0, const C2<T>* __restrict__ q1,
                    const C2<T>* __restrict__ q2, const T* __restrict__ coef,
                    T* __restrict__ out, int N, int M, int RB, const C2<T>* __restrict__ twL,
                    const C2<T>* __restrict__ twM, const int* __restrict__ skip,
                    const C2<T>* __restrict__ symx) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* sm = reinterpret_cast<C2<T>*>(smem_raw);
  const int L = M / 2, TPT = L / 32, LP = L + L / 32;
  // transform index: (term, row) = (g / RB, g % RB); buffers [term][row][LP]
  const int g = threadIdx.x / TPT, t = threadIdx.x - g * TPT;
  const int term = g / RB, q = g - term * RB;
  const int row0 = blockIdx.x * RB, row = row0 + q;
  const bool active = row < N;
  const int stride = RB * LP;
  C2<T>* buf = sm + term * stride + q * LP;
  const int la = __ffs(L) - 1;
  for (int idx = threadIdx.x; idx < RB * L; idx += blockDim.x) {
    const int qq = idx >> la, k = idx & (L - 1);
    if (row0 + qq < N) {
      const size_t o = (size_t)(row0 + qq) * L + k;
      const C2<T> x0 = q0[o], x1 = q1[o], x2 = q2[o];
      C2<T>* b = sm + qq * LP + pad32(k);
      b[0] = row_symbol_apply<T>(x0, k, 2, symx);
      b[stride] = row_symbol_apply<T>(x0, k, 1, symx);
      b[2 * stride] = row_symbol_apply<T>(x1, k, 1, symx);
      b[3 * stride] = x1;
      b[4 * stride] = x2;
    }
  }
  __syncthreads();
  c2r_pre_w<T>(buf, L, t, TPT, active, twM);
  fft_warp<T, +1>(buf, L, t, active, twL);
  __syncthreads();
  const size_t P = (size_t)N * M;
  for (int idx = threadIdx.x; idx < RB * L; idx += blockDim.x) {
    const int qq = idx >> la, n = idx & (L - 1);
    const int r = row0 + qq;
    if (r < N) {
      const size_t o = (size_t)r * M;
      const C2<T>* b = sm + qq * LP + pad32(n);
      const C2<T> y0 = b[0], y1 = b[stride], y2 = b[2 * stride], y3 = b[3 * stride],
                  y4 = b[4 * stride];
      const C2<T> a11 = reinterpret_cast<const C2<T>*>(coef + o)[n];
      const C2<T> a12 = reinterpret_cast<const C2<T>*>(coef + P + o)[n];
      const C2<T> a22 = reinterpret_cast<const C2<T>*>(coef + 2 * P + o)[n];
      const C2<T> b1 = reinterpret_cast<const C2<T>*>(coef + 3 * P + o)[n];
      const C2<T> b2 = reinterpret_cast<const C2<T>*>(coef + 4 * P + o)[n];
      C2<T> acc;
      acc.x = a11.x * y0.x + b1.x * y1.x + (T)2 * a12.x * y2.x + b2.x * y3.x + a22.x * y4.x;
      acc.y = a11.y * y0.y + b1.y * y1.y + (T)2 * a12.y * y2.y + b2.y * y3.y + a22.y * y4.y;
      reinterpret_cast<C2<T>*>(out + o)[n] = acc;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------------------
inline int fft_E(int L) { return (L % 3 == 0) ? 12 : 8; }

// A kernel's launch limits, queried once per kernel and device: the largest block (its
// launch bounds and registers) and its static shared memory.
struct KernelLimits {
  int threads = 0;
  size_t static_smem = 0;
  size_t dyn_set = 0;  // the dynamic shared-memory limit raised so far (0: the default)
};
inline KernelLimits* kernel_limits(const void* fn, int dev) {
  struct Rec {
    const void* fn;
    int dev;
    KernelLimits lim;
  };
  static std::deque<Rec> recs;  // (stable addresses as it grows)
  for (auto& r : recs)
    if (r.fn == fn && r.dev == dev) return &r.lim;
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, fn) != cudaSuccess) return nullptr;
  recs.push_back({fn, dev, KernelLimits{a.maxThreadsPerBlock, a.sharedSizeBytes, 0}});
  return &recs.back().lim;
}

// Check a launch configuration on the host and raise the kernel's shared-memory limit: a
// block larger than the kernel allows, or more shared memory (static + dynamic) than a block
// can have, is returned as an error here, never launched (a launch the runtime rejects inside
// a stream capture invalidates the capture).  The dynamic limit is raised whenever static and
// dynamic shared memory together pass the default 48 KB.  The limits and the attribute belong
// to the kernel (and device): the records are keyed by the kernel's address.
inline cudaError_t prepare_launch_fn(const void* fn, long threads, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  KernelLimits* lim = kernel_limits(fn, dev);
  if (!lim) return cudaErrorInvalidDeviceFunction;
  if (threads < 1 || threads > lim->threads) return cudaErrorInvalidConfiguration;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (lim->static_smem + bytes > (size_t)optin) return cudaErrorInvalidConfiguration;
  if (lim->static_smem + bytes <= 48 * 1024 || lim->dyn_set >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  lim->dyn_set = bytes;
  return cudaSuccess;
}
template <typename K>
inline cudaError_t prepare_launch(K kernel, long threads, size_t bytes) {
  return prepare_launch_fn(reinterpret_cast<const void*>(kernel), threads, bytes);
}

template <typename T, int E>
cudaError_t row_r2c_E(const T* x, size_t xs, const int* jptr, const double* scale, C2<T>* spec,
                      int N, int M, const SpecTables& tb, const int* skip, cudaStream_t st,
                      Bat bat = Bat(), const DevScalars* msc = nullptr) {
  const int L = M / 2, TPT = L / E;
  int RB = MaxThreads<T>::value / TPT;
  if (RB < 1) RB = 1;
  while (RB > 1 && RB * TPT > 128 && (N + RB - 1) / RB < 4 * 152) RB /= 2;
  if (RB > N) RB = N;
  const size_t sm = (size_t)RB * FB(L) * sizeof(C2<T>);
  cudaError_t e = prepare_launch(k_row_r2c<T, E>, RB * TPT, sm);
  if (e != cudaSuccess) return e;
  k_row_r2c<T, E><<<bgrid(dim3((N + RB - 1) / RB), bat), RB * TPT, sm, st>>>(
      x, xs, jptr, scale, spec, N, M, (const C2<T>*)tb.twL, (const C2<T>*)tb.twM, skip, bat,
      msc);
  return cudaGetLastError();
}

template <typename T, int E, int MODE>
cudaError_t col_E(const C2<T>* spec, C2<T>* o0, C2<T>* o1, C2<T>* o2, int N, int M,
                  const SpecTables& tb, const DevScalars* sc, const int* skip,
                  cudaStream_t st, Bat bat = Bat()) {
  const int Lc = M / 2, TPT = N / E;
  const size_t colb = (size_t)col_nbuf<T, E, MODE>() * FB(N) * sizeof(C2<T>);
  int Q = MaxThreads<T>::value / TPT;
  if (Q < 1) Q = 1;
  while (Q > 1 && (size_t)Q * colb > 160 * 1024) Q /= 2;
  while (Q > 2 && (Lc + Q - 1) / Q < 2 * 152) Q /= 2;
  if (sizeof(T) == 4 && MODE == COL_MATVEC && tb.col_q > 0) {
    // tuned: more columns per block make the strided column accesses longer runs
    Q = tb.col_q;
    while (Q > 1 && (Q * TPT > MaxThreads<T>::value || (size_t)Q * colb > 160 * 1024)) Q /= 2;
  }
  if (Q > Lc) Q = Lc;
  size_t sm = (size_t)Q * colb;
  if (col_nbuf<T, E, MODE>() == 3) sm += (size_t)N * sizeof(C2<T>);  // stage twiddle table
  cudaError_t e = prepare_launch(k_col<T, E, MODE>, Q * TPT, sm);
  if (e != cudaSuccess) return e;
  k_col<T, E, MODE><<<bgrid(dim3((Lc + Q - 1) / Q), bat), Q * TPT, sm, st>>>(
      spec, o0, o1, o2, N, M, Q, 1.0 / ((double)N * (double)M), (const C2<T>*)tb.twN,
      (const C2<T>*)tb.twM, sc, skip, (const C2<T>*)tb.symx, (const C2<T>*)tb.symy, bat);
  return cudaGetLastError();
}

template <typename T, int E, int MODE>
cudaError_t row_c2r_E(const C2<T>* q0, const C2<T>* q1, const C2<T>* q2, const T* coef, T* out,
                      const double* u_in, double* u_out, double step, double out_scale, int N,
                      int M, const SpecTables& tb, const int* skip, cudaStream_t st,
                      const DevScalars* sc, Bat bat = Bat()) {
  const int L = M / 2, TPT = L / E;
  const size_t rowb = (size_t)row_nbuf<T, E, MODE>() * FB(L) * sizeof(C2<T>);
  int RB = MaxThreads<T>::value / TPT;
  if (RB < 1) RB = 1;
  while (RB > 1 && RB * rowb > 160 * 1024) RB /= 2;
  while (RB > 1 && RB * TPT > 128 && (N + RB - 1) / RB < 4 * 152) RB /= 2;
  if (RB > N) RB = N;
  const size_t sm = (size_t)RB * rowb;
  cudaError_t e = prepare_launch(k_row_c2r<T, E, MODE>, RB * TPT, sm);
  if (e != cudaSuccess) return e;
  k_row_c2r<T, E, MODE><<<bgrid(dim3((N + RB - 1) / RB), bat), RB * TPT, sm, st>>>(
      q0, q1, q2, coef, out, u_in, u_out, step, out_scale, N, M, (const C2<T>*)tb.twL,
      (const C2<T>*)tb.twM, skip, sc, (const C2<T>*)tb.symx, bat);
  return cudaGetLastError();
}

template <typename T>
cudaError_t row_r2c_w_launch(const T* x, size_t xs, const int* jptr, const double* scale,
                             C2<T>* spec, int N, int M, const SpecTables& tb, const int* skip,
                             cudaStream_t st) {
  const int L = M / 2, TPT = L / 32;
  int RB = 64 / TPT;  // two warps per block at most
  if (RB < 1) RB = 1;
  if (RB > N) RB = N;
  const size_t sm = (size_t)RB * (L + L / 32) * sizeof(C2<T>);
  cudaError_t e = prepare_launch(k_row_r2c_w<T>, RB * TPT, sm);
  if (e != cudaSuccess) return e;
  k_row_r2c_w<T><<<(N + RB - 1) / RB, RB * TPT, sm, st>>>(
      x, xs, jptr, scale, spec, N, M, RB, (const C2<T>*)tb.twL, (const C2<T>*)tb.twM, skip);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_row_r2c(const T* x, size_t xs, const int* jptr, const double* scale,
                           C2<T>* spec, int N, int M, const SpecTables& tb, const int* skip,
                           cudaStream_t st, Bat bat, const DevScalars* msc) {
  if (bat.on) {  // batched: the generic kernels
    if (fft_E(M / 2) == 12)
      return row_r2c_E<T, 12>(x, xs, jptr, scale, spec, N, M, tb, skip, st, bat, msc);
    return row_r2c_E<T, 8>(x, xs, jptr, scale, spec, N, M, tb, skip, st, bat, msc);
  }
  if constexpr (sizeof(T) == 4) {
    if (tb.var_r2c == VAR_PAIR && !msc && comb_pair_supported(N, M))
      return launch_row_r2c_pair(reinterpret_cast<const float*>(x), xs, jptr, scale,
                                 reinterpret_cast<float2*>(spec), N, M, tb, skip, st);
  }
  if (sizeof(T) == 4 && tb.var_r2c == VAR_WARP && warp_fft_ok(M / 2))
    return row_r2c_w_launch<T>(x, xs, jptr, scale, spec, N, M, tb, skip, st);
  if (sizeof(T) == 4 && (tb.var_r2c == VAR_E4 || tb.var_r2c == VAR_PAIR) && fft_E(M / 2) == 8 &&
      M / 2 >= 4)
    return row_r2c_E<T, 4>(x, xs, jptr, scale, spec, N, M, tb, skip, st);
  if (fft_E(M / 2) == 12) return row_r2c_E<T, 12>(x, xs, jptr, scale, spec, N, M, tb, skip, st);
  return row_r2c_E<T, 8>(x, xs, jptr, scale, spec, N, M, tb, skip, st);
}

template <typename T, int E>
cudaError_t col_matvec_par_E(const C2<T>* spec, C2<T>* o0, C2<T>* o1, C2<T>* o2, int N, int M,
                             const SpecTables& tb, const DevScalars* sc, const int* skip,
                             cudaStream_t st) {
  const int Lc = M / 2, TPT = N / E;
  int Q = OTGB_PAR_THREADS / (3 * TPT);
  if (Q < 1) Q = 1;
  if (Q > 4) Q = 4;
  if (Q > Lc) Q = Lc;
  const size_t sm = (size_t)3 * Q * FB(N) * sizeof(C2<T>);
  cudaError_t e = prepare_launch(k_col_matvec_par<T, E>, 3 * Q * TPT, sm);
  if (e != cudaSuccess) return e;
  k_col_matvec_par<T, E><<<(Lc + Q - 1) / Q, 3 * Q * TPT, sm, st>>>(
      spec, o0, o1, o2, N, M, Q, 1.0 / ((double)N * (double)M), (const C2<T>*)tb.twN, sc,
      skip, (const C2<T>*)tb.symx, (const C2<T>*)tb.symy);
  return cudaGetLastError();
}

template <typename T>
cudaError_t col_matvec_w_launch(const C2<T>* spec, C2<T>* o0, C2<T>* o1, C2<T>* o2, int N,
                                int M, const SpecTables& tb, const DevScalars* sc,
                                const int* skip, cudaStream_t st) {
  const int Lc = M / 2, TPT = N / 32;
  int Q = 1;
  while (Q * 2 * 3 * TPT <= 384 && Q < 2) Q *= 2;
  if (Q > Lc) Q = Lc;
  const size_t sm = (size_t)3 * Q * (N + N / 32) * sizeof(C2<T>);
  cudaError_t e = prepare_launch(k_col_matvec_w<T>, 3 * Q * TPT, sm);
  if (e != cudaSuccess) return e;
  k_col_matvec_w<T><<<(Lc + Q - 1) / Q, 3 * Q * TPT, sm, st>>>(
      spec, o0, o1, o2, N, M, Q, 1.0 / ((double)N * (double)M), (const C2<T>*)tb.twN, sc,
      skip, (const C2<T>*)tb.symx, (const C2<T>*)tb.symy);
  return cudaGetLastError();
}

template <typename T, int E>
cudaError_t col_dispatch(int mode, const C2<T>* spec, C2<T>* o0, C2<T>* o1, C2<T>* o2, int N,
                         int M, const SpecTables& tb, const DevScalars* sc, const int* skip,
                         cudaStream_t st) {
  if (sizeof(T) == 4 && mode == COL_MATVEC && tb.var_col == VAR_WARP && warp_fft_ok(N) &&
      3 * (N / 32) <= 384)
    return col_matvec_w_launch<T>(spec, o0, o1, o2, N, M, tb, sc, skip, st);
  if (sizeof(T) == 4 && mode == COL_MATVEC && tb.var_col != VAR_GENERIC &&
      3 * (N / E) <= OTGB_PAR_THREADS)
    return col_matvec_par_E<T, E>(spec, o0, o1, o2, N, M, tb, sc, skip, st);
  switch (mode) {
    case COL_FWD: return col_E<T, E, COL_FWD>(spec, o0, o1, o2, N, M, tb, sc, skip, st);
    case COL_INV: return col_E<T, E, COL_INV>(spec, o0, o1, o2, N, M, tb, sc, skip, st);
    case COL_MATVEC: return col_E<T, E, COL_MATVEC>(spec, o0, o1, o2, N, M, tb, sc, skip, st);
    case COL_LBARINV: return col_E<T, E, COL_LBARINV>(spec, o0, o1, o2, N, M, tb, sc, skip, st);
    case COL_POISSON:
      return col_E<T, E, COL_POISSON>(spec, o0, o1, o2, N, M, tb, sc, skip, st);
    case COL_POISSON_LP:
      return col_E<T, E, COL_POISSON_LP>(spec, o0, o1, o2, N, M, tb, sc, skip, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_col(int mode, const C2<T>* spec, C2<T>* o0, C2<T>* o1, C2<T>* o2, int N,
                       int M, const SpecTables& tb, const DevScalars* sc, const int* skip,
                       cudaStream_t st, Bat bat) {
  if (bat.on) {  // batched: the generic kernels (the matvec mode only)
    if (mode != COL_MATVEC) return cudaErrorInvalidValue;
    if (fft_E(N) == 12)
      return col_E<T, 12, COL_MATVEC>(spec, o0, o1, o2, N, M, tb, sc, skip, st, bat);
    return col_E<T, 8, COL_MATVEC>(spec, o0, o1, o2, N, M, tb, sc, skip, st, bat);
  }
  if constexpr (sizeof(T) == 4) {
    if (mode == COL_MATVEC && tb.var_col == VAR_PAIR && col_pair_supported(N, M))
      return launch_col_pair(reinterpret_cast<const float2*>(spec),
                             reinterpret_cast<float2*>(o0), reinterpret_cast<float2*>(o1),
                             reinterpret_cast<float2*>(o2), N, M, tb, sc, skip, st);
  }
  if (sizeof(T) == 4 && mode == COL_MATVEC &&
      (tb.var_col == VAR_E4 || tb.var_col == VAR_PAIR) && fft_E(N) == 8 && N >= 4)
    return col_E<T, 4, COL_MATVEC>(spec, o0, o1, o2, N, M, tb, sc, skip, st);
  if (fft_E(N) == 12) return col_dispatch<T, 12>(mode, spec, o0, o1, o2, N, M, tb, sc, skip, st);
  return col_dispatch<T, 8>(mode, spec, o0, o1, o2, N, M, tb, sc, skip, st);
}

template <typename T, int E>
cudaError_t row_combine_par_E(const C2<T>* q0, const C2<T>* q1, const C2<T>* q2, const T* coef,
                              T* out, int N, int M, const SpecTables& tb, const int* skip,
                              cudaStream_t st) {
  const int L = M / 2, TPT = L / E;
  int RB = 1;
  while (RB * 2 * 5 * TPT <= OTGB_PAR_THREADS && RB < 8) RB *= 2;
  if (RB > N) RB = N;
  const size_t sm = (size_t)5 * RB * FB(L) * sizeof(C2<T>);
  cudaError_t e = prepare_launch(k_row_combine_par<T, E>, 5 * RB * TPT, sm);
  if (e != cudaSuccess) return e;
  k_row_combine_par<T, E><<<(N + RB - 1) / RB, 5 * RB * TPT, sm, st>>>(
      q0, q1, q2, coef, out, N, M, RB, (const C2<T>*)tb.twL, (const C2<T>*)tb.twM, skip,
      (const C2<T>*)tb.symx);
  return cudaGetLastError();
}

template <typename T>
cudaError_t row_combine_w_launch(const C2<T>* q0, const C2<T>* q1, const C2<T>* q2,
                                 const T* coef, T* out, int N, int M, const SpecTables& tb,
                                 const int* skip, cudaStream_t st) {
  const int L = M / 2, TPT = L / 32;
  int RB = 1;
  while (RB * 2 * 5 * TPT <= 320 && RB < 8) RB *= 2;
  if (RB > N) RB = N;
  const size_t sm = (size_t)5 * RB * (L + L / 32) * sizeof(C2<T>);
  cudaError_t e = prepare_launch(k_row_combine_w<T>, 5 * RB * TPT, sm);
  if (e != cudaSuccess) return e;
  k_row_combine_w<T><<<(N + RB - 1) / RB, 5 * RB * TPT, sm, st>>>(
      q0, q1, q2, coef, out, N, M, RB, (const C2<T>*)tb.twL, (const C2<T>*)tb.twM, skip,
      (const C2<T>*)tb.symx);
  return cudaGetLastError();
}

template <typename T, int E>
cudaError_t row_c2r_dispatch(int mode, const C2<T>* q0, const C2<T>* q1, const C2<T>* q2,
                             const T* coef, T* out, const double* u_in, double* u_out,
                             double step, double os, int N, int M, const SpecTables& tb,
                             const int* skip, cudaStream_t st, const DevScalars* sc) {
  if (sizeof(T) == 4 && mode == ROWINV_COMBINE && tb.var_comb != VAR_GENERIC &&
      tb.var_comb != VAR_PAR && warp_fft_ok(M / 2) && 5 * (M / 64) <= 320)
    return row_combine_w_launch<T>(q0, q1, q2, coef, out, N, M, tb, skip, st);
  if (sizeof(T) == 4 && mode == ROWINV_COMBINE && tb.var_comb != VAR_GENERIC &&
      5 * ((M / 2) / E) <= OTGB_PAR_THREADS)
    return row_combine_par_E<T, E>(q0, q1, q2, coef, out, N, M, tb, skip, st);
  switch (mode) {
    case ROWINV_PLAIN:
      return row_c2r_E<T, E, ROWINV_PLAIN>(q0, q1, q2, coef, out, u_in, u_out, step, os, N, M,
                                           tb, skip, st, sc);
    case ROWINV_COMBINE:
      return row_c2r_E<T, E, ROWINV_COMBINE>(q0, q1, q2, coef, out, u_in, u_out, step, os, N,
                                             M, tb, skip, st, sc);
    case ROWINV_UPDATE:
      return row_c2r_E<T, E, ROWINV_UPDATE>(q0, q1, q2, coef, out, u_in, u_out, step, os, N, M,
                                            tb, skip, st, sc);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_row_c2r(int mode, const C2<T>* q0, const C2<T>* q1, const C2<T>* q2,
                           const T* coef, T* out, const double* u_in, double* u_out,
                           double step, double os, int N, int M, const SpecTables& tb,
                           const int* skip, cudaStream_t st, const DevScalars* sc, Bat bat) {
  if (bat.on) {  // batched: the generic kernels (the combine mode only)
    if (mode != ROWINV_COMBINE) return cudaErrorInvalidValue;
    if (fft_E(M / 2) == 12)
      return row_c2r_E<T, 12, ROWINV_COMBINE>(q0, q1, q2, coef, out, u_in, u_out, step, os, N,
                                              M, tb, skip, st, sc, bat);
    return row_c2r_E<T, 8, ROWINV_COMBINE>(q0, q1, q2, coef, out, u_in, u_out, step, os, N, M,
                                           tb, skip, st, sc, bat);
  }
  if constexpr (sizeof(T) == 4) {
    if (mode == ROWINV_COMBINE && tb.var_comb == VAR_PAIR && comb_pair_supported(N, M))
      return launch_comb_pair(reinterpret_cast<const float2*>(q0),
                              reinterpret_cast<const float2*>(q1),
                              reinterpret_cast<const float2*>(q2),
                              reinterpret_cast<const float*>(coef), reinterpret_cast<float*>(out),
                              N, M, tb, skip, st);
  }
  if (sizeof(T) == 4 && mode == ROWINV_COMBINE &&
      (tb.var_comb == VAR_E4 || tb.var_comb == VAR_PAIR) && fft_E(M / 2) == 8 && M / 2 >= 4)
    return row_c2r_E<T, 4, ROWINV_COMBINE>(q0, q1, q2, coef, out, u_in, u_out, step, os, N, M,
                                           tb, skip, st, sc);
  if (fft_E(M / 2) == 12)
    return row_c2r_dispatch<T, 12>(mode, q0, q1, q2, coef, out, u_in, u_out, step, os, N, M,
                                   tb, skip, st, sc);
  return row_c2r_dispatch<T, 8>(mode, q0, q1, q2, coef, out, u_in, u_out, step, os, N, M, tb,
                                skip, st, sc);
}

template <int E>
cudaError_t col_lbarinv_mixed_E(const float2* spec, double2* out, int N, int M,
                                const SpecTables& tb32, const SpecTables& tb64,
                                const DevScalars* sc, cudaStream_t st) {
  const int Lc = M / 2, TPT = N / E;
  int Q = 256 / TPT;
  if (Q < 1) Q = 1;
  while (Q > 1 && (Lc + Q - 1) / Q < 2 * 152) Q /= 2;
  if (Q > Lc) Q = Lc;
  const size_t sm = (size_t)Q * FB(N) * sizeof(double2);
  cudaError_t e = prepare_launch(k_col_lbarinv_mixed<E>, Q * TPT, sm);
  if (e != cudaSuccess) return e;
  k_col_lbarinv_mixed<E><<<(Lc + Q - 1) / Q, Q * TPT, sm, st>>>(
      spec, out, N, M, Q, 1.0 / ((double)N * (double)M), (const float2*)tb32.twN,
      (const double2*)tb64.twN, sc, (const float2*)tb32.symx, (const float2*)tb32.symy);
  return cudaGetLastError();
}

template <int E, int MODE>
cudaError_t col_lbarinv_dd_E(const float2* spec, ddc* out, int N, int M,
                             const SpecTables& tb32, const SpecTables& tbdd,
                             const DevScalars* sc, cudaStream_t st, Bat bat = Bat()) {
  const int Lc = M / 2, TPT = N / E;
  int Q = 256 / TPT;
  if (Q < 1) Q = 1;
  while (Q > 1 && (size_t)Q * FB(N) * sizeof(ddc) > 160 * 1024) Q /= 2;
  while (Q > 1 && (Lc + Q - 1) / Q < 2 * 152) Q /= 2;
  if (Q > Lc) Q = Lc;
  const size_t sm = (size_t)Q * FB(N) * sizeof(ddc);
  cudaError_t e = prepare_launch(k_col_lbarinv_dd<E, MODE>, Q * TPT, sm);
  if (e != cudaSuccess) return e;
  k_col_lbarinv_dd<E, MODE><<<bgrid(dim3((Lc + Q - 1) / Q), bat), Q * TPT, sm, st>>>(
      spec, out, N, M, Q, 1.0 / ((double)N * (double)M), (const float2*)tb32.twN,
      (const float2*)tb32.twM, (const ddc*)tbdd.twN, sc, (const float2*)tb32.symx,
      (const float2*)tb32.symy, bat);
  return cudaGetLastError();
}

template <int E>
cudaError_t row_c2r_update_dd_E(const ddc* q, const double* u_in, double* u_out, double step,
                                int N, int M, const SpecTables& tbdd, const DevScalars* sc,
                                cudaStream_t st, Bat bat = Bat()) {
  const int L = M / 2, TPT = L / E;
  int RB = 256 / TPT;
  if (RB < 1) RB = 1;
  while (RB > 1 && (size_t)RB * FB(L) * sizeof(ddc) > 160 * 1024) RB /= 2;
  while (RB > 1 && (N + RB - 1) / RB < 2 * 152) RB /= 2;
  const size_t sm = (size_t)RB * FB(L) * sizeof(ddc);
  cudaError_t e = prepare_launch(k_row_c2r_update_dd<E>, RB * TPT, sm);
  if (e != cudaSuccess) return e;
  k_row_c2r_update_dd<E><<<bgrid(dim3((N + RB - 1) / RB), bat), RB * TPT, sm, st>>>(
      q, u_in, u_out, step, N, M, (const ddc*)tbdd.twL, (const ddc*)tbdd.twM, sc, bat);
  return cudaGetLastError();
}

#define OTGB_INSTANTIATE_SPECTRAL(T)                                                         \
  template cudaError_t launch_row_r2c<T>(const T*, size_t, const int*, const double*,        \
                                         C2<T>*, int, int, const SpecTables&, const int*,    \
                                         cudaStream_t, Bat, const DevScalars*);              \
  template cudaError_t launch_col<T>(int, const C2<T>*, C2<T>*, C2<T>*, C2<T>*, int, int,    \
                                     const SpecTables&, const DevScalars*, const int*,       \
                                     cudaStream_t, Bat);                                     \
  template cudaError_t launch_row_c2r<T>(int, const C2<T>*, const C2<T>*, const C2<T>*,      \
                                         const T*, T*, const double*, double*, double,       \
                                         double, int, int, const SpecTables&, const int*,    \
                                         cudaStream_t, const DevScalars*, Bat);

}  // namespace otgb
