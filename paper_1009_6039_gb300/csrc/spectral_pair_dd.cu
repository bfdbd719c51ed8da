// theta = Lbar^{-1} sigma (Sec. 4.2) and the warm start's Poisson solves on column and row
// pairs, with the double-float inverse transforms in packed FP32 arithmetic.
//
// These compute what k_col_lbarinv_dd and k_row_c2r_update_dd compute, but hold two
// columns (rows) side by side: a double-float value is the pair (hi, lo) of FP32 numbers,
// and the two columns' values share register pairs, (hi_a, hi_b) and (lo_a, lo_b).  Every
// step of the error-free transformations (TwoSum, FastTwoSum, the FMA TwoProduct of dd.cuh)
// then runs once for both columns as a packed instruction (add/sub/mul/fma.rn.f32x2, per
// lane the scalar round-to-nearest operation), in the scalar kernels' order of operations,
// so a lane computes bit for bit the scalar double-float result from the same inputs.  The
// column pass's forward transform and symbol step are FP32 (the forward on packed pairs as in
// k_col_pair).  Double-float elements live in two shared-memory planes, the high words
// (re, im) and the low words, 16 bytes per element each, under the swizzle of pair.cuh.
#include "dd2.cuh"
#include "pair.cuh"

namespace otgb {
namespace {

using namespace pair;

// two double-float complex numbers
struct DC {
  D2 re, im;
};
__device__ __forceinline__ DC dc_add(DC a, DC b) {
  return DC{d2_add(a.re, b.re), d2_add(a.im, b.im)};
}
__device__ __forceinline__ DC dc_sub(DC a, DC b) {
  return DC{d2_sub(a.re, b.re), d2_sub(a.im, b.im)};
}
// a * w, w = (wx, wy) broadcast to both lanes (the scalar complex product's order)
__device__ __forceinline__ DC dc_mul(DC a, D2 wx, D2 wy) {
  return DC{d2_sub(d2_mul(a.re, wx), d2_mul(a.im, wy)),
            d2_add(d2_mul(a.re, wy), d2_mul(a.im, wx))};
}
// SIGN i a
template <int SIGN>
__device__ __forceinline__ DC dc_mul_si(DC a) {
  return SIGN > 0 ? DC{d2_neg(a.im), a.re} : DC{a.im, d2_neg(a.re)};
}

template <int R, int SIGN> struct BflyDC;
template <int SIGN> struct BflyDC<2, SIGN> {
  __device__ __forceinline__ static void run(DC* v) {
    const DC a = v[0], b = v[1];
    v[0] = dc_add(a, b);
    v[1] = dc_sub(a, b);
  }
};
template <int SIGN> struct BflyDC<4, SIGN> {
  __device__ __forceinline__ static void run(DC* v) {
    const DC t0 = dc_add(v[0], v[2]), t1 = dc_sub(v[0], v[2]);
    const DC t2 = dc_add(v[1], v[3]), t3 = dc_mul_si<SIGN>(dc_sub(v[1], v[3]));
    v[0] = dc_add(t0, t2);
    v[2] = dc_sub(t0, t2);
    v[1] = dc_add(t1, t3);
    v[3] = dc_sub(t1, t3);
  }
};

// a double-float complex pair buffer: high words (re, im) and low words, L elements each
struct DBuf {
  ulonglong2* h;
  ulonglong2* l;
};
__device__ __forceinline__ DC dld(DBuf b, int i) {
  const ulonglong2 x = b.h[i], y = b.l[i];
  return DC{D2{x.x, y.x}, D2{x.y, y.y}};
}
__device__ __forceinline__ void dst(DBuf b, int i, DC v) {
  b.h[i] = make_ulonglong2(v.re.h, v.im.h);
  b.l[i] = make_ulonglong2(v.re.l, v.im.l);
}
__device__ __forceinline__ DC dc_from(ddc a, ddc b) {
  return DC{D2{pk(a.x.hi, b.x.hi), pk(a.x.lo, b.x.lo)},
            D2{pk(a.y.hi, b.y.hi), pk(a.y.lo, b.y.lo)}};
}
__device__ __forceinline__ void dc_to(DC v, ddc& a, ddc& b) {
  upk(v.re.h, a.x.hi, b.x.hi);
  upk(v.re.l, a.x.lo, b.x.lo);
  upk(v.im.h, a.y.hi, b.y.hi);
  upk(v.im.l, a.y.lo, b.y.lo);
}

// the stage twiddles of the 4-element double-float transforms of length L, broadcast to both
// lanes: high words (x, y) in th, low words in tl
template <int L>
__device__ __forceinline__ void load_twdd(ulonglong2* th, ulonglong2* tl,
                                          const ddc* __restrict__ twb, int t, int nthreads) {
  const ddc* __restrict__ st = twb + (size_t)stage_table_slot<4>() * L;
  for (int i = t; i < L; i += nthreads) {
    const ddc w = st[i];
    th[i] = make_ulonglong2(pk(w.x.hi, w.x.hi), pk(w.y.hi, w.y.hi));
    tl[i] = make_ulonglong2(pk(w.x.lo, w.x.lo), pk(w.y.lo, w.y.lo));
  }
}

// one double-float stage of radix R (span Ns), 4 elements per thread, in -> out (in place:
// the stores wait for every thread's loads)
template <int R, int SIGN, int L, int Ns, bool INPLACE>
__device__ __forceinline__ void dstage(DBuf in, DBuf out, int t,
                                       const ulonglong2* __restrict__ th,
                                       const ulonglong2* __restrict__ tl) {
  constexpr int E = 4, TPT = L / E, LR = L / R;
  constexpr int a = Ns == 1 ? 0 : __builtin_ctz(Ns);
  DC v[E];
#pragma unroll
  for (int b = 0; b < E / R; ++b) {
    const int j = t + b * TPT;
#pragma unroll
    for (int r = 0; r < R; ++r) v[b * R + r] = dld(in, swz(j + r * LR));
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
        const int ti = (Ns - 1) + (r - 1) * Ns + k;
        const ulonglong2 wh = th[ti], wl = tl[ti];
        const D2 wx{wh.x, wl.x};
        D2 wy{wh.y, wl.y};
        if (SIGN > 0) wy = d2_neg(wy);
        v[b * R + r] = dc_mul(v[b * R + r], wx, wy);
      }
    }
    BflyDC<R, SIGN>::run(&v[b * R]);
    const int d = qd * (Ns * R) + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst(out, swz(d + r * Ns), v[b * R + r]);
  }
  __syncthreads();
}

// the inverse transform: in place (INPLACE), or alternating between a and b from a (the
// result ends in a for an even number of stages, in b for an odd one)
template <int SIGN, int L, int Ns, int REM, bool INPLACE, bool FROM_A>
__device__ __forceinline__ void dfft(DBuf a, DBuf b, int t, const ulonglong2* __restrict__ th,
                                     const ulonglong2* __restrict__ tl) {
  if constexpr (REM > 1) {
    constexpr int R = REM % 4 == 0 ? 4 : 2;
    if constexpr (INPLACE)
      dstage<R, SIGN, L, Ns, true>(a, a, t, th, tl);
    else if constexpr (FROM_A)
      dstage<R, SIGN, L, Ns, false>(a, b, t, th, tl);
    else
      dstage<R, SIGN, L, Ns, false>(b, a, t, th, tl);
    dfft<SIGN, L, Ns * R, REM / R, INPLACE, !FROM_A>(a, b, t, th, tl);
  }
}

template <int REM>
__host__ __device__ constexpr int dstage_count() {
  if constexpr (REM > 1)
    return 1 + dstage_count<REM / (REM % 4 == 0 ? 4 : 2)>();
  else
    return 0;
}

// theta's column pass (MODE COL_LBARINV: S = rho-bar(abar_n) sigma-hat / (N M)) or the
// Poisson solves' (COL_POISSON, COL_POISSON_LP: division by the 4th-order FD Laplacian's
// eigenvalues, zero mode -> 0, _LP with the Gaussian low-pass) on column pairs: the FP32
// forward column transform, the scalar symbol step of k_col_lbarinv_dd per column, the
// double-float inverse column transform (out of place), ddc output
template <int N, int MODE>
__global__ void __launch_bounds__(N / 4, N <= 1024 ? 2 : 1)
    k_col_lbarinv_pair(const float2* __restrict__ spec, ddc* __restrict__ out, int M,
                       float inv, const float2* __restrict__ twN32,
                       const float2* __restrict__ twM32, const ddc* __restrict__ twNdd,
                       const DevScalars* __restrict__ sc, const float2* __restrict__ symx,
                       const float2* __restrict__ symy) {
  constexpr int TPT = N / 4;
  constexpr bool FODD = dstage_count<N>() % 2 == 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ulonglong2* tw4 = reinterpret_cast<ulonglong2*>(smem_raw);
  ulonglong2* th = tw4 + N;
  ulonglong2* tl = th + N;
  ulonglong2* base = tl + N;
  // double-float buffers A (h, l) and B (h, l); the FP32 forward ping-pongs inside A
  const DBuf A{base, base + N}, B{base + 2 * N, base + 3 * N};
  PC* const F0 = reinterpret_cast<PC*>(A.h);
  PC* const F1 = reinterpret_cast<PC*>(A.l);
  const int Lc = M / 2;
  const int c0 = 2 * blockIdx.x;
  const int t = threadIdx.x;
  // the column pair's loads first, so that they are in flight with the twiddle tables' loads
  float4 xs[4];
#pragma unroll
  for (int e = 0; e < 4; ++e)
    xs[e] = *reinterpret_cast<const float4*>(spec + (size_t)(t + e * TPT) * Lc + c0);
  load_tw4<N>(tw4, twN32, t, TPT);
  load_twdd<N>(th, tl, twNdd, t, TPT);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    PC v;
    v.re = pk(xs[e].x, xs[e].z);
    v.im = pk(xs[e].y, xs[e].w);
    F0[swz(t + e * TPT)] = v;
  }
  __syncthreads();
  {
    PC* const a[1] = {F0};
    PC* const b[1] = {F1};
    pfft_rec<-1, N, 1, N, 1, true>(a, b, t, tw4);
  }
  const PC* const F = FODD ? F1 : F0;

  float ab[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) ab[q] = MODE == COL_LBARINV ? (float)sc->abar_n[q] : 0.f;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int k = t + e * TPT;
    const PC z2 = F[swz(k)];
    float2 zc[2];
    upk(z2.re, zc[0].x, zc[1].x);
    upk(z2.im, zc[0].y, zc[1].y);
    float2 s[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int col = c0 + h;
      const float2 z = zc[h];
      float2 r;
      if (col == 0) {
        const PC p2 = F[swz((N - k) % N)];
        float2 pz, pother;
        upk(p2.re, pz.x, pother.x);
        upk(p2.im, pz.y, pother.y);
        float2 Av = mk2<float>(0.5f * (z.x + pz.x), 0.5f * (z.y - pz.y));
        float2 Bv = mk2<float>(0.5f * (z.y + pz.y), -0.5f * (z.x - pz.x));
        if (MODE == COL_LBARINV) {
          Av = cmul<float>(rho_bar<float>(ab, symx[0], symy[k]), Av);
          Bv = cmul<float>(rho_bar<float>(ab, symx[M / 2], symy[k]), Bv);
        } else {
          bool nyq2;
          const int k2 = sfreq(k, N, &nyq2);
          const float ly = fd_lap_w(twN32[k], N);
          const float lxn = -16.f / 3.f * (float)M * (float)M;  // k1 = M/2 (cos t = -1)
          Av = cscale<float>(Av, inv_or_zero<float>(ly) * lowpass_f<MODE>(0, k2, M, N));
          Bv = cscale<float>(Bv,
                             inv_or_zero<float>(lxn + ly) * lowpass_f<MODE>(M / 2, k2, M, N));
        }
        r = mk2<float>(Av.x - Bv.y, Av.y + Bv.x);
      } else if (MODE == COL_LBARINV) {
        r = cmul<float>(rho_bar<float>(ab, symx[col], symy[k]), z);
      } else {
        bool nyq2;
        const int k2 = sfreq(k, N, &nyq2);
        r = cscale<float>(z, inv_or_zero<float>(fd_lap_w(twM32[col], M) +
                                                fd_lap_w(twN32[k], N)) *
                                 lowpass_f<MODE>(col, k2, M, N));
      }
      s[h] = mk2<float>(r.x * inv, r.y * inv);
    }
    DC v;
    v.re = D2{pk(s[0].x, s[1].x), 0ull};
    v.im = D2{pk(s[0].y, s[1].y), 0ull};
    dst(B, swz(k), v);
  }
  __syncthreads();
  // inverse in double-float from B (scratch A)
  dfft<+1, N, 1, N, false, true>(B, A, t, th, tl);
  const DBuf res = FODD ? A : B;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int n = t + e * TPT;
    ddc a, b;
    dc_to(dld(res, swz(n)), a, b);
    ddc* o = out + (size_t)n * Lc + c0;
    o[0] = a;
    o[1] = b;
  }
}

// theta's rows (complex-to-real, double-float) on row pairs, then u_out = u_in + step theta
// in FP64 (u_in == nullptr: u_out = step theta; with sc the step and the current / candidate
// buffers come from the device scalars, as in k_row_c2r_update_dd); in-place stages
template <int L>
__global__ void __launch_bounds__(L / 4, L <= 512 ? 4 : 2)
    k_row_update_pair(const ddc* __restrict__ q, const double* __restrict__ u_in,
                      double* __restrict__ u_out, double step, int N,
                      const ddc* __restrict__ twL, const ddc* __restrict__ twM,
                      const DevScalars* __restrict__ sc) {
  if (sc) {
    step = sc->step_s;
    if (sc->upar & 1) {
      double* tmp = const_cast<double*>(u_in);
      u_in = u_out;
      u_out = tmp;
    }
  }
  constexpr int TPT = L / 4;
  constexpr int M = 2 * L;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ulonglong2* th = reinterpret_cast<ulonglong2*>(smem_raw);
  ulonglong2* tl = th + L;
  const DBuf A{tl + L, tl + 2 * L};
  const int r0 = 2 * blockIdx.x;
  const int t = threadIdx.x;
  // the rows' loads first, so that they are in flight with the twiddle table's loads
  const ddc* qa = q + (size_t)r0 * L;
  const ddc* qb = qa + L;
  ddc ra[4], rb[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    ra[e] = qa[t + e * TPT];
    rb[e] = qb[t + e * TPT];
  }
  load_twdd<L>(th, tl, twL, t, TPT);
#pragma unroll
  for (int e = 0; e < 4; ++e) dst(A, swz(t + e * TPT), dc_from(ra[e], rb[e]));
  __syncthreads();
  // complex-to-real pre-processing (as c2r_preprocess on dd): each pair (k, L - k) by one
  // thread
  for (int k = t; k <= L / 2; k += TPT) {
    if (k == 0) {
      const int d = swz(0);
      const DC x = dld(A, d);
      dst(A, d, DC{d2_add(x.re, x.im), d2_sub(x.re, x.im)});
    } else {
      const ddc w = twM[k];
      const D2 wx{pk(w.x.hi, w.x.hi), pk(w.x.lo, w.x.lo)};
      // conj(W_M^k)
      const D2 wy = d2_neg(D2{pk(w.y.hi, w.y.hi), pk(w.y.lo, w.y.lo)});
      const int dk = swz(k), dm = swz(L - k);
      const DC xk = dld(A, dk), xm = dld(A, dm);
      const DC Ev{d2_add(xk.re, xm.re), d2_sub(xk.im, xm.im)};
      const DC dv{d2_sub(xk.re, xm.re), d2_add(xk.im, xm.im)};
      const DC Ov = dc_mul(dv, wx, wy);
      dst(A, dk, DC{d2_sub(Ev.re, Ov.im), d2_add(Ev.im, Ov.re)});
      if (2 * k != L) dst(A, dm, DC{d2_add(Ev.re, Ov.im), d2_add(d2_neg(Ev.im), Ov.re)});
    }
  }
  __syncthreads();
  dfft<+1, L, 1, L, true, true>(A, A, t, th, tl);
  const double2* uia = u_in ? reinterpret_cast<const double2*>(u_in + (size_t)r0 * M) : nullptr;
  const double2* uib = u_in ? uia + L : nullptr;
  double2* uoa = reinterpret_cast<double2*>(u_out + (size_t)r0 * M);
  double2* uob = uoa + L;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int n = t + e * TPT;
    ddc za, zb;
    dc_to(dld(A, swz(n)), za, zb);
    double2 a = uia ? uia[n] : make_double2(0.0, 0.0);
    double2 b = uib ? uib[n] : make_double2(0.0, 0.0);
    a.x += step * dd_to_double(za.x);
    a.y += step * dd_to_double(za.y);
    b.x += step * dd_to_double(zb.x);
    b.y += step * dd_to_double(zb.y);
    uoa[n] = a;
    uob[n] = b;
  }
}

template <int N, int MODE>
cudaError_t col_lbarinv_pair_N(const float2* spec, ddc* out, int M, const SpecTables& tb32,
                               const SpecTables& tbdd, const DevScalars* sc, cudaStream_t st) {
  const size_t sm = 7 * (size_t)N * sizeof(ulonglong2);
  cudaError_t e = prepare_launch(k_col_lbarinv_pair<N, MODE>, N / 4, sm);
  if (e != cudaSuccess) return e;
  k_col_lbarinv_pair<N, MODE><<<M / 4, N / 4, sm, st>>>(
      spec, out, M, (float)(1.0 / ((double)N * (double)M)), (const float2*)tb32.twN,
      (const float2*)tb32.twM, (const ddc*)tbdd.twN, sc, (const float2*)tb32.symx,
      (const float2*)tb32.symy);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t col_lbarinv_pair_mode(const float2* spec, ddc* out, int N, int M,
                                  const SpecTables& tb32, const SpecTables& tbdd,
                                  const DevScalars* sc, cudaStream_t st) {
  switch (N) {
    case 256: return col_lbarinv_pair_N<256, MODE>(spec, out, M, tb32, tbdd, sc, st);
    case 512: return col_lbarinv_pair_N<512, MODE>(spec, out, M, tb32, tbdd, sc, st);
    case 1024: return col_lbarinv_pair_N<1024, MODE>(spec, out, M, tb32, tbdd, sc, st);
    case 2048: return col_lbarinv_pair_N<2048, MODE>(spec, out, M, tb32, tbdd, sc, st);
  }
  return cudaErrorInvalidValue;
}

template <int L>
cudaError_t row_update_pair_L(const ddc* q, const double* u_in, double* u_out, double step,
                              int N, const SpecTables& tbdd, const DevScalars* sc,
                              cudaStream_t st) {
  const size_t sm = 4 * (size_t)L * sizeof(ulonglong2);
  cudaError_t e = prepare_launch(k_row_update_pair<L>, L / 4, sm);
  if (e != cudaSuccess) return e;
  k_row_update_pair<L><<<N / 2, L / 4, sm, st>>>(q, u_in, u_out, step, N, (const ddc*)tbdd.twL,
                                                 (const ddc*)tbdd.twM, sc);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_col_lbarinv_pair(const float2* spec, ddc* out, int N, int M,
                                    const SpecTables& tb32, const SpecTables& tbdd,
                                    const DevScalars* sc, cudaStream_t st, int mode) {
  if (!col_pair_supported(N, M)) return cudaErrorInvalidValue;
  if ((uintptr_t)spec & 15) return cudaErrorMisalignedAddress;
  switch (mode) {
    case COL_LBARINV:
      if (!sc) return cudaErrorInvalidValue;
      return col_lbarinv_pair_mode<COL_LBARINV>(spec, out, N, M, tb32, tbdd, sc, st);
    case COL_POISSON:
      return col_lbarinv_pair_mode<COL_POISSON>(spec, out, N, M, tb32, tbdd, sc, st);
    case COL_POISSON_LP:
      return col_lbarinv_pair_mode<COL_POISSON_LP>(spec, out, N, M, tb32, tbdd, sc, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_row_update_pair(const ddc* q, const double* u_in, double* u_out,
                                   double step, int N, int M, const SpecTables& tbdd,
                                   const DevScalars* sc, cudaStream_t st) {
  if (!comb_pair_supported(N, M)) return cudaErrorInvalidValue;
  switch (M / 2) {
    case 256: return row_update_pair_L<256>(q, u_in, u_out, step, N, tbdd, sc, st);
    case 512: return row_update_pair_L<512>(q, u_in, u_out, step, N, tbdd, sc, st);
    case 1024: return row_update_pair_L<1024>(q, u_in, u_out, step, N, tbdd, sc, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace otgb
