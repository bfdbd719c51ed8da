// Column pass of the FP32 matvec (Sec. 4.2) on column pairs with packed FP32 arithmetic.
//
// The pass computes what k_col<float, E, COL_MATVEC> computes -- per column of the packed
// N x M/2 half spectrum: the forward column FFT, S = rho-bar sigma-hat / (N M), and the
// inverse column FFTs of S (its Nyquist channel premultiplied), (i s1(k2)) S and s2(k2) S --
// but one block takes two neighbouring columns c0 = 2b and c0 + 1 and holds them side by
// side: the element n of a transform pair is the 16-byte word (a.x, b.x, a.y, b.y) of the
// two columns' values a and b.  The real parts and the imaginary parts of the pair are then
// register pairs, so every complex addition of a butterfly is one packed instruction
// (add/sub.rn.f32x2) for both columns, and every twiddle multiplication two packed
// multiply-adds per part, with the twiddle broadcast to both lanes; the multiplication by
// +-i exchanges the parts and costs nothing.  A thread holds 4 elements (radix-4 stages,
// one radix-2 stage for odd powers of two), the length is fixed at compile time
// (256 ... 2048), and the stages run out of place between two buffer sets (one barrier a
// stage).  Shared memory is addressed through an XOR swizzle of the 16-byte element index,
// i ^ ((i >> 2) & 7), under which every stage's reads and writes of a quarter warp fall in
// distinct bank groups.  The symbol multiplies are the scalar operations of k_col.
#include "pair.cuh"

namespace otgb {
namespace {

using namespace pair;

template <int N>
__global__ void __launch_bounds__(N / 4, N <= 1024 ? 2 : 1)
    k_col_pair(const float2* __restrict__ spec, float2* __restrict__ out0,
               float2* __restrict__ out1, float2* __restrict__ out2, int M, float inv,
               const float2* __restrict__ twN, const DevScalars* __restrict__ sc,
               const int* __restrict__ skip, const float2* __restrict__ symx,
               const float2* __restrict__ symy) {
  if (skip && *skip) return;
  constexpr int TPT = N / 4;
  constexpr bool ODD = pstage_count<N>() % 2 == 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ulonglong2* tw4 = reinterpret_cast<ulonglong2*>(smem_raw);
  PC* pb = reinterpret_cast<PC*>(smem_raw + (size_t)N * sizeof(ulonglong2));
  PC* const P[6] = {pb, pb + N, pb + 2 * N, pb + 3 * N, pb + 4 * N, pb + 5 * N};
  const int Lc = M / 2;
  const int c0 = 2 * blockIdx.x;
  const int t = threadIdx.x;

  // the column pair: one 16-byte load per row, issued before the twiddle table is built so
  // that both sets of loads are in flight together, then regrouped into (re, im) pairs
  float4 xs[4];
#pragma unroll
  for (int e = 0; e < 4; ++e)
    xs[e] = *reinterpret_cast<const float4*>(spec + (size_t)(t + e * TPT) * Lc + c0);
  load_tw4<N>(tw4, twN, t, TPT);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    PC v;
    v.re = pk(xs[e].x, xs[e].z);
    v.im = pk(xs[e].y, xs[e].w);
    P[0][swz(t + e * TPT)] = v;
  }
  __syncthreads();

  // forward column transforms of both columns (from P0, scratch P3)
  {
    PC* const a[1] = {P[0]};
    PC* const b[1] = {P[3]};
    pfft_rec<-1, N, 1, N, 1, true>(a, b, t, tw4);
  }
  PC* const F = ODD ? P[3] : P[0];
  // the inverse transforms start in the set that does not hold F
  PC* const I0 = ODD ? P[0] : P[3];
  PC* const I1 = ODD ? P[1] : P[4];
  PC* const I2 = ODD ? P[2] : P[5];

  float ab[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) ab[q] = sc ? (float)sc->abar[q] : 0.f;
  const float2 sxa = symx[c0], sxb = symx[c0 + 1];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int k = t + e * TPT;
    const PC z = F[swz(k)];
    float2 za, zb;
    upk(z.re, za.x, zb.x);
    upk(z.im, za.y, zb.y);
    const float2 sy = symy[k];
    float2 sa, s0a;
    if (c0 == 0) {
      // the two real columns k1 = 0 and k1 = M/2 carried as X0 + i XL (as in k_col)
      const PC pz = F[swz((N - k) % N)];
      float2 p, pbv;
      upk(pz.re, p.x, pbv.x);
      upk(pz.im, p.y, pbv.y);
      float2 A = mk2<float>(0.5f * (za.x + p.x), 0.5f * (za.y - p.y));
      float2 B = mk2<float>(0.5f * (za.y + p.y), -0.5f * (za.x - p.x));
      A = cmul<float>(rho_bar<float>(ab, symx[0], sy), A);
      B = cmul<float>(rho_bar<float>(ab, symx[M / 2], sy), B);
      const float2 Bn = cscale<float>(B, symx[M / 2].y);
      s0a = cscale<float>(mk2<float>(A.x - Bn.y, A.y + Bn.x), inv);
      sa = cscale<float>(mk2<float>(A.x - B.y, A.y + B.x), inv);
    } else {
      sa = cscale<float>(cmul<float>(rho_bar<float>(ab, sxa, sy), za), inv);
      s0a = sa;
    }
    const float2 sb = cscale<float>(cmul<float>(rho_bar<float>(ab, sxb, sy), zb), inv);
    const int d = swz(k);
    PC q;
    q.re = pk(s0a.x, sb.x);
    q.im = pk(s0a.y, sb.y);
    I0[d] = q;
    q.re = pk(-sy.x * sa.y, -sy.x * sb.y);
    q.im = pk(sy.x * sa.x, sy.x * sb.x);
    I1[d] = q;
    q.re = pk(sa.x * sy.y, sb.x * sy.y);
    q.im = pk(sa.y * sy.y, sb.y * sy.y);
    I2[d] = q;
  }
  __syncthreads();

  // the three inverse transforms interleaved
  PC* const ia[3] = {I0, I1, I2};
  PC* const ib[3] = {ODD ? P[3] : P[0], ODD ? P[4] : P[1], ODD ? P[5] : P[2]};
  pfft_rec<+1, N, 1, N, 3, true>(ia, ib, t, tw4);
  PC* const* res = ODD ? ib : ia;
  float2* const outs[3] = {out0, out1, out2};
#pragma unroll
  for (int o = 0; o < 3; ++o) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int n = t + e * TPT;
      const PC v = res[o][swz(n)];
      float4 x;
      upk(v.re, x.x, x.z);
      upk(v.im, x.y, x.w);
      *reinterpret_cast<float4*>(outs[o] + (size_t)n * Lc + c0) = x;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Row combine pass of the FP32 matvec on row pairs (Sec. 4.2): the five complex-to-real
// row transforms d_xx Q0, d_x Q0, d_x Q1, Q1, Q2 of two neighbouring rows r0 = 2b and
// r0 + 1, held side by side as in k_col_pair, weighted by a11, b1, 2 a12, b2, a22 and summed
// into w = L Lbar^{-1} sigma.  The row symbols, the complex-to-real pre-processing, the
// transforms and the weighting all run on the packed pairs; the stages run in place (two
// barriers a stage), which keeps a block at 48 KB of shared memory at length 512, so that
// the N / 2 blocks of a 1024 x 1024 grid run in one wave.
// ---------------------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(L / 4, L <= 512 ? 4 : 2)
    k_comb_pair(const float2* __restrict__ q0, const float2* __restrict__ q1,
                const float2* __restrict__ q2, const float* __restrict__ coef,
                float* __restrict__ out, int N, const float2* __restrict__ twL,
                const float2* __restrict__ twM, const int* __restrict__ skip,
                const float2* __restrict__ symx) {
  if (skip && *skip) return;
  constexpr int TPT = L / 4;
  constexpr int M = 2 * L;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ulonglong2* tw4 = reinterpret_cast<ulonglong2*>(smem_raw);
  PC* pb = reinterpret_cast<PC*>(smem_raw + (size_t)L * sizeof(ulonglong2));
  PC* const B[5] = {pb, pb + L, pb + 2 * L, pb + 3 * L, pb + 4 * L};
  const int r0 = 2 * blockIdx.x;
  const int t = threadIdx.x;
  // the five terms of both rows: d_xx Q0, d_x Q0, d_x Q1, Q1, Q2 (row symbols of k1 = k; the
  // packed entry k = 0 holds (X0, X_L): d_x is 0 on both, d_xx keeps the Nyquist channel,
  // which Q0 carries premultiplied); the rows' loads are issued before the twiddle table is
  // built, so that both sets of loads are in flight together
  const size_t oa = (size_t)r0 * L, ob = oa + L;
  float2 ld[4][6];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int k = t + e * TPT;
    ld[e][0] = q0[oa + k];
    ld[e][1] = q0[ob + k];
    ld[e][2] = q1[oa + k];
    ld[e][3] = q1[ob + k];
    ld[e][4] = q2[oa + k];
    ld[e][5] = q2[ob + k];
  }
  load_tw4<L>(tw4, twL, t, TPT);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int k = t + e * TPT;
    const float2 a0 = ld[e][0], b0 = ld[e][1];
    const float2 a1 = ld[e][2], b1 = ld[e][3];
    const float2 a2 = ld[e][4], b2 = ld[e][5];
    PC x0, x1, x2;
    x0.re = pk(a0.x, b0.x);
    x0.im = pk(a0.y, b0.y);
    x1.re = pk(a1.x, b1.x);
    x1.im = pk(a1.y, b1.y);
    x2.re = pk(a2.x, b2.x);
    x2.im = pk(a2.y, b2.y);
    PC dxx, dx0, dx1;
    if (k == 0) {
      dxx.re = 0ull;
      dxx.im = x0.im;
      dx0.re = dx0.im = dx1.re = dx1.im = 0ull;
    } else {
      const float2 sx = symx[k];
      const u64 s2 = pk(sx.y, sx.y), s1 = pk(sx.x, sx.x), ns1 = pk(-sx.x, -sx.x);
      dxx.re = mul2(x0.re, s2);
      dxx.im = mul2(x0.im, s2);
      dx0.re = mul2(x0.im, ns1);
      dx0.im = mul2(x0.re, s1);
      dx1.re = mul2(x1.im, ns1);
      dx1.im = mul2(x1.re, s1);
    }
    const int d = swz(k);
    B[0][d] = dxx;
    B[1][d] = dx0;
    B[2][d] = dx1;
    B[3][d] = x1;
    B[4][d] = x2;
  }
  __syncthreads();

  // complex-to-real pre-processing: Z_k = (X_k + conj X_(L-k)) + i (X_k - conj X_(L-k))
  // conj(W_M^k), Z_(L-k) likewise, each pair (k, L - k) by one thread
  for (int k = t; k <= L / 2; k += TPT) {
    if (k == 0) {
      const int d = swz(0);
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const PC x = B[q][d];
        PC z;
        z.re = add2(x.re, x.im);
        z.im = sub2(x.re, x.im);
        B[q][d] = z;
      }
    } else {
      const float2 w = twM[k];
      const u64 wx = pk(w.x, w.x), wy = pk(w.y, w.y), nwy = pk(-w.y, -w.y);
      const int dk = swz(k), dm = swz(L - k);
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const PC xk = B[q][dk], xm = B[q][dm];
        PC E, D;
        E.re = add2(xk.re, xm.re);
        E.im = sub2(xk.im, xm.im);
        D.re = sub2(xk.re, xm.re);
        D.im = add2(xk.im, xm.im);
        const PC O = cmulp<+1>(D, wx, wy, nwy);
        PC zk;
        zk.re = sub2(E.re, O.im);
        zk.im = add2(E.im, O.re);
        B[q][dk] = zk;
        if (2 * k != L) {
          PC zm;
          zm.re = add2(E.re, O.im);
          zm.im = sub2(O.re, E.im);
          B[q][dm] = zm;
        }
      }
    }
  }
  __syncthreads();
  pfft_inplace<+1, L, 1, L, 5>(B, t, tw4);

  // w = a11 y0 + b1 y1 + 2 a12 y2 + b2 y3 + a22 y4 on both rows (the coefficient planes a11,
  // a12, a22, b1, b2 in that order)
  const size_t P = (size_t)N * M;
  const size_t ra = (size_t)r0 * M, rb = ra + M;
  const float2* c0 = reinterpret_cast<const float2*>(coef);
  const float2* c1 = reinterpret_cast<const float2*>(coef + P);
  const float2* c2 = reinterpret_cast<const float2*>(coef + 2 * P);
  const float2* c3 = reinterpret_cast<const float2*>(coef + 3 * P);
  const float2* c4 = reinterpret_cast<const float2*>(coef + 4 * P);
  float2* ov = reinterpret_cast<float2*>(out);
  const u64 two = pk(2.f, 2.f);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int n = t + e * TPT;
    const int d = swz(n);
    const size_t ia = ra / 2 + n, ib = rb / 2 + n;
    const float2 a11a = c0[ia], a11b = c0[ib], a12a = c1[ia], a12b = c1[ib];
    const float2 a22a = c2[ia], a22b = c2[ib], b1a = c3[ia], b1b = c3[ib];
    const float2 b2a = c4[ia], b2b = c4[ib];
    const PC y0 = B[0][d], y1 = B[1][d], y2 = B[2][d], y3 = B[3][d], y4 = B[4][d];
    u64 rr = mul2(pk(a11a.x, a11b.x), y0.re);
    rr = fma2(pk(b1a.x, b1b.x), y1.re, rr);
    rr = fma2(mul2(two, pk(a12a.x, a12b.x)), y2.re, rr);
    rr = fma2(pk(b2a.x, b2b.x), y3.re, rr);
    rr = fma2(pk(a22a.x, a22b.x), y4.re, rr);
    u64 ri = mul2(pk(a11a.y, a11b.y), y0.im);
    ri = fma2(pk(b1a.y, b1b.y), y1.im, ri);
    ri = fma2(mul2(two, pk(a12a.y, a12b.y)), y2.im, ri);
    ri = fma2(pk(b2a.y, b2b.y), y3.im, ri);
    ri = fma2(pk(a22a.y, a22b.y), y4.im, ri);
    float2 wa, wb;
    upk(rr, wa.x, wb.x);
    upk(ri, wa.y, wb.y);
    ov[ia] = wa;
    ov[ib] = wb;
  }
}

template <int L>
cudaError_t comb_pair_L(const float2* q0, const float2* q1, const float2* q2, const float* coef,
                        float* out, int N, const SpecTables& tb, const int* skip,
                        cudaStream_t st) {
  const size_t sm = (size_t)L * sizeof(ulonglong2) + 5 * (size_t)L * sizeof(PC);
  cudaError_t e = prepare_launch(k_comb_pair<L>, L / 4, sm);
  if (e != cudaSuccess) return e;
  k_comb_pair<L><<<N / 2, L / 4, sm, st>>>(q0, q1, q2, coef, out, N, (const float2*)tb.twL,
                                           (const float2*)tb.twM, skip,
                                           (const float2*)tb.symx);
  return cudaGetLastError();
}

template <int N>
cudaError_t col_pair_N(const float2* spec, float2* o0, float2* o1, float2* o2, int M,
                       const SpecTables& tb, const DevScalars* sc, const int* skip,
                       cudaStream_t st) {
  const size_t sm = (size_t)N * sizeof(ulonglong2) + 6 * (size_t)N * sizeof(PC);
  cudaError_t e = prepare_launch(k_col_pair<N>, N / 4, sm);
  if (e != cudaSuccess) return e;
  k_col_pair<N><<<M / 4, N / 4, sm, st>>>(
      spec, o0, o1, o2, M, (float)(1.0 / ((double)N * (double)M)), (const float2*)tb.twN, sc,
      skip, (const float2*)tb.symx, (const float2*)tb.symy);
  return cudaGetLastError();
}

}  // namespace

bool comb_pair_supported(int N, int M) {
  const int L = M / 2;
  return (L == 256 || L == 512 || L == 1024) && M == 2 * L && N >= 2 && N % 2 == 0;
}

cudaError_t launch_comb_pair(const float2* q0, const float2* q1, const float2* q2,
                             const float* coef, float* out, int N, int M, const SpecTables& tb,
                             const int* skip, cudaStream_t st) {
  if (!comb_pair_supported(N, M)) return cudaErrorInvalidValue;
  switch (M / 2) {
    case 256: return comb_pair_L<256>(q0, q1, q2, coef, out, N, tb, skip, st);
    case 512: return comb_pair_L<512>(q0, q1, q2, coef, out, N, tb, skip, st);
    case 1024: return comb_pair_L<1024>(q0, q1, q2, coef, out, N, tb, skip, st);
  }
  return cudaErrorInvalidValue;
}

bool col_pair_supported(int N, int M) {
  return (N == 256 || N == 512 || N == 1024 || N == 2048) && M >= 4 && M % 4 == 0;
}

cudaError_t launch_col_pair(const float2* spec, float2* o0, float2* o1, float2* o2, int N,
                            int M, const SpecTables& tb, const DevScalars* sc, const int* skip,
                            cudaStream_t st) {
  if (!col_pair_supported(N, M)) return cudaErrorInvalidValue;
  // 16-byte loads and stores of a column pair need 16-byte aligned planes
  if (((uintptr_t)spec | (uintptr_t)o0 | (uintptr_t)o1 | (uintptr_t)o2) & 15)
    return cudaErrorMisalignedAddress;
  switch (N) {
    case 256: return col_pair_N<256>(spec, o0, o1, o2, M, tb, sc, skip, st);
    case 512: return col_pair_N<512>(spec, o0, o1, o2, M, tb, sc, skip, st);
    case 1024: return col_pair_N<1024>(spec, o0, o1, o2, M, tb, sc, skip, st);
    case 2048: return col_pair_N<2048>(spec, o0, o1, o2, M, tb, sc, skip, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace otgb
