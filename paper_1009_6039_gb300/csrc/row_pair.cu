// The FP32 row real-to-complex pass (the first pass of the matvec, Sec. 4.2) on row pairs,
// and the Arnoldi update of GMRES(m) fused with it (as k_gmres_update_r2c, on row pairs).
//
// One block takes two neighbouring rows r0 = 2b and r0 + 1 side by side, as the column and
// combine pair passes do (pair.cuh): the row's length-M/2 complex transform of its M real
// values packed as z_n = x_2n + i x_(2n+1) runs on packed register pairs, and so does the
// real-to-complex split into the packed half spectrum (X_0 and X_(M/2) as one complex entry).
// The fused kernel forms v_(j+1) = w - sum_i h_i scale_i V_i on both rows with the scalar
// update's own arithmetic (the stored basis vector is bit for bit the split update's), then
// transforms v_(j+1) / hn while it is in shared memory; its transform and split are the row
// pair pass's own functions, so the fused and the separate launches agree bit for bit.
#include "gmres_dev.cuh"
#include "pair.cuh"

namespace otgb {
namespace {

using namespace pair;

__device__ __forceinline__ void st_pair(float2* outa, float2* outb, int k, PC v) {
  float2 a, b;
  upk(v.re, a.x, b.x);
  upk(v.im, a.y, b.y);
  outa[k] = a;
  outb[k] = b;
}

// the row pair's transform (from P0, scratch P1; buf: where it ends) and its split into the
// two rows' half spectra: X_k = E + W_M^k O, X_(L-k) = conj(E - W_M^k O) with
// E = (Z_k + conj Z_(L-k)) / 2, O = -i (Z_k - conj Z_(L-k)) / 2, X_0 packed as (X_0, X_L)
template <int L>
__device__ __forceinline__ void r2c_pair_transform_split(PC* P0, PC* P1, float2* outa,
                                                         float2* outb, int t,
                                                         const ulonglong2* __restrict__ tw4,
                                                         const float2* __restrict__ twM) {
  constexpr int TPT = L / 4;
  {
    PC* const a[1] = {P0};
    PC* const b[1] = {P1};
    pfft_rec<-1, L, 1, L, 1, true>(a, b, t, tw4);
  }
  const PC* buf = pstage_count<L>() % 2 == 1 ? P1 : P0;
  const u64 half = pk(0.5f, 0.5f), nhalf = pk(-0.5f, -0.5f);
  for (int k = t; k <= L / 2; k += TPT) {
    if (k == 0) {
      const PC z = buf[swz(0)];
      PC o;
      o.re = add2(z.re, z.im);
      o.im = sub2(z.re, z.im);
      st_pair(outa, outb, 0, o);
    } else {
      const PC zk = buf[swz(k)], zm = buf[swz(L - k)];
      PC Ev, Ov;
      Ev.re = mul2(half, add2(zk.re, zm.re));
      Ev.im = mul2(half, sub2(zk.im, zm.im));
      Ov.re = mul2(half, add2(zk.im, zm.im));
      Ov.im = mul2(nhalf, sub2(zk.re, zm.re));
      const float2 w = twM[k];
      const PC wo = cmulp<-1>(Ov, pk(w.x, w.x), pk(w.y, w.y), pk(-w.y, -w.y));
      PC xk;
      xk.re = add2(Ev.re, wo.re);
      xk.im = add2(Ev.im, wo.im);
      st_pair(outa, outb, k, xk);
      if (2 * k != L) {
        PC xm;
        xm.re = sub2(Ev.re, wo.re);
        xm.im = sub2(wo.im, Ev.im);
        st_pair(outa, outb, L - k, xm);
      }
    }
  }
}

// shared memory of both kernels: the broadcast stage twiddles and two pair buffers
template <int L>
constexpr size_t row_pair_smem() {
  return (size_t)L * sizeof(ulonglong2) + 2 * (size_t)L * sizeof(PC);
}

// rows of x = xbase + (*jptr) x_stride (jptr NULL: xbase), times scale[*jptr] (NULL: 1)
template <int L>
__global__ void __launch_bounds__(L / 4)
    k_row_r2c_pair(const float* __restrict__ xbase, size_t x_stride, const int* __restrict__ jptr,
                   const double* __restrict__ scale, float2* __restrict__ spec,
                   const float2* __restrict__ twL, const float2* __restrict__ twM,
                   const int* __restrict__ skip) {
  if (skip && *skip) return;
  constexpr int TPT = L / 4, M = 2 * L;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ulonglong2* tw4 = reinterpret_cast<ulonglong2*>(smem_raw);
  PC* P0 = reinterpret_cast<PC*>(tw4 + L);
  PC* P1 = P0 + L;
  const int r0 = 2 * blockIdx.x;
  const int t = threadIdx.x;
  const int jv = jptr ? *jptr : 0;
  const float* x = xbase + (size_t)jv * x_stride;
  const float s = scale ? (float)scale[jv] : 1.f;
  load_tw4<L>(tw4, twL, t, TPT);
  const float2* xa = reinterpret_cast<const float2*>(x + (size_t)r0 * M);
  const float2* xb = xa + L;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int n = t + e * TPT;
    const float2 za = xa[n], zb = xb[n];
    PC v;
    v.re = pk(za.x * s, zb.x * s);
    v.im = pk(za.y * s, zb.y * s);
    P0[swz(n)] = v;
  }
  __syncthreads();
  r2c_pair_transform_split<L>(P0, P1, spec + (size_t)r0 * L, spec + (size_t)(r0 + 1) * L, t,
                              tw4, twM);
}

template <int J, int L>
__device__ __forceinline__ void update_r2c_pair_j(float* __restrict__ V,
                                                  const float* __restrict__ w, long P,
                                                  const double* partials, int nb,
                                                  DevScalars* sc, float2* __restrict__ spec,
                                                  const float2* __restrict__ twL,
                                                  const float2* __restrict__ twM) {
  constexpr int j = J - 1;
  constexpr int TPT = L / 4, M = 2 * L;
  double hv[J], hn = 0.0, inv_hn = 0.0;
  bool weak = false;
  float coefs[J];
  finish_multidot_f32<J>(partials, nb, sc, hv, hn, inv_hn, weak, coefs);
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) {
#pragma unroll
      for (int i = 0; i < J; ++i) sc->hcol[i] = hv[i];
      arnoldi_close_j<J, true>(sc, hv, hn, weak, inv_hn);
    }
    return;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ulonglong2* tw4 = reinterpret_cast<ulonglong2*>(smem_raw);
  PC* P0 = reinterpret_cast<PC*>(tw4 + L);
  PC* P1 = P0 + L;
  const int r0 = 2 * (blockIdx.x - 1);
  const int t = threadIdx.x;
  const float s = (float)inv_hn;  // the row pass's (float) scale[j + 1]
  const bool next = J < sc->m;    // a next product (block-uniform)
  if (next) load_tw4<L>(tw4, twL, t, TPT);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int n = t + e * TPT;
    float2 xr[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const size_t ro = (size_t)(r0 + h) * M;
      float2 x = reinterpret_cast<const float2*>(w + ro)[n];
#pragma unroll
      for (int i = 0; i < J; ++i) {
        const float2 y = reinterpret_cast<const float2*>(V + (size_t)i * P + ro)[n];
        x.x -= coefs[i] * y.x;
        x.y -= coefs[i] * y.y;
      }
      reinterpret_cast<float2*>(V + (size_t)(j + 1) * P + ro)[n] = x;
      xr[h] = x;
    }
    if (next) {
      PC v;
      v.re = pk(xr[0].x * s, xr[1].x * s);
      v.im = pk(xr[0].y * s, xr[1].y * s);
      P0[swz(n)] = v;
    }
  }
  if (!next) return;  // the cycle's last step: no next product
  __syncthreads();
  r2c_pair_transform_split<L>(P0, P1, spec + (size_t)r0 * L, spec + (size_t)(r0 + 1) * L, t,
                              tw4, twM);
}

template <int L>
__global__ void __launch_bounds__(L / 4)
    k_gmres_update_r2c_pair(float* __restrict__ V, const float* __restrict__ w, long P,
                            const double* partials, int nb, DevScalars* sc,
                            float2* __restrict__ spec, const float2* __restrict__ twL,
                            const float2* __restrict__ twM) {
  if (sc->cycle_done) return;
  switch (sc->jd) {
#define OTGB_UPDR2CP_CASE(k)                                                            \
  case k:                                                                               \
    update_r2c_pair_j<k + 1, L>(V, w, P, partials, nb, sc, spec, twL, twM); break;
    OTGB_UPDR2CP_CASE(0) OTGB_UPDR2CP_CASE(1) OTGB_UPDR2CP_CASE(2) OTGB_UPDR2CP_CASE(3)
    OTGB_UPDR2CP_CASE(4) OTGB_UPDR2CP_CASE(5) OTGB_UPDR2CP_CASE(6) OTGB_UPDR2CP_CASE(7)
    OTGB_UPDR2CP_CASE(8) OTGB_UPDR2CP_CASE(9) OTGB_UPDR2CP_CASE(10) OTGB_UPDR2CP_CASE(11)
    OTGB_UPDR2CP_CASE(12) OTGB_UPDR2CP_CASE(13) OTGB_UPDR2CP_CASE(14)
#undef OTGB_UPDR2CP_CASE
  }
}

template <int L>
cudaError_t row_r2c_pair_L(const float* x, size_t xs, const int* jptr, const double* scale,
                           float2* spec, int N, const SpecTables& tb, const int* skip,
                           cudaStream_t st) {
  const size_t sm = row_pair_smem<L>();
  cudaError_t e = prepare_launch(k_row_r2c_pair<L>, L / 4, sm);
  if (e != cudaSuccess) return e;
  k_row_r2c_pair<L><<<N / 2, L / 4, sm, st>>>(x, xs, jptr, scale, spec, (const float2*)tb.twL,
                                              (const float2*)tb.twM, skip);
  return cudaGetLastError();
}

template <int L>
cudaError_t update_r2c_pair_L(float* V, const float* w, long P, const double* partials, int nb,
                              DevScalars* sc, float2* spec, int N, const SpecTables& tb,
                              cudaStream_t st) {
  const size_t sm = row_pair_smem<L>();
  cudaError_t e = prepare_launch(k_gmres_update_r2c_pair<L>, L / 4, sm);
  if (e != cudaSuccess) return e;
  k_gmres_update_r2c_pair<L><<<1 + N / 2, L / 4, sm, st>>>(
      V, w, P, partials, nb, sc, spec, (const float2*)tb.twL, (const float2*)tb.twM);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_row_r2c_pair(const float* x, size_t xs, const int* jptr, const double* scale,
                                float2* spec, int N, int M, const SpecTables& tb,
                                const int* skip, cudaStream_t st) {
  if (!comb_pair_supported(N, M)) return cudaErrorInvalidValue;
  switch (M / 2) {
    case 256: return row_r2c_pair_L<256>(x, xs, jptr, scale, spec, N, tb, skip, st);
    case 512: return row_r2c_pair_L<512>(x, xs, jptr, scale, spec, N, tb, skip, st);
    case 1024: return row_r2c_pair_L<1024>(x, xs, jptr, scale, spec, N, tb, skip, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_gmres_update_r2c_pair(float* V, const float* w, long P,
                                         const double* partials, int nb, DevScalars* sc,
                                         float2* spec, int N, int M, const SpecTables& tb,
                                         cudaStream_t st) {
  if (!comb_pair_supported(N, M)) return cudaErrorInvalidValue;
  switch (M / 2) {
    case 256: return update_r2c_pair_L<256>(V, w, P, partials, nb, sc, spec, N, tb, st);
    case 512: return update_r2c_pair_L<512>(V, w, P, partials, nb, sc, spec, N, tb, st);
    case 1024: return update_r2c_pair_L<1024>(V, w, P, partials, nb, sc, spec, N, tb, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace otgb
