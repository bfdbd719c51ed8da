// The FP32 Arnoldi update of step j fused with the row real-to-complex pass of step j + 1's
// matrix-vector product (Sec. 4.2: GMRES(m) on L Lbar^{-1} sigma, the product's first
// transform pass).  v_(j+1) is consumed by the next product's row transforms as soon as it
// exists: the kernel forms it row by row and transforms each row while it is still in shared
// memory, instead of writing it, ending the launch, and reading it back in the next one.
//
// Block 0 closes the step (the Givens close of one thread, as in the split update); blocks
// 1.. take RB whole rows each: v = w - sum_i h_i scale_i V_i on the row (stored unscaled, the
// update's own result, bit for bit), then the row's transform of v * (1 / hn) -- the next
// step's scale, which every block has from the same finished multi-dot -- and its
// real-to-complex split into the half spectrum (the row pass's own result, bit for bit).
// After the last step of a cycle (j + 1 = m) there is no next product and the rows stop
// after the update.
#include "gmres_dev.cuh"
#include "spectral.cuh"

namespace otgb {

template <int J, int E>
__device__ __forceinline__ void update_r2c_j(float* __restrict__ V, const float* __restrict__ w,
                                             long P, const double* partials, int nb,
                                             DevScalars* sc, float2* __restrict__ spec, int N,
                                             int M, int RB, const float2* __restrict__ twL,
                                             const float2* __restrict__ twM) {
  constexpr int j = J - 1;
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
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  const int L = M / 2, TPT = L / E;
  const int q = threadIdx.x / TPT, t = threadIdx.x % TPT;
  const int row = (blockIdx.x - 1) * RB + q;
  const bool active = row < N;
  float2* buf = sm + q * FB(L);
  const float s = (float)inv_hn;  // the row pass's (float) scale[j + 1]
  if (active) {
    const float2* wr = reinterpret_cast<const float2*>(w + (size_t)row * M);
    float2* vr = reinterpret_cast<float2*>(V + (size_t)(j + 1) * P + (size_t)row * M);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int n = t + e * TPT;
      float2 x = wr[n];
#pragma unroll
      for (int i = 0; i < J; ++i) {
        const float2 y =
            reinterpret_cast<const float2*>(V + (size_t)i * P + (size_t)row * M)[n];
        x.x -= coefs[i] * y.x;
        x.y -= coefs[i] * y.y;
      }
      vr[n] = x;
      buf[n] = make_float2(x.x * s, x.y * s);
    }
  }
  if (J >= sc->m) return;  // the cycle's last step: no next product (block-uniform)
  __syncthreads();
  fft_smem<float, E, -1>(buf, L, t, active, twL);
  if (active) r2c_split_store<float>(buf, spec + (size_t)row * L, L, t, TPT, twM);
}

template <int E>
__global__ void __launch_bounds__(512)
    k_gmres_update_r2c(float* __restrict__ V, const float* __restrict__ w, long P,
                       const double* partials, int nb, DevScalars* sc,
                       float2* __restrict__ spec, int N, int M, int RB,
                       const float2* __restrict__ twL, const float2* __restrict__ twM) {
  if (sc->cycle_done) return;
  // the step closed by this launch: jd, set by the multi-dot (sc->j moves on in the close)
  switch (sc->jd) {
#define OTGB_UPDR2C_CASE(k)                                                             \
  case k:                                                                               \
    update_r2c_j<k + 1, E>(V, w, P, partials, nb, sc, spec, N, M, RB, twL, twM); break;
    OTGB_UPDR2C_CASE(0) OTGB_UPDR2C_CASE(1) OTGB_UPDR2C_CASE(2) OTGB_UPDR2C_CASE(3)
    OTGB_UPDR2C_CASE(4) OTGB_UPDR2C_CASE(5) OTGB_UPDR2C_CASE(6) OTGB_UPDR2C_CASE(7)
    OTGB_UPDR2C_CASE(8) OTGB_UPDR2C_CASE(9) OTGB_UPDR2C_CASE(10) OTGB_UPDR2C_CASE(11)
    OTGB_UPDR2C_CASE(12) OTGB_UPDR2C_CASE(13) OTGB_UPDR2C_CASE(14)
#undef OTGB_UPDR2C_CASE
  }
}

// elements per thread of the fused kernel's row transform: the row pass's own choice (4 for
// the radix-4 variant, else the generic 8); 0 where the row pass has no such form (lengths
// with a factor 3, the warp-synchronous variant)
static int update_r2c_E(int M, int var_r2c) {
  const int L = M / 2;
  if (L < 8 || fft_E(L) != 8) return 0;
  if (var_r2c == VAR_E4 || var_r2c == VAR_PAIR) return 4;
  if (var_r2c == VAR_DEFAULT || var_r2c == VAR_GENERIC) return 8;
  return 0;
}

// rows per block as the row pass chooses them (RB = 0: no launch form, fewer than 32
// threads for the multi-dot finish's warps)
static int update_r2c_rows(int N, int M, int E) {
  const int L = M / 2, TPT = L / E;
  int RB = 512 / TPT;
  if (RB < 1) RB = 1;
  while (RB > 1 && RB * TPT > 128 && (N + RB - 1) / RB < 4 * 152) RB /= 2;
  if (RB > N) RB = N;
  return RB * TPT >= 32 ? RB : 0;
}

bool update_r2c_fits(int N, int M, int var_r2c) {
  if (var_r2c == VAR_PAIR && comb_pair_supported(N, M)) return true;
  const int E = update_r2c_E(M, var_r2c);
  return E != 0 && update_r2c_rows(N, M, E) > 0;
}

template <int E>
static cudaError_t update_r2c_launch(float* V, const float* w, long P, const double* partials,
                                     int nb, DevScalars* sc, float2* spec, int N, int M,
                                     const SpecTables& tb, cudaStream_t st) {
  const int L = M / 2, TPT = L / E;
  const int RB = update_r2c_rows(N, M, E);
  if (RB == 0) return cudaErrorInvalidConfiguration;
  const size_t sm = (size_t)RB * FB(L) * sizeof(float2);
  cudaError_t e = prepare_launch(k_gmres_update_r2c<E>, RB * TPT, sm);
  if (e != cudaSuccess) return e;
  k_gmres_update_r2c<E><<<1 + (N + RB - 1) / RB, RB * TPT, sm, st>>>(
      V, w, P, partials, nb, sc, spec, N, M, RB, (const float2*)tb.twL, (const float2*)tb.twM);
  return cudaGetLastError();
}

cudaError_t launch_gmres_update_r2c(float* V, const float* w, long P, const double* partials,
                                    int nb, DevScalars* sc, float2* spec, int N, int M,
                                    const SpecTables& tb, cudaStream_t st) {
  // the row pair pass's fused form (the same transform and split as that pass)
  if (tb.var_r2c == VAR_PAIR && comb_pair_supported(N, M))
    return launch_gmres_update_r2c_pair(V, w, P, partials, nb, sc, spec, N, M, tb, st);
  switch (update_r2c_E(M, tb.var_r2c)) {
    case 4: return update_r2c_launch<4>(V, w, P, partials, nb, sc, spec, N, M, tb, st);
    case 8: return update_r2c_launch<8>(V, w, P, partials, nb, sc, spec, N, M, tb, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace otgb
