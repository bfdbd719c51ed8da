// FP32 instantiation of the spectral kernels (inner precision of the mixed mode).
#include "spectral.cuh"
namespace otgb {
OTGB_INSTANTIATE_SPECTRAL(float)

cudaError_t launch_col_lbarinv_mixed(const float2* spec, double2* out, int N, int M,
                                     const SpecTables& tb32, const SpecTables& tb64,
                                     const DevScalars* sc, cudaStream_t st) {
  if (fft_E(N) == 12) return col_lbarinv_mixed_E<12>(spec, out, N, M, tb32, tb64, sc, st);
  return col_lbarinv_mixed_E<8>(spec, out, N, M, tb32, tb64, sc, st);
}
template <int MODE>
static cudaError_t col_lbarinv_dd_mode(const float2* spec, ddc* out, int N, int M,
                                       const SpecTables& tb32, const SpecTables& tbdd,
                                       const DevScalars* sc, cudaStream_t st, Bat bat = Bat()) {
  if (fft_E(N) == 12)
    return col_lbarinv_dd_E<12, MODE>(spec, out, N, M, tb32, tbdd, sc, st, bat);
  // 4 elements per thread while a column fits one block of 256 threads (the kernel's bound)
  if (N >= 16 && N / 4 <= 256)
    return col_lbarinv_dd_E<4, MODE>(spec, out, N, M, tb32, tbdd, sc, st, bat);
  return col_lbarinv_dd_E<8, MODE>(spec, out, N, M, tb32, tbdd, sc, st, bat);
}
cudaError_t launch_col_lbarinv_dd(const float2* spec, ddc* out, int N, int M,
                                  const SpecTables& tb32, const SpecTables& tbdd,
                                  const DevScalars* sc, cudaStream_t st, int mode, Bat bat) {
  if (!bat.on && tb32.theta_pair && col_pair_supported(N, M) && (mode != COL_LBARINV || sc))
    return launch_col_lbarinv_pair(spec, out, N, M, tb32, tbdd, sc, st, mode);
  switch (mode) {
    case COL_LBARINV:
      return col_lbarinv_dd_mode<COL_LBARINV>(spec, out, N, M, tb32, tbdd, sc, st, bat);
    case COL_POISSON:
      return col_lbarinv_dd_mode<COL_POISSON>(spec, out, N, M, tb32, tbdd, sc, st);
    case COL_POISSON_LP:
      return col_lbarinv_dd_mode<COL_POISSON_LP>(spec, out, N, M, tb32, tbdd, sc, st);
  }
  return cudaErrorInvalidValue;
}
cudaError_t launch_row_c2r_update_dd(const ddc* q, const double* u_in, double* u_out,
                                     double step, int N, int M, const SpecTables& tbdd,
                                     const DevScalars* sc, cudaStream_t st, Bat bat) {
  if (!bat.on && tbdd.theta_pair && comb_pair_supported(N, M))
    return launch_row_update_pair(q, u_in, u_out, step, N, M, tbdd, sc, st);
  if (fft_E(M / 2) == 12)
    return row_c2r_update_dd_E<12>(q, u_in, u_out, step, N, M, tbdd, sc, st, bat);
  if (M / 2 >= 16 && (M / 2) / 4 <= 256)
    return row_c2r_update_dd_E<4>(q, u_in, u_out, step, N, M, tbdd, sc, st, bat);
  return row_c2r_update_dd_E<8>(q, u_in, u_out, step, N, M, tbdd, sc, st, bat);
}
}
