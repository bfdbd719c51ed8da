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
}
