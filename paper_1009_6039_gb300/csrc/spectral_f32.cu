// FP32 instantiation of the spectral kernels (inner precision of the mixed mode).
#include "spectral.cuh"
namespace otgb {
OTGB_INSTANTIATE_SPECTRAL(float)
}
