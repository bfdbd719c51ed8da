// FP64 instantiation of the spectral kernels.
#include "spectral.cuh"
namespace otgb {
OTGB_INSTANTIATE_SPECTRAL(double)
}
