// Residual/coefficient evaluation that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that hands all device memory to its own pool
// (a framework's caching allocator, a fixed-budget service), and latency-critical loops
// that cannot afford cudaMalloc's implicit device-wide synchronisation.  For them this file
// provides ot_eval_residual_noalloc, the same residual kernel as ot_eval_residual but with
// its scratch -- the per-block reduction partials and the device scalar block -- in a
// file-scope __device__ array of fixed size, which every GPU that loads the library holds
// until the process exits.  The caller still passes all inputs and outputs.
#include <mutex>
#include <string.h>

#include "../../include/otgb.h"
#include "otgb_internal.cuh"

namespace {

// Largest grid served: N, M <= 2048.  The residual kernel uses one block per 32 x 32 tile,
// i.e. at most 64 * 64 = 4096 blocks with 10 partials each; the l2 reduction uses 2 blocks
// per SM with 1 partial each (far fewer).
constexpr int kMaxSide = 2048;
constexpr size_t kMaxResidualBlocks = (kMaxSide / 32) * (kMaxSide / 32);
constexpr size_t kHeaderBytes = (sizeof(otgb::DevScalars) + 255) / 256 * 256;
constexpr size_t kPartialBytes = kMaxResidualBlocks * 10 * sizeof(double);
constexpr size_t kScratchBytes = kHeaderBytes + kPartialBytes;  // about 330 KB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch, looked up once per device with that device current.
// (In host code the symbol names a host-side stand-in, not device memory.)
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};

int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return OT_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return OT_ECUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return OT_ECUDA;
    }
    g_scratch_addr[dev] = (unsigned char*)ptr;
  }
  *out = g_scratch_addr[dev];
  return OT_OK;
}

}  // namespace

using namespace otgb;

extern "C" int ot_eval_residual_noalloc(int32_t N, int32_t M, const double* f, const double* c,
                                        const double* u, double* F, double* coef, double* scal,
                                        void* cuda_stream) {
  if (!f || !c || !u || !F || !coef) return OT_EINVAL;
  if (N < 8 || M < 8) return OT_EINVAL;
  if (N > kMaxSide || M > kMaxSide) return OT_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (st) {
    // the scratch array is the current device's: a stream of another device is refused
    int cur = 0, sdev = 0;
    if (cudaGetDevice(&cur) != cudaSuccess || cudaStreamGetDevice(st, &sdev) != cudaSuccess) {
      cudaGetLastError();
      return OT_EINVAL;
    }
    if (sdev != cur) return OT_EINVAL;
  }
  unsigned char* base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc != OT_OK) return rc;
  DevScalars* sc = (DevScalars*)base;
  double* partials = (double*)(base + kHeaderBytes);
  // the array keeps the previous call's contents: the reduction tickets must start at zero
  if (cudaMemsetAsync(sc, 0, sizeof(DevScalars), st) != cudaSuccess) return OT_ECUDA;
  // F receives f - f_n first, then the mass translation shift in place
  if (launch_residual<double>(f, c, u, N, M, F, coef, partials, sc, st) != cudaSuccess)
    return OT_ECUDA;
  if (launch_residual_l2(F, N, M, partials, sc, st) != cudaSuccess) return OT_ECUDA;
  if (launch_shifted_residual(F, F, N, M, sc, st) != cudaSuccess) return OT_ECUDA;
  DevScalars h;
  if (cudaMemcpyAsync(&h, sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return OT_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return OT_ECUDA;
  if (scal) {
    scal[0] = h.mean_fn;
    scal[1] = h.res_inf;
    scal[2] = sqrt(h.res_l2sum / ((double)N * (double)M));
    scal[3] = h.min_det;
    scal[4] = h.k1_nonfinite;
    for (int a = 0; a < 5; ++a) scal[5 + a] = h.abar[a];
  }
  return OT_OK;
}
