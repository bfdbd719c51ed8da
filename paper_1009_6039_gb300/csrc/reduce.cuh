// FP64 block and grid reductions shared by the kernel files: warp shuffles, a block
// reduction of NV values (sum, max or min), and the last-block pattern (every block writes
// its partials and takes a ticket; the last block reduces the partials in block order, so the
// result is bit-reproducible).
#pragma once
#include <math.h>

#include "otgb_internal.cuh"

namespace otgb {

// ---------------------------------------------------------------------------------------
// block reductions
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Reduce NV values per thread over the block (kind: 0 sum, 1 max, 2 min per value);
// result valid in thread 0.  Needs blockDim.x a multiple of 32 and <= 1024.
template <int NV>
__device__ void block_reduce(double (&v)[NV], const int (&kind)[NV]) {
  __shared__ double red[32][NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int a = 0; a < NV; ++a)
    v[a] = kind[a] == 0 ? warp_sum(v[a]) : (kind[a] == 1 ? warp_max(v[a]) : warp_min(v[a]));
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int a = 0; a < NV; ++a) red[wid][a] = v[a];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      double init = kind[a] == 0 ? 0.0 : (kind[a] == 1 ? -INFINITY : INFINITY);
      double x = lane < nw ? red[lane][a] : init;
      v[a] = kind[a] == 0 ? warp_sum(x) : (kind[a] == 1 ? warp_max(x) : warp_min(x));
    }
  }
  __syncthreads();
}

// Write the block's partials, take a ticket; returns true in the (whole) last block,
// after which `partials` of all blocks are visible.
template <int NV>
__device__ bool publish_partials(const double (&v)[NV], double* partials, unsigned int* ticket) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    const size_t bid = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    for (int a = 0; a < NV; ++a) partials[bid * NV + a] = v[a];
    __threadfence();
    unsigned int nb = gridDim.x * gridDim.y;
    unsigned int k = atomicAdd(ticket, 1u);
    last = (k == nb - 1);
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// In the last block: reduce the per-block partials in block order (each thread a strided
// subset, then a block reduction).
template <int NV>
__device__ void reduce_partials(double (&v)[NV], const int (&kind)[NV], const double* partials,
                                unsigned int nb) {
#pragma unroll
  for (int a = 0; a < NV; ++a) v[a] = kind[a] == 0 ? 0.0 : (kind[a] == 1 ? -INFINITY : INFINITY);
  for (unsigned int b = threadIdx.x; b < nb; b += blockDim.x) {
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      double x = ((volatile const double*)partials)[(size_t)b * NV + a];
      v[a] = kind[a] == 0 ? v[a] + x : (kind[a] == 1 ? fmax(v[a], x) : fmin(v[a], x));
    }
  }
  block_reduce<NV>(v, kind);
}

}  // namespace otgb
