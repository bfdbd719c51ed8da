// Device pieces of the GMRES(m) Arnoldi step (Sec. 4.2) shared by the Krylov kernels: the
// finish of the FP32 multi-dot's block sums and the step's Givens close.
#pragma once

#include <math.h>

#include "otgb_internal.cuh"

namespace otgb {

// Finish the FP32 multi-dot of step j = J - 1 from the dots kernel's per-block sums (nb
// blocks, J + 1 values each: V_i.w for i < J, then w.w): every sum is taken by one warp in a
// fixed order (lane-strided, then a shuffle tree), so that every block of the calling grid
// obtains the same values.  h_i = scale_i V_i.w, and ||w - sum h_i v_i||^2 = w.w - sum h_i^2
// (Pythagoras, v_i orthonormal): below 1e-6 w.w the step is weak and the cycle ends (the
// restart's explicit residual decides).  The FP64 scalars are formed by thread 0 alone (FP64
// runs at a small fraction of the FP32 rate on this GPU, and every thread of a large grid
// forming them had become a visible part of the step) and shared through shared memory.
// Out, in every thread: the update's coefficients h_i scale_i (the basis is stored unscaled)
// and 1 / hn (0 when weak); in thread 0 only: h, hn = ||w - sum h_i v_i|| and weak.  All
// threads of the block call it (two barriers).
template <int J>
__device__ __forceinline__ void finish_multidot_f32(const double* partials, int nb,
                                                    const DevScalars* sc, double (&hv)[J],
                                                    double& hn, double& inv_hn, bool& weak,
                                                    float (&coefs)[J]) {
  // (the sums in FP32, as the block sums themselves)
  __shared__ float sv[OTGB_MAXM + 1];
  __shared__ float scoef[OTGB_MAXM];
  __shared__ double sinv;
  const float* pf = reinterpret_cast<const float*>(partials);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int a = wid; a <= J; a += nw) {
    float x = 0.f;
    for (int b = lane; b < nb; b += 32) x += pf[(size_t)b * (J + 1) + a];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sv[a] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double hs = 0.0;
#pragma unroll
    for (int i = 0; i < J; ++i) {
      hv[i] = sc->scale[i] * (double)sv[i];
      hs += hv[i] * hv[i];
    }
    const double ww = (double)sv[J], hn2 = ww - hs;
    weak = !(hn2 > 1e-6 * ww);
    inv_hn = weak ? 0.0 : rsqrt(hn2);
    hn = hn2 * inv_hn;
#pragma unroll
    for (int i = 0; i < J; ++i) scoef[i] = (float)(hv[i] * sc->scale[i]);
    sinv = inv_hn;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < J; ++i) coefs[i] = scoef[i];
  inv_hn = sinv;
}

// The Givens close of Arnoldi step j = J - 1 for the single-reduction step, with column j of
// H (h, before the rotations) in registers: the previous rotations on the column, the new
// rotation, g, the convergence test against eta ||b||, the next basis scale 1 / hn, the step
// count, and (in a graph) the conditional handle of the next step.  Every scalar it needs is
// loaded first, as independent loads, so that the one thread that runs it waits for one
// memory round trip instead of one per dependent access.
// FAST (the FP32 step): the rotation from one reciprocal square root, c = a / r = a rsqrt(r^2)
// and s = b rsqrt(r^2), and the basis scale 1 / hn passed in (rsqrt of the Pythagorean
// square), in place of a square root and divisions, whose FP64 forms are slow on this GPU
// (the close is one thread on the step's critical path); the FP64 step keeps them.
template <int J, bool FAST = false>
__device__ void arnoldi_close_j(DevScalars* sc, const double (&h)[J], double hn, bool weak,
                                double inv_hn = 0.0) {
  constexpr int j = J - 1;
  double cs[J], sn[J];
#pragma unroll
  for (int i = 0; i < j; ++i) {
    cs[i] = sc->cs[i];
    sn[i] = sc->sn[i];
  }
  const double gvj = sc->gv[j], bnorm = sc->bnorm, eta = sc->eta;
  const int m = sc->m, iters = sc->iters, graph = sc->graph;
  const unsigned long long hnext = j + 1 < OTGB_MAXM ? sc->h_step[j + 1] : 0ull;
  double col[J + 1];
#pragma unroll
  for (int i = 0; i < J; ++i) col[i] = h[i];
  col[J] = hn;
#pragma unroll
  for (int i = 0; i < j; ++i) {  // previous rotations on column j
    const double t0 = col[i], t1 = col[i + 1];
    col[i] = cs[i] * t0 + sn[i] * t1;
    col[i + 1] = -sn[i] * t0 + cs[i] * t1;
  }
  const double a = col[j], b = col[j + 1];
  double r, c, sj;
  if (FAST) {
    const double r2 = a * a + b * b;
    const double y = r2 > 0.0 ? rsqrt(r2) : 0.0;
    r = r2 * y;
    c = (r2 > 0.0) ? a * y : 1.0;
    sj = (r2 > 0.0) ? b * y : 0.0;
  } else {
    r = sqrt(a * a + b * b);
    c = (r == 0.0) ? 1.0 : a / r;
    sj = (r == 0.0) ? 0.0 : b / r;
  }
  col[j] = r;
  col[j + 1] = 0.0;
#pragma unroll
  for (int i = 0; i <= J; ++i) sc->H[i * m + j] = col[i];
  sc->cs[j] = c;
  sc->sn[j] = sj;
  const double g1 = -sj * gvj;
  sc->gv[j + 1] = g1;
  sc->gv[j] = c * gvj;
  sc->iters = iters + 1;
  sc->jend = j + 1;
  if (!FAST) sc->relres = fabs(g1) / bnorm;  // informational (the FP32 step skips it)
  int done = 0;
  if (weak) {
    done = 1;
  } else if (fabs(g1) <= eta * bnorm || hn == 0.0) {
    sc->converged = 1;
    done = 1;
  } else {
    sc->scale[j + 1] = FAST ? inv_hn : 1.0 / hn;
    if (j + 1 == m) done = 1;
  }
  if (done) sc->cycle_done = 1;
  sc->j = j + 1;
  if (graph && hnext) cudaGraphSetConditional(hnext, done ? 0u : 1u);
}

}  // namespace otgb
