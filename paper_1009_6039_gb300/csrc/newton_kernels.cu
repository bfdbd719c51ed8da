// Nonlinear residual + linearised coefficients (Eq. ma2, linearmaeq, translation), input
// translation, and the GMRES(m) kernels (Sec. 4.2) of the damped-Newton solver.
//
// Reductions: every block writes its partials to a scratch array; the last block to take
// a ticket reduces them in block order and finalises the scalars in DevScalars.  The
// order is fixed, so results are bit-reproducible from run to run.
#include <math.h>

#include "otgb_internal.cuh"

namespace otgb {

#define RTX 32  // residual tile width (x / columns)
#define RTY 8   // residual tile height (y / rows)

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

// ---------------------------------------------------------------------------------------
// Input translation (Eq. translation applied to both densities, as for the images of
// Sec. 5.2): d <- d - mean(d) + 1; rejects non-finite input or a non-positive result.
// ---------------------------------------------------------------------------------------
__global__ void k_input_stats(const double* __restrict__ f, const double* __restrict__ g,
                              long P, double* partials, DevScalars* sc) {
  double v[6] = {0.0, 0.0, INFINITY, INFINITY, 0.0, 0.0};
  const int kind[6] = {0, 0, 2, 2, 0, 0};
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x) {
    double a = f[p], b = g[p];
    v[0] += a;
    v[1] += b;
    v[2] = fmin(v[2], a);
    v[3] = fmin(v[3], b);
    v[4] += isfinite(a) ? 0.0 : 1.0;
    v[5] += isfinite(b) ? 0.0 : 1.0;
  }
  block_reduce<6>(v, kind);
  if (!publish_partials<6>(v, partials, &sc->ticket[TK_INPUT])) return;
  reduce_partials<6>(v, kind, partials, gridDim.x);
  if (threadIdx.x == 0) {
    sc->in_mean[0] = v[0] / (double)P;
    sc->in_mean[1] = v[1] / (double)P;
    sc->in_min[0] = v[2];
    sc->in_min[1] = v[3];
    sc->in_nonfinite[0] = (int)v[4];
    sc->in_nonfinite[1] = (int)v[5];
    bool bad = v[4] > 0 || v[5] > 0 || !(v[2] - sc->in_mean[0] + 1.0 > 0.0) ||
               !(v[3] - sc->in_mean[1] + 1.0 > 0.0);
    sc->in_bad = bad ? 1 : 0;
    sc->ticket[TK_INPUT] = 0;
  }
}

__global__ void k_input_apply(const double* __restrict__ f, const double* __restrict__ g,
                              double* __restrict__ ft, double* __restrict__ gt, long P,
                              const DevScalars* __restrict__ sc) {
  const double sf = 1.0 - sc->in_mean[0], sg = 1.0 - sc->in_mean[1];
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x) {
    ft[p] = f[p] + sf;
    gt[p] = g[p] + sg;
  }
}

static int reduce_blocks() {
  static int nb = 0;
  if (nb == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    nb = (sms > 0 ? sms : 148) * 2;
  }
  return nb;
}

cudaError_t launch_translate_inputs(const double* f, const double* g, double* ft, double* gt,
                                    int N, int M, double* partials, DevScalars* sc,
                                    cudaStream_t st) {
  const long P = (long)N * M;
  const int nb = reduce_blocks();
  k_input_stats<<<nb, 256, 0, st>>>(f, g, P, partials, sc);
  k_input_apply<<<nb, 256, 0, st>>>(f, g, ft, gt, P, sc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Residual + coefficients (K1).  One thread per grid point of a 32 x 8 tile; u is staged
// in shared memory with a periodic halo of 2 for the 4th-order centred stencils.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int wrapi(int a, int L) {
  int r = a % L;
  return r < 0 ? r + L : r;
}

__device__ __forceinline__ void bspline_w(double t, double w[4], double dw[4]) {
  const double s = 1.0 - t;
  w[0] = s * s * s * (1.0 / 6.0);
  w[1] = (3.0 * t * t * t - 6.0 * t * t + 4.0) * (1.0 / 6.0);
  w[2] = (-3.0 * t * t * t + 3.0 * t * t + 3.0 * t + 1.0) * (1.0 / 6.0);
  w[3] = t * t * t * (1.0 / 6.0);
  dw[0] = -0.5 * s * s;
  dw[1] = 0.5 * (3.0 * t * t - 4.0 * t);
  dw[2] = 0.5 * (-3.0 * t * t + 2.0 * t + 1.0);
  dw[3] = 0.5 * t * t;
}

template <typename T>
__global__ void __launch_bounds__(RTX* RTY)
    k_residual(const double* __restrict__ f, const double* __restrict__ c,
               const double* __restrict__ u, int N, int M, double* __restrict__ Fraw,
               T* __restrict__ coef, double* partials, DevScalars* sc) {
  __shared__ double tile[RTY + 4][RTX + 4];
  const int bx = blockIdx.x * RTX, by = blockIdx.y * RTY;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < (RTY + 4) * (RTX + 4); idx += RTX * RTY) {
    const int r = idx / (RTX + 4), cc = idx % (RTX + 4);
    tile[r][cc] = u[(size_t)wrapi(by + r - 2, N) * M + wrapi(bx + cc - 2, M)];
  }
  __syncthreads();
  const int tx = tid % RTX, ty = tid / RTX;
  const int i = by + ty, j = bx + tx;
  const bool valid = (i < N) && (j < M);
  // partials: sum fn, Simpson sums of a11 a12 a22 b1 b2, max Fraw, min Fraw, min det,
  // non-finite count
  double v[10] = {0, 0, 0, 0, 0, 0, -INFINITY, INFINITY, INFINITY, 0};
  const int kind[10] = {0, 0, 0, 0, 0, 0, 1, 2, 2, 0};
  if (valid) {
    const int r = ty + 2, q = tx + 2;
    const double Mh = (double)M / 12.0, Nh = (double)N / 12.0;
    const double Mh2 = (double)M * (double)M / 12.0, Nh2 = (double)N * (double)N / 12.0;
    const double ux =
        (-tile[r][q + 2] + 8.0 * tile[r][q + 1] - 8.0 * tile[r][q - 1] + tile[r][q - 2]) * Mh;
    const double uy =
        (-tile[r + 2][q] + 8.0 * tile[r + 1][q] - 8.0 * tile[r - 1][q] + tile[r - 2][q]) * Nh;
    const double uxx = (-tile[r][q + 2] + 16.0 * tile[r][q + 1] - 30.0 * tile[r][q] +
                        16.0 * tile[r][q - 1] - tile[r][q - 2]) * Mh2;
    const double uyy = (-tile[r + 2][q] + 16.0 * tile[r + 1][q] - 30.0 * tile[r][q] +
                        16.0 * tile[r - 1][q] - tile[r - 2][q]) * Nh2;
    double dyc[5];
#pragma unroll
    for (int a = -2; a <= 2; ++a)
      dyc[a + 2] = (-tile[r + 2][q + a] + 8.0 * tile[r + 1][q + a] -
                    8.0 * tile[r - 1][q + a] + tile[r - 2][q + a]) * Nh;
    const double uxy = (-dyc[4] + 8.0 * dyc[3] - 8.0 * dyc[1] + dyc[0]) * Mh;
    // g at the displaced point x + grad u, in grid units, periodic cubic B-spline
    const double gxp = (double)j + (double)M * ux, gyp = (double)i + (double)N * uy;
    const double fj = floor(gxp), fi = floor(gyp);
    double wx[4], dwx[4], wy[4], dwy[4];
    bspline_w(gxp - fj, wx, dwx);
    bspline_w(gyp - fi, wy, dwy);
    const int j0 = (int)fj, i0 = (int)fi;
    int jj[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) jj[a] = wrapi(j0 + a - 1, M);
    double G = 0.0, Gx = 0.0, Gy = 0.0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const double* crow = c + (size_t)wrapi(i0 + b - 1, N) * M;
      double sv = 0.0, sd = 0.0;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const double cv = __ldg(crow + jj[a]);
        sv += cv * wx[a];
        sd += cv * dwx[a];
      }
      G += sv * wy[b];
      Gx += sd * wy[b];
      Gy += sv * dwy[b];
    }
    Gx *= (double)M;
    Gy *= (double)N;
    const double det = (1.0 + uxx) * (1.0 + uyy) - uxy * uxy;
    const double fn = G * det;
    const size_t p = (size_t)i * M + j;
    const double fr = f[p] - fn;
    Fraw[p] = fr;
    const double a11 = G * (1.0 + uyy), a12 = -G * uxy, a22 = G * (1.0 + uxx);
    const double b1 = det * Gx, b2 = det * Gy;
    const size_t P = (size_t)N * M;
    coef[p] = (T)a11;
    coef[P + p] = (T)a12;
    coef[2 * P + p] = (T)a22;
    coef[3 * P + p] = (T)b1;
    coef[4 * P + p] = (T)b2;
    const double w = ((i & 1) ? 4.0 : 2.0) / (3.0 * (double)N) * ((j & 1) ? 4.0 : 2.0) /
                     (3.0 * (double)M);
    const bool fin = isfinite(fn);
    v[0] = fin ? fn : 0.0;
    v[1] = w * a11;
    v[2] = w * a12;
    v[3] = w * a22;
    v[4] = w * b1;
    v[5] = w * b2;
    v[6] = fin ? fr : -INFINITY;
    v[7] = fin ? fr : INFINITY;
    v[8] = det;
    v[9] = fin ? 0.0 : 1.0;
  }
  block_reduce<10>(v, kind);
  if (!publish_partials<10>(v, partials, &sc->ticket[TK_RESID])) return;
  const unsigned int nb = gridDim.x * gridDim.y;
  reduce_partials<10>(v, kind, partials, nb);
  if (threadIdx.x == 0) {
    const double P = (double)N * (double)M;
    const double mean_fn = v[0] / P;
    const double shift = mean_fn - 1.0;
    sc->mean_fn = mean_fn;
    sc->shift = shift;
    sc->res_inf = fmax(fabs(v[6] + shift), fabs(v[7] + shift));
    for (int a = 0; a < 5; ++a) sc->abar[a] = v[1 + a];
    sc->min_det = v[8];
    sc->k1_nonfinite = (int)v[9];
    sc->admissible = (v[9] == 0.0 && isfinite(sc->res_inf) && v[8] > 0.0) ? 1 : 0;
    sc->ticket[TK_RESID] = 0;
  }
}

int residual_partial_blocks(int N, int M) {
  return ((M + RTX - 1) / RTX) * ((N + RTY - 1) / RTY);
}

template <typename T>
cudaError_t launch_residual(const double* f, const double* c, const double* u, int N, int M,
                            double* Fraw, T* coef, double* partials, DevScalars* sc,
                            cudaStream_t st) {
  dim3 grid((M + RTX - 1) / RTX, (N + RTY - 1) / RTY);
  k_residual<T><<<grid, RTX * RTY, 0, st>>>(f, c, u, N, M, Fraw, coef, partials, sc);
  return cudaGetLastError();
}

// sum of (Fraw + shift)^2 -> res_l2sum
__global__ void k_residual_l2(const double* __restrict__ Fraw, long P, double* partials,
                              DevScalars* sc) {
  const double s = sc->shift;
  double v[1] = {0.0};
  const int kind[1] = {0};
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x) {
    const double r = Fraw[p] + s;
    v[0] += r * r;
  }
  block_reduce<1>(v, kind);
  if (!publish_partials<1>(v, partials, &sc->ticket[TK_NORM])) return;
  reduce_partials<1>(v, kind, partials, gridDim.x);
  if (threadIdx.x == 0) {
    sc->res_l2sum = v[0];
    sc->ticket[TK_NORM] = 0;
  }
}

cudaError_t launch_residual_l2(const double* Fraw, int N, int M, double* partials,
                               DevScalars* sc, cudaStream_t st) {
  k_residual_l2<<<reduce_blocks(), 256, 0, st>>>(Fraw, (long)N * M, partials, sc);
  return cudaGetLastError();
}

__global__ void k_shifted(const double* __restrict__ Fraw, double* __restrict__ F, long P,
                          const DevScalars* __restrict__ sc) {
  const double s = sc->shift;
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x)
    F[p] = Fraw[p] + s;
}

cudaError_t launch_shifted_residual(const double* Fraw, double* F, int N, int M,
                                    const DevScalars* sc, cudaStream_t st) {
  k_shifted<<<reduce_blocks(), 256, 0, st>>>(Fraw, F, (long)N * M, sc);
  return cudaGetLastError();
}

// mean-zero gauge: u <- u - mean(u) (two launches: sum, then subtract)
__global__ void k_sum(const double* __restrict__ u, long P, double* partials, DevScalars* sc,
                      double* mean_out) {
  double v[1] = {0.0};
  const int kind[1] = {0};
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x)
    v[0] += u[p];
  block_reduce<1>(v, kind);
  if (!publish_partials<1>(v, partials, &sc->ticket[TK_NORM])) return;
  reduce_partials<1>(v, kind, partials, gridDim.x);
  if (threadIdx.x == 0) {
    *mean_out = v[0] / (double)P;
    sc->ticket[TK_NORM] = 0;
  }
}

__global__ void k_sub(double* __restrict__ u, long P, const double* __restrict__ mean) {
  const double m = *mean;
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x)
    u[p] -= m;
}

cudaError_t launch_subtract_mean(double* u, int N, int M, double* partials, DevScalars* sc,
                                 double* mean_out, cudaStream_t st) {
  const int nb = reduce_blocks();
  k_sum<<<nb, 256, 0, st>>>(u, (long)N * M, partials, sc, mean_out);
  k_sub<<<nb, 256, 0, st>>>(u, (long)N * M, mean_out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// GMRES(m) (Sec. 4.2).  The basis V_i is stored unnormalised with v_i = scale[i] V_i so
// that no kernel pass is spent on normalisation.  Arnoldi uses classical Gram-Schmidt:
// one fused multi-dot pass and one fused update pass (which also forms ||w||^2).  The
// Givens rotations and the small triangular solve run in the last block on the device.
// Every kernel returns at once when the current cycle is finished (cycle_done), so a fixed
// sequence of launches can be queued without host round trips.
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void k_gmres_init(const double* __restrict__ Fraw, const T* __restrict__ w,
                             T* __restrict__ V0, long P, int restart, double* partials,
                             DevScalars* sc) {
  const double s = sc->shift, inv_tau = 1.0 / sc->tau;
  double v[1] = {0.0};
  const int kind[1] = {0};
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x) {
    double b = (Fraw[p] + s) * inv_tau;  // h = (f - f~_n) / tau
    if (restart) b -= (double)w[p];
    const T bt = (T)b;
    V0[p] = bt;
    v[0] += (double)bt * (double)bt;
  }
  block_reduce<1>(v, kind);
  if (!publish_partials<1>(v, partials, &sc->ticket[TK_INIT])) return;
  reduce_partials<1>(v, kind, partials, gridDim.x);
  if (threadIdx.x == 0) {
    const double beta = sqrt(v[0]);
    if (!restart) {
      sc->bnorm = beta;
      sc->iters = 0;
      sc->cycles = 0;
      sc->converged = (beta == 0.0);
      sc->relres = 0.0;
    } else {
      sc->relres = sc->bnorm > 0.0 ? beta / sc->bnorm : 0.0;
      if (beta <= sc->eta * sc->bnorm) sc->converged = 1;
    }
    sc->beta = beta;
    sc->j = 0;
    sc->jend = 0;
    sc->cycle_done = sc->converged;
    if (!sc->converged) sc->cycles += 1;
    for (int k = 0; k <= OTGB_MAXM; ++k) sc->gv[k] = 0.0;
    sc->gv[0] = beta;
    sc->scale[0] = beta > 0.0 ? 1.0 / beta : 0.0;
    sc->ticket[TK_INIT] = 0;
  }
}

template <typename T>
__global__ void k_gmres_dots(const T* __restrict__ V, const T* __restrict__ w, long P,
                             double* partials, DevScalars* sc) {
  if (sc->cycle_done) return;
  const int j = sc->j;
  double v[OTGB_MAXM];
  int kind[OTGB_MAXM];
#pragma unroll
  for (int i = 0; i < OTGB_MAXM; ++i) {
    v[i] = 0.0;
    kind[i] = 0;
  }
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x) {
    const double wp = (double)w[p];
#pragma unroll
    for (int i = 0; i < OTGB_MAXM; ++i)
      if (i <= j) v[i] += (double)V[(size_t)i * P + p] * wp;
  }
  block_reduce<OTGB_MAXM>(v, kind);
  if (!publish_partials<OTGB_MAXM>(v, partials, &sc->ticket[TK_DOTS])) return;
  reduce_partials<OTGB_MAXM>(v, kind, partials, gridDim.x);
  if (threadIdx.x == 0) {
    const int m = sc->m;
    for (int i = 0; i <= j; ++i) sc->H[i * m + j] = sc->scale[i] * v[i];
    sc->ticket[TK_DOTS] = 0;
  }
}

template <typename T>
__global__ void k_gmres_update(T* __restrict__ V, const T* __restrict__ w, long P,
                               double* partials, DevScalars* sc) {
  if (sc->cycle_done) return;
  const int j = sc->j, m = sc->m;
  double coefs[OTGB_MAXM];
#pragma unroll
  for (int i = 0; i < OTGB_MAXM; ++i) coefs[i] = (i <= j) ? sc->H[i * m + j] * sc->scale[i] : 0.0;
  T* Vn = V + (size_t)(j + 1) * P;
  double v[1] = {0.0};
  const int kind[1] = {0};
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x) {
    double x = (double)w[p];
#pragma unroll
    for (int i = 0; i < OTGB_MAXM; ++i)
      if (i <= j) x -= coefs[i] * (double)V[(size_t)i * P + p];
    const T xt = (T)x;
    Vn[p] = xt;
    v[0] += (double)xt * (double)xt;
  }
  block_reduce<1>(v, kind);
  if (!publish_partials<1>(v, partials, &sc->ticket[TK_UPDATE])) return;
  reduce_partials<1>(v, kind, partials, gridDim.x);
  if (threadIdx.x == 0) {
    double* H = sc->H;
    const double hn = sqrt(v[0]);
    H[(j + 1) * m + j] = hn;
    for (int i = 0; i < j; ++i) {  // previous rotations on column j
      const double t0 = H[i * m + j], t1 = H[(i + 1) * m + j];
      H[i * m + j] = sc->cs[i] * t0 + sc->sn[i] * t1;
      H[(i + 1) * m + j] = -sc->sn[i] * t0 + sc->cs[i] * t1;
    }
    const double a = H[j * m + j], b = H[(j + 1) * m + j];
    const double r = sqrt(a * a + b * b);
    sc->cs[j] = (r == 0.0) ? 1.0 : a / r;
    sc->sn[j] = (r == 0.0) ? 0.0 : b / r;
    H[j * m + j] = r;
    H[(j + 1) * m + j] = 0.0;
    sc->gv[j + 1] = -sc->sn[j] * sc->gv[j];
    sc->gv[j] = sc->cs[j] * sc->gv[j];
    sc->iters += 1;
    sc->jend = j + 1;
    sc->relres = fabs(sc->gv[j + 1]) / sc->bnorm;
    if (fabs(sc->gv[j + 1]) <= sc->eta * sc->bnorm || hn == 0.0) {
      sc->converged = 1;
      sc->cycle_done = 1;
    } else {
      sc->scale[j + 1] = 1.0 / hn;
      if (j + 1 == m) sc->cycle_done = 1;
    }
    sc->j = j + 1;
    sc->ticket[TK_UPDATE] = 0;
  }
}

// y = R^{-1} g by back substitution (one thread)
__global__ void k_gmres_finish(DevScalars* sc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int n = sc->jend, m = sc->m;
  for (int i = n - 1; i >= 0; --i) {
    double s = sc->gv[i];
    for (int k = i + 1; k < n; ++k) s -= sc->H[i * m + k] * sc->y[k];
    sc->y[i] = s / sc->H[i * m + i];
  }
}

cudaError_t launch_gmres_finish(DevScalars* sc, cudaStream_t st) {
  k_gmres_finish<<<1, 32, 0, st>>>(sc);
  return cudaGetLastError();
}

// sigma += sum_i y_i scale_i V_i
template <typename T>
__global__ void k_gmres_combine(const T* __restrict__ V, T* __restrict__ sigma, long P,
                                const DevScalars* __restrict__ sc) {
  const int n = sc->jend;
  if (n == 0) return;
  double coefs[OTGB_MAXM];
#pragma unroll
  for (int i = 0; i < OTGB_MAXM; ++i) coefs[i] = (i < n) ? sc->y[i] * sc->scale[i] : 0.0;
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x) {
    double x = (double)sigma[p];
#pragma unroll
    for (int i = 0; i < OTGB_MAXM; ++i)
      if (i < n) x += coefs[i] * (double)V[(size_t)i * P + p];
    sigma[p] = (T)x;
  }
}

template <typename T>
cudaError_t launch_gmres_init(const double* Fraw, const T* w, T* V0, long P, int restart,
                              double* partials, DevScalars* sc, int nblocks, cudaStream_t st) {
  k_gmres_init<T><<<nblocks, 256, 0, st>>>(Fraw, w, V0, P, restart, partials, sc);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_gmres_dots(const T* V, const T* w, long P, double* partials, DevScalars* sc,
                              int nblocks, cudaStream_t st) {
  k_gmres_dots<T><<<nblocks, 256, 0, st>>>(V, w, P, partials, sc);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_gmres_update(T* V, const T* w, long P, double* partials, DevScalars* sc,
                                int nblocks, cudaStream_t st) {
  k_gmres_update<T><<<nblocks, 256, 0, st>>>(V, w, P, partials, sc);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_gmres_combine(const T* V, T* sigma, long P, const DevScalars* sc,
                                 int nblocks, cudaStream_t st) {
  k_gmres_combine<T><<<nblocks, 256, 0, st>>>(V, sigma, P, sc);
  return cudaGetLastError();
}

template <typename TI, typename TO>
__global__ void k_convert(const TI* __restrict__ in, TO* __restrict__ out, long n) {
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < n;
       p += (long)gridDim.x * blockDim.x)
    out[p] = (TO)in[p];
}

template <typename T>
cudaError_t launch_convert(const void* in, int in_d, void* out, int out_d, long n,
                           cudaStream_t st) {
  const int nb = reduce_blocks();
  if (in_d && out_d)
    k_convert<double, double><<<nb, 256, 0, st>>>((const double*)in, (double*)out, n);
  else if (in_d)
    k_convert<double, float><<<nb, 256, 0, st>>>((const double*)in, (float*)out, n);
  else if (out_d)
    k_convert<float, double><<<nb, 256, 0, st>>>((const float*)in, (double*)out, n);
  else
    k_convert<float, float><<<nb, 256, 0, st>>>((const float*)in, (float*)out, n);
  return cudaGetLastError();
}

#define OTGB_INST_NEWTON(T)                                                                   \
  template cudaError_t launch_residual<T>(const double*, const double*, const double*, int,   \
                                          int, double*, T*, double*, DevScalars*,             \
                                          cudaStream_t);                                      \
  template cudaError_t launch_gmres_init<T>(const double*, const T*, T*, long, int, double*,  \
                                            DevScalars*, int, cudaStream_t);                  \
  template cudaError_t launch_gmres_dots<T>(const T*, const T*, long, double*, DevScalars*,   \
                                            int, cudaStream_t);                               \
  template cudaError_t launch_gmres_update<T>(T*, const T*, long, double*, DevScalars*, int,  \
                                              cudaStream_t);                                  \
  template cudaError_t launch_gmres_combine<T>(const T*, T*, long, const DevScalars*, int,    \
                                               cudaStream_t);                                 \
  template cudaError_t launch_convert<T>(const void*, int, void*, int, long, cudaStream_t);

OTGB_INST_NEWTON(float)
OTGB_INST_NEWTON(double)

}  // namespace otgb
