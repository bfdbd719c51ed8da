// Nonlinear residual + linearised coefficients (Eq. ma2, linearmaeq, translation), input
// translation, and the GMRES(m) kernels (Sec. 4.2) of the damped-Newton solver.
//
// Reductions: every block writes its partials to a scratch array; the last block to take
// a ticket reduces them in block order and finalises the scalars in DevScalars.  The
// order is fixed, so results are bit-reproducible from run to run.
#include <math.h>
#include <string.h>

#include "dd.cuh"
#include "dd2.cuh"
#include "otgb_internal.cuh"
#include "gmres_dev.cuh"
#include "reduce.cuh"

namespace otgb {

#define RTX 32  // residual tile width (x / columns)
#define RTY 32  // residual tile height (y / rows); 8 warps, 4 rows per thread
#define RPT 4   // rows per thread

// Block sum of NV floats (result valid in thread 0).
template <int NV>
__device__ void block_sum_f(float (&v)[NV]) {
  __shared__ float redf[32][NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int a = 0; a < NV; ++a)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[a] += __shfl_xor_sync(0xffffffffu, v[a], o);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int a = 0; a < NV; ++a) redf[wid][a] = v[a];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      float x = lane < nw ? redf[lane][a] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      v[a] = x;
    }
  }
  __syncthreads();
}

// FP32 sum of NV values over the grid (1-D grid), for the FP32 Krylov vectors of the mixed
// mode: block tree sums, per-block partials, and the last block to take a ticket sums them
// in block order (fixed order: bit-reproducible).  Returns true in that block, with the
// totals in thread 0.  GB300 runs FP32 at ~60x its FP64 rate, and FP64 tree reductions
// (shuffle + add per level) had become a visible part of these short kernels.
template <int NV>
__device__ bool grid_sum_f(float (&v)[NV], double* partials, unsigned int* ticket) {
  __shared__ bool last;
  float* pf = reinterpret_cast<float*>(partials);
  block_sum_f<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) pf[(size_t)blockIdx.x * NV + a] = v[a];
    __threadfence();
    const unsigned int k = atomicAdd(ticket, 1u);
    last = (k == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int a = 0; a < NV; ++a) v[a] = 0.f;
  for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] += ((volatile const float*)pf)[(size_t)b * NV + a];
  block_sum_f<NV>(v);
  return true;
}

// Double-float reductions (dd.cuh) of NV values with kinds 0 sum, 1 max, 2 min, on the FP32
// pipes: the FP64-accuracy grid reductions of the mixed-mode residual.
__device__ __forceinline__ dd dd_combine(dd a, dd b, int kind) {
  if (kind == 0) return dd_add(a, b);
  if (kind == 1) return dd_gt(b, a) ? b : a;
  return dd_gt(a, b) ? b : a;
}
__device__ __forceinline__ dd dd_identity(int kind) {
  return kind == 0 ? dd{0.f, 0.f} : (kind == 1 ? dd{-INFINITY, 0.f} : dd{INFINITY, 0.f});
}
__device__ __forceinline__ dd warp_reduce_dd(dd v, int kind) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const dd w = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = dd_combine(v, w, kind);
  }
  return v;
}
// result valid in thread 0 (all of warp 0)
template <int NV>
__device__ void block_reduce_dd(dd (&v)[NV], const int (&kind)[NV]) {
  __shared__ float2 redd[32][NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int a = 0; a < NV; ++a) v[a] = warp_reduce_dd(v[a], kind[a]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int a = 0; a < NV; ++a) redd[wid][a] = make_float2(v[a].hi, v[a].lo);
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      const dd x = lane < nw ? dd{redd[lane][a].x, redd[lane][a].y} : dd_identity(kind[a]);
      v[a] = warp_reduce_dd(x, kind[a]);
    }
  }
  __syncthreads();
}
// a double as (hi, lo) floats; infinities keep lo = 0
__device__ __forceinline__ dd dd_of_double(double a) {
  const float h = __double2float_rn(a);
  return dd{h, isfinite(h) ? __double2float_rn(a - (double)h) : 0.0f};
}
// grid-wide: per-block (hi, lo) partials, the last block to take a ticket combines them in
// block order; true in that block, totals in thread 0 (2-D grids allowed)
template <int NV>
__device__ bool grid_reduce_dd(dd (&v)[NV], const int (&kind)[NV], double* partials,
                               unsigned int* ticket) {
  __shared__ bool last;
  float2* pf = reinterpret_cast<float2*>(partials);
  const unsigned int nb = gridDim.x * gridDim.y;
  block_reduce_dd<NV>(v, kind);
  if (threadIdx.x == 0) {
    const size_t bid = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
    for (int a = 0; a < NV; ++a) pf[bid * NV + a] = make_float2(v[a].hi, v[a].lo);
    __threadfence();
    const unsigned int k = atomicAdd(ticket, 1u);
    last = (k == nb - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int a = 0; a < NV; ++a) v[a] = dd_identity(kind[a]);
  for (unsigned int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      const volatile float2* q = (const volatile float2*)pf + (size_t)b * NV + a;
      v[a] = dd_combine(v[a], dd{q->x, q->y}, kind[a]);
    }
  block_reduce_dd<NV>(v, kind);
  return true;
}

// ---------------------------------------------------------------------------------------
// Input translation (Eq. translation applied to both densities, as for the images of
// Sec. 5.2): d <- d - mean(d) + 1; rejects non-finite input or a non-positive result.
// ---------------------------------------------------------------------------------------
__global__ void k_input_stats(const double* __restrict__ f, const double* __restrict__ g,
                              long P, double* partials, DevScalars* sc, Bat bat) {
  f = badv(f, bat);
  g = badv(g, bat);
  partials = badv(partials, bat);
  sc = badv(sc, bat);
  if (bskip(sc, bat)) return;
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
  // per-thread FP64, then the block and grid reductions in double-float (FP32 pipes)
  dd r[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) r[a] = dd_of_double(v[a]);
  if (!grid_reduce_dd<6>(r, kind, partials, &sc->ticket[TK_INPUT])) return;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < 6; ++a) v[a] = (double)r[a].hi + (double)r[a].lo;
    sc->in_mean[0] = v[0] / (double)P;
    sc->in_mean[1] = v[1] / (double)P;
    sc->in_min[0] = v[2];
    sc->in_min[1] = v[3];
    sc->in_nonfinite[0] = (int)v[4];
    sc->in_nonfinite[1] = (int)v[5];
    // translated inputs must be positive after the translation, inputs used as given
    // (in_plain) as they are
    const double sf = sc->in_plain ? 0.0 : 1.0 - sc->in_mean[0];
    const double sg = sc->in_plain ? 0.0 : 1.0 - sc->in_mean[1];
    bool bad = v[4] > 0 || v[5] > 0 || !(v[2] + sf > 0.0) || !(v[3] + sg > 0.0);
    sc->in_bad = bad ? 1 : 0;
    sc->ticket[TK_INPUT] = 0;
  }
}

__global__ void k_input_apply(const double* __restrict__ f, const double* __restrict__ g,
                              double* __restrict__ ft, double* __restrict__ gt, long P,
                              const DevScalars* __restrict__ sc, Bat bat) {
  f = badv(f, bat);
  g = badv(g, bat);
  ft = badv(ft, bat);
  gt = badv(gt, bat);
  sc = badv(sc, bat);
  if (bskip(sc, bat)) return;
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

// ---------------------------------------------------------------------------------------
// Cubic B-spline prefilter (Sec. 4, interpolation of g: the coefficients c, with
// (c[k-1] + 4 c[k] + c[k+1]) / 6 = g[k] along each axis, periodic) as recursive filters.
// The periodic inverse of the stencil (1, 4, 1) / 6 is 6 h * with h[k] = z z^|k| / (z^2 - 1),
// z = sqrt(3) - 2 the root of z^2 + 4 z + 1 inside the unit circle (its DTFT is
// 1 / (4 + 2 cos t)), and sum_k z^|k| s[i - k] = cp[i] + ca[i] - s[i] with the first-order
// recursions cp[i] = s[i] + z cp[i - 1] (causal) and ca[i] = s[i] + z ca[i + 1]
// (anticausal).  A thread runs both over a chunk of PRE_CH points of one line, starting each
// from PRE_K periodic terms beyond the chunk (|z|^PRE_K < 1e-22, below FP64 round-off): the
// circular deconvolution to FP64 round-off with a few multiply-adds per point, where the
// spectral form takes three FP64 transform passes.  (256 threads = 32 lines x 8 chunks of
// PRE_CH = 32 points per tile of 256 points.)
// ---------------------------------------------------------------------------------------
constexpr int PRE_K = 40, PRE_CH = 32;

// One axis, tiled: a block stages 32 lines x (256 points + PRE_K on each side, periodic) in
// shared memory with coalesced loads (all of them in flight at once: the recursions
// themselves are short serial chains, so the loads' latency is what a direct version waits
// on), runs the two recursions per thread over a chunk of PRE_CH points of one line, and
// writes the tile back coalesced.  XPASS: lines are rows (points along x), else columns.
// dd_out (optional) also receives the result split as (hi, lo) floats.
constexpr int PT_LN = 32, PT_TP = 256, PT_SW = PT_LN + 1;
constexpr size_t PT_SMEM = (size_t)(PT_TP + 2 * PRE_K) * PT_SW * sizeof(double);

template <bool XPASS>
__global__ void __launch_bounds__(256)
    k_prefilter_tile(const double* __restrict__ s, double* __restrict__ out,
                     float2* __restrict__ dd_out, int N, int M, double z, double A, Bat bat) {
  extern __shared__ __align__(16) double smp[];  // [k][line], k = point - p0 + PRE_K
  s = badv(s, bat);
  out = badv(out, bat);
  dd_out = badv(dd_out, bat);
  const int tid = threadIdx.x;
  const int L = XPASS ? M : N, nlines = XPASS ? N : M;
  const long ls = XPASS ? M : 1, ps = XPASS ? 1 : M;
  const int line0 = blockIdx.x * PT_LN, p0 = blockIdx.y * PT_TP;
  const int tpl = min(PT_TP, L - p0), nk = tpl + 2 * PRE_K;
  // stage (lines fastest for columns, points fastest for rows: both coalesced)
  for (int e = tid; e < nk * PT_LN; e += blockDim.x) {
    const int k = XPASS ? e % nk : e / PT_LN, ln = XPASS ? e / nk : e % PT_LN;
    const int line = line0 + ln;
    const int pt = ((p0 - PRE_K + k) % L + L) % L;
    smp[k * PT_SW + ln] = line < nlines ? s[line * ls + pt * ps] : 0.0;
  }
  __syncthreads();
  const int ln = tid % PT_LN, c0 = (tid / PT_LN) * PRE_CH, n = min(PRE_CH, tpl - c0);
  double v[PRE_CH];
  if (n > 0) {
    double cp = 0.0, ca = 0.0;
    for (int k = c0; k < c0 + PRE_K; ++k) cp = fma(z, cp, smp[k * PT_SW + ln]);
    for (int k = c0 + n + 2 * PRE_K - 1; k >= c0 + n + PRE_K; --k)
      ca = fma(z, ca, smp[k * PT_SW + ln]);
#pragma unroll
    for (int i = 0; i < PRE_CH; ++i)
      if (i < n) {
        cp = fma(z, cp, smp[(c0 + PRE_K + i) * PT_SW + ln]);
        v[i] = cp;
      }
#pragma unroll
    for (int i = PRE_CH - 1; i >= 0; --i)
      if (i < n) {
        const double xi = smp[(c0 + PRE_K + i) * PT_SW + ln];
        ca = fma(z, ca, xi);
        v[i] = A * (v[i] + ca - xi);
      }
  }
  __syncthreads();  // every chunk has read its neighbours' points
  if (n > 0) {
#pragma unroll
    for (int i = 0; i < PRE_CH; ++i)
      if (i < n) smp[(c0 + PRE_K + i) * PT_SW + ln] = v[i];
  }
  __syncthreads();
  for (int e = tid; e < tpl * PT_LN; e += blockDim.x) {
    const int k = XPASS ? e % tpl : e / PT_LN, l2 = XPASS ? e / tpl : e % PT_LN;
    const int line = line0 + l2;
    if (line >= nlines) continue;
    const double r = smp[(k + PRE_K) * PT_SW + l2];
    const long o = line * ls + (long)(p0 + k) * ps;
    out[o] = r;
    if (dd_out) {
      const float hi = __double2float_rn(r);
      dd_out[o] = make_float2(hi, __double2float_rn(r - (double)hi));
    }
  }
}

// The same two passes in double-float arithmetic for the mixed mode (FP64 runs at a small
// fraction of the FP32 rate on this GPU, and the FP64 recursions had become the largest of a
// solve's one-off kernels): the columns' pass reads g in FP64 and leaves the dd result in
// `mid`, the rows' pass reads that and writes c as dd (hi, lo) and as its FP64 sum.  The
// recursions, the chunking and the warm-up length are those of the FP64 kernel; each step
// z cp + s is a dd product and sum (relative error ~2^-47 per step, damped by |z| = 0.27).
template <bool XPASS>
__global__ void __launch_bounds__(256)
    k_prefilter_tile_dd(const double* __restrict__ s64, const float2* __restrict__ sdd,
                        float2* __restrict__ out_dd, double* __restrict__ out64, int N, int M,
                        double z, double A, Bat bat) {
  extern __shared__ __align__(16) float2 smq[];  // [k][line] as (hi, lo)
  s64 = badv(s64, bat);
  sdd = badv(sdd, bat);
  out_dd = badv(out_dd, bat);
  out64 = badv(out64, bat);
  const int tid = threadIdx.x;
  const int L = XPASS ? M : N, nlines = XPASS ? N : M;
  const long ls = XPASS ? M : 1, ps = XPASS ? 1 : M;
  const int line0 = blockIdx.x * PT_LN, p0 = blockIdx.y * PT_TP;
  const int tpl = min(PT_TP, L - p0), nk = tpl + 2 * PRE_K;
  for (int e = tid; e < nk * PT_LN; e += blockDim.x) {
    const int k = XPASS ? e % nk : e / PT_LN, ln = XPASS ? e / nk : e % PT_LN;
    const int line = line0 + ln;
    const int pt = ((p0 - PRE_K + k) % L + L) % L;
    float2 x = make_float2(0.f, 0.f);
    if (line < nlines) {
      const long o = line * ls + pt * ps;
      if (s64) {
        const dd d = dd_from_double(s64[o]);
        x = make_float2(d.hi, d.lo);
      } else {
        x = sdd[o];
      }
    }
    smq[k * PT_SW + ln] = x;
  }
  __syncthreads();
  const dd zd = dd(z), Ad = dd(A);
  const int ln = tid % PT_LN, c0 = (tid / PT_LN) * PRE_CH, n = min(PRE_CH, tpl - c0);
  dd v[PRE_CH];
  auto at = [&](int k) {
    const float2 q = smq[k * PT_SW + ln];
    return dd{q.x, q.y};
  };
  if (n > 0) {
    dd cp{0.f, 0.f}, ca{0.f, 0.f};
    for (int k = c0; k < c0 + PRE_K; ++k) cp = dd_add(dd_mul(zd, cp), at(k));
    for (int k = c0 + n + 2 * PRE_K - 1; k >= c0 + n + PRE_K; --k)
      ca = dd_add(dd_mul(zd, ca), at(k));
#pragma unroll
    for (int i = 0; i < PRE_CH; ++i)
      if (i < n) {
        cp = dd_add(dd_mul(zd, cp), at(c0 + PRE_K + i));
        v[i] = cp;
      }
#pragma unroll
    for (int i = PRE_CH - 1; i >= 0; --i)
      if (i < n) {
        const dd xi = at(c0 + PRE_K + i);
        ca = dd_add(dd_mul(zd, ca), xi);
        v[i] = dd_mul(Ad, dd_sub(dd_add(v[i], ca), xi));
      }
  }
  __syncthreads();  // every chunk has read its neighbours' points
  if (n > 0) {
#pragma unroll
    for (int i = 0; i < PRE_CH; ++i)
      if (i < n) smq[(c0 + PRE_K + i) * PT_SW + ln] = make_float2(v[i].hi, v[i].lo);
  }
  __syncthreads();
  for (int e = tid; e < tpl * PT_LN; e += blockDim.x) {
    const int k = XPASS ? e % tpl : e / PT_LN, l2 = XPASS ? e / tpl : e % PT_LN;
    const int line = line0 + l2;
    if (line >= nlines) continue;
    const float2 r = smq[(k + PRE_K) * PT_SW + l2];
    const long o = line * ls + (long)(p0 + k) * ps;
    out_dd[o] = r;
    if (out64) out64[o] = (double)r.x + (double)r.y;
  }
}

cudaError_t launch_prefilter(const double* g, double* scratch, double* c, float2* cdd, int N,
                             int M, cudaStream_t st, Bat bat) {
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_prefilter_tile<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, PT_SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_prefilter_tile<true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, PT_SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_prefilter_tile_dd<false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, PT_SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_prefilter_tile_dd<true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, PT_SMEM);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  const double z = sqrt(3.0) - 2.0;
  const double A = 6.0 * z / (z * z - 1.0);
  // columns (along y), then rows (along x)
  const dim3 gy((M + PT_LN - 1) / PT_LN, (N + PT_TP - 1) / PT_TP);
  const dim3 gx((N + PT_LN - 1) / PT_LN, (M + PT_TP - 1) / PT_TP);
  if (cdd) {  // mixed mode: double-float passes (the scratch plane holds the dd middle)
    float2* mid = reinterpret_cast<float2*>(scratch);
    k_prefilter_tile_dd<false><<<bgrid(gy, bat), 256, PT_SMEM, st>>>(g, nullptr, mid, nullptr,
                                                                      N, M, z, A, bat);
    k_prefilter_tile_dd<true><<<bgrid(gx, bat), 256, PT_SMEM, st>>>(nullptr, mid, cdd, c, N, M,
                                                                     z, A, bat);
    return cudaGetLastError();
  }
  k_prefilter_tile<false><<<bgrid(gy, bat), 256, PT_SMEM, st>>>(g, scratch, nullptr, N, M, z, A,
                                                                 bat);
  k_prefilter_tile<true><<<bgrid(gx, bat), 256, PT_SMEM, st>>>(scratch, c, cdd, N, M, z, A, bat);
  return cudaGetLastError();
}

cudaError_t launch_input_stats(const double* f, const double* g, int N, int M,
                               double* partials, DevScalars* sc, cudaStream_t st, Bat bat) {
  k_input_stats<<<bgrid(dim3(reduce_blocks()), bat), 256, 0, st>>>(f, g, (long)N * M, partials,
                                                                   sc, bat);
  return cudaGetLastError();
}

// %globaltimer: the GPU's nanosecond clock (PTX special register)
__global__ void k_stamp(DevScalars* sc, int cls) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  const int prev = sc->stamp_cls;
  if (prev >= 0 && prev < PH_COUNT && t > sc->stamp_t) sc->phase_ns[prev] += t - sc->stamp_t;
  if (prev >= 100 && prev < 116 && t > sc->stamp_t) sc->class_ns[prev - 100] += t - sc->stamp_t;
  sc->stamp_t = t;
  sc->stamp_cls = cls;
}

cudaError_t launch_stamp(DevScalars* sc, int cls, cudaStream_t st) {
  k_stamp<<<1, 1, 0, st>>>(sc, cls);
  return cudaGetLastError();
}

cudaError_t launch_translate_inputs(const double* f, const double* g, double* ft, double* gt,
                                    int N, int M, double* partials, DevScalars* sc,
                                    cudaStream_t st, Bat bat) {
  const long P = (long)N * M;
  const dim3 nb = bgrid(dim3(reduce_blocks()), bat);
  k_input_stats<<<nb, 256, 0, st>>>(f, g, P, partials, sc, bat);
  k_input_apply<<<nb, 256, 0, st>>>(f, g, ft, gt, P, sc, bat);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Residual + coefficients (K1).  A block covers a 32 x 32 tile (each thread 4 points, one
// column); u is staged in shared memory with a periodic halo of 2 for the 4th-order
// centred stencils.  GB300's FP64 rate is low, so the kernel avoids FP64 divisions (all
// reciprocal factors come in as arguments), integer divisions in the inner code, and in the
// mixed mode evaluates the gradient of the interpolant (which enters only the Jacobian, not
// the residual) in FP32.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int wrapi(int a, int L) {
  int r = a % L;
  return r < 0 ? r + L : r;
}

__device__ __forceinline__ int wrap_near(int a, int L) {  // a in [-L, 2L)
  return a < 0 ? a + L : (a >= L ? a - L : a);
}

struct ResidConsts {
  double Mh, Nh, Mh2, Nh2;  // M/12, N/12, M^2/12, N^2/12
  double MNh;               // M N / 144
  double w3M, w3N;          // 1/(3M), 1/(3N): Simpson weights (2 or 4) x these
  int nob;                  // 1: the simplified operator (b = 0, Sec. 3.3 remark)
  // interpolation of g (Sec. 4 intro; Sec. 5.2, 5.3): 0 cubic B-spline of the coefficients c;
  // 1 bilinear, 2 nearest node of the grid values (then c = g) and of the grid gradient gx, gy
  int interp;
  const double* gx;
  const double* gy;
};

template <typename G>
__device__ __forceinline__ void bspline_w(G t, G w[4], G dw[4]) {
  const G s = (G)1 - t;
  const G t2 = t * t, t3 = t2 * t;
  const G sixth = (G)(1.0 / 6.0);
  w[0] = s * s * s * sixth;
  w[1] = ((G)3 * t3 - (G)6 * t2 + (G)4) * sixth;
  w[2] = ((G)-3 * t3 + (G)3 * t2 + (G)3 * t + (G)1) * sixth;
  w[3] = t3 * sixth;
  dw[0] = (G)-0.5 * s * s;
  dw[1] = (G)0.5 * ((G)3 * t2 - (G)4 * t);
  dw[2] = (G)0.5 * ((G)-3 * t2 + (G)2 * t + (G)1);
  dw[3] = (G)0.5 * t2;
}

// value weights only; w[2] from the partition of unity sum w = 1
__device__ __forceinline__ void bspline_v(double t, double w[4]) {
  const double s = 1.0 - t;
  const double t2 = t * t, t3 = t2 * t;
  const double sixth = 1.0 / 6.0;
  w[0] = s * s * s * sixth;
  w[1] = fma(0.5, t3, (2.0 / 3.0) - t2);
  w[3] = t3 * sixth;
  w[2] = 1.0 - w[0] - w[1] - w[3];
}

template <typename T>
__global__ void __launch_bounds__(RTX * RTY / RPT)
    k_residual(const double* __restrict__ f, const double* __restrict__ c,
               const float* __restrict__ c32, const double* __restrict__ ua,
               const double* __restrict__ ub, int sel, int N, int M, ResidConsts K,
               double* __restrict__ Fraw, T* __restrict__ coef, double* partials,
               DevScalars* sc) {
  __shared__ double tile[RTY + 4][RTX + 4];
  __shared__ double dyt[RTY][RTX + 4];  // unscaled y-difference of u (halo 2 in x)
  const double* __restrict__ u = (ub && ((sc->upar ^ sel) & 1)) ? ub : ua;
  const int bx = blockIdx.x * RTX, by = blockIdx.y * RTY;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < (RTY + 4) * (RTX + 4); idx += blockDim.x) {
    const int r = idx / (RTX + 4), cc = idx - r * (RTX + 4);
    int gi = by + r - 2, gj = bx + cc - 2;
    while (gi < 0) gi += N;
    while (gi >= N) gi -= N;
    while (gj < 0) gj += M;
    while (gj >= M) gj -= M;
    tile[r][cc] = u[(size_t)gi * M + gj];
  }
  __syncthreads();
  for (int idx = tid; idx < RTY * (RTX + 4); idx += blockDim.x) {
    const int r = idx / (RTX + 4), cc = idx - r * (RTX + 4);
    dyt[r][cc] = -tile[r + 4][cc] + 8.0 * tile[r + 3][cc] - 8.0 * tile[r + 1][cc] + tile[r][cc];
  }
  __syncthreads();
  // FP64 partials: sum fn, max Fraw, min Fraw, min det, non-finite count; Simpson sums of
  // the coefficients (Jacobian only) in the coefficient precision T
  double v64[5] = {0.0, -INFINITY, INFINITY, INFINITY, 0.0};
  const int kind64[5] = {0, 1, 2, 2, 0};
  T simp[5] = {(T)0, (T)0, (T)0, (T)0, (T)0};
  const int tx = tid % RTX, ty0 = tid / RTX;
  const int j = bx + tx;
  const size_t P = (size_t)N * M;
  const T wx = (T)(((j & 1) ? 4.0 : 2.0) * K.w3M);
#pragma unroll 1
  for (int rr = 0; rr < RPT; ++rr) {
    const int ty = ty0 + rr * (RTY / RPT);
    const int i = by + ty;
    if (i >= N || j >= M) continue;
    const int r = ty + 2, q = tx + 2;
    const double ux =
        (-tile[r][q + 2] + 8.0 * tile[r][q + 1] - 8.0 * tile[r][q - 1] + tile[r][q - 2]) * K.Mh;
    const double uy = dyt[ty][q] * K.Nh;
    const double uxx = (-tile[r][q + 2] + 16.0 * tile[r][q + 1] - 30.0 * tile[r][q] +
                        16.0 * tile[r][q - 1] - tile[r][q - 2]) * K.Mh2;
    const double uyy = (-tile[r + 2][q] + 16.0 * tile[r + 1][q] - 30.0 * tile[r][q] +
                        16.0 * tile[r - 1][q] - tile[r - 2][q]) * K.Nh2;
    const double uxy = (-dyt[ty][q + 2] + 8.0 * dyt[ty][q + 1] - 8.0 * dyt[ty][q - 1] +
                        dyt[ty][q - 2]) * K.MNh;
    // g at the displaced point x + grad u, in grid units, periodic cubic B-spline
    const double gxp = (double)j + (double)M * ux, gyp = (double)i + (double)N * uy;
    const double fj = floor(gxp), fi = floor(gyp);
    const double tx_ = gxp - fj, ty_ = gyp - fi;
    const int j0 = wrapi((int)fj, M), i0 = wrapi((int)fi, N);
    int jj[4], ii[4];
    jj[0] = j0 == 0 ? M - 1 : j0 - 1;
    jj[1] = j0;
    jj[2] = wrap_near(j0 + 1, M);
    jj[3] = wrap_near(j0 + 2, M);
    ii[0] = i0 == 0 ? N - 1 : i0 - 1;
    ii[1] = i0;
    ii[2] = wrap_near(i0 + 1, N);
    ii[3] = wrap_near(i0 + 2, N);
    double G = 0.0;
    T Gx, Gy;
    if (K.interp == 2) {  // nearest node (round half up)
      const size_t q = (size_t)wrapi((int)floor(gyp + 0.5), N) * M + wrapi((int)floor(gxp + 0.5), M);
      G = __ldg(c + q);
      Gx = (T)__ldg(K.gx + q);
      Gy = (T)__ldg(K.gy + q);
    } else if (K.interp == 1) {  // bilinear on the cell (i0, j0) .. (i0 + 1, j0 + 1)
      const double w[4] = {(1.0 - tx_) * (1.0 - ty_), tx_ * (1.0 - ty_), (1.0 - tx_) * ty_,
                           tx_ * ty_};
      const size_t q[4] = {(size_t)ii[1] * M + jj[1], (size_t)ii[1] * M + jj[2],
                           (size_t)ii[2] * M + jj[1], (size_t)ii[2] * M + jj[2]};
      double a = 0.0, b = 0.0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        G += w[k] * __ldg(c + q[k]);
        a += w[k] * __ldg(K.gx + q[k]);
        b += w[k] * __ldg(K.gy + q[k]);
      }
      Gx = (T)a;
      Gy = (T)b;
    } else if (sizeof(T) == 8) {
      double wxv[4], dwx[4], wyv[4], dwy[4];
      bspline_w<double>(tx_, wxv, dwx);
      bspline_w<double>(ty_, wyv, dwy);
      double gx = 0.0, gy = 0.0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const double* crow = c + (size_t)ii[b] * M;
        double sv = 0.0, sd = 0.0;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const double cv = __ldg(crow + jj[a]);
          sv += cv * wxv[a];
          sd += cv * dwx[a];
        }
        G += sv * wyv[b];
        gx += sd * wyv[b];
        gy += sv * dwy[b];
      }
      Gx = (T)(gx * (double)M);
      Gy = (T)(gy * (double)N);
    } else {
      // value in FP64 (it enters the residual); gradient (Jacobian only) in FP32 from the
      // FP32 copy of the coefficients
      double wxv[4], wyv[4];
      bspline_v(tx_, wxv);
      bspline_v(ty_, wyv);
      float wxf[4], dwx[4], wyf[4], dwy[4];
      bspline_w<float>((float)tx_, wxf, dwx);
      bspline_w<float>((float)ty_, wyf, dwy);
      float gx = 0.f, gy = 0.f;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const double* crow = c + (size_t)ii[b] * M;
        const float* crow32 = c32 + (size_t)ii[b] * M;
        double sv = 0.0;
        float svf = 0.f, sdf = 0.f;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          sv += __ldg(crow + jj[a]) * wxv[a];
          const float cf = __ldg(crow32 + jj[a]);
          svf += cf * wxf[a];
          sdf += cf * dwx[a];
        }
        G += sv * wyv[b];
        gx += sdf * wyf[b];
        gy += svf * dwy[b];
      }
      Gx = (T)(gx * (float)M);
      Gy = (T)(gy * (float)N);
    }
    const double det = (1.0 + uxx) * (1.0 + uyy) - uxy * uxy;
    const double fn = G * det;
    const size_t p = (size_t)i * M + j;
    const double fr = f[p] - fn;
    Fraw[p] = fr;
    // coefficients of the linearisation (Jacobian only): precision T
    const T Gt = (T)G, dett = (T)det;
    const T a11 = Gt * ((T)1 + (T)uyy), a12 = -Gt * (T)uxy, a22 = Gt * ((T)1 + (T)uxx);
    const T b1 = K.nob ? (T)0 : dett * Gx, b2 = K.nob ? (T)0 : dett * Gy;
    coef[p] = a11;
    coef[P + p] = a12;
    coef[2 * P + p] = a22;
    coef[3 * P + p] = b1;
    coef[4 * P + p] = b2;
    const T w = (T)((i & 1) ? 4.0 : 2.0) * (T)K.w3N * wx;
    simp[0] += w * a11;
    simp[1] += w * a12;
    simp[2] += w * a22;
    simp[3] += w * b1;
    simp[4] += w * b2;
    if (isfinite(fn)) {
      v64[0] += fn;
      v64[1] = fmax(v64[1], fr);
      v64[2] = fmin(v64[2], fr);
    } else {
      v64[4] += 1.0;
    }
    v64[3] = fmin(v64[3], det);
  }
  double v[10];
  const int kind[10] = {0, 0, 0, 0, 0, 0, 1, 2, 2, 0};
  block_reduce<5>(v64, kind64);
  if (sizeof(T) == 8) {
    double sd[5];
    const int k5[5] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int a = 0; a < 5; ++a) sd[a] = (double)simp[a];
    block_reduce<5>(sd, k5);
#pragma unroll
    for (int a = 0; a < 5; ++a) v[1 + a] = sd[a];
  } else {
    float sf[5];
#pragma unroll
    for (int a = 0; a < 5; ++a) sf[a] = (float)simp[a];
    block_sum_f<5>(sf);
#pragma unroll
    for (int a = 0; a < 5; ++a) v[1 + a] = (double)sf[a];
  }
  v[0] = v64[0];
  v[6] = v64[1];
  v[7] = v64[2];
  v[8] = v64[3];
  v[9] = v64[4];
  if (!publish_partials<10>(v, partials, &sc->ticket[TK_RESID])) return;
  const unsigned int nb = gridDim.x * gridDim.y;
  reduce_partials<10>(v, kind, partials, nb);
  if (threadIdx.x == 0) {
    const double Pd = (double)N * (double)M;
    const double mean_fn = v[0] / Pd;
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

// ---------------------------------------------------------------------------------------
// Mixed-mode residual: the same evaluation with every FP64-accuracy quantity (the stencils
// of u, the displaced point, the B-spline value gather, det, f_n and F) in double-float
// arithmetic on the FP32 pipes (dd.cuh, unit round-off 2^-48), the Jacobian coefficients,
// the interpolant's gradient and the Simpson sums in FP32.  Inputs: u (FP64), f and c
// pre-split into (hi, lo) float pairs; output F_raw in FP64.
// ---------------------------------------------------------------------------------------
struct ResidConstsDD {
  dd Mh, Nh, Mh2, Nh2, MNh;  // M/12, N/12, M^2/12, N^2/12, MN/144
  dd inv36;                  // 1/36 (the value weights are computed x6 per axis)
  float M, N;
  float w3M, w3N;            // 1/(3M), 1/(3N)
  int nob;                   // 1: the simplified operator (b = 0)
  int interp;                // as ResidConsts::interp (then cdd = g as (hi, lo) pairs)
  const float* gx;           // grid gradient of g (FP32: the Jacobian only)
  const float* gy;
};

__device__ __forceinline__ dd ldd(const float2* __restrict__ a, size_t i) {
  const float2 v = __ldg(a + i);
  return dd{v.x, v.y};
}

// 6 x the cubic B-spline value weights at t in [0, 1) (taps -1, 0, 1, 2): s^3,
// 3 t^3 - 6 t^2 + 4, 6 - (the other three), t^3, with s = 1 - t; all coefficients exact
__device__ __forceinline__ void bspline6_dd(dd t, dd w[4]) {
  const dd s = dd_add_f(dd_neg(t), 1.0f);
  const dd t2 = dd_mul(t, t), t3 = dd_mul(t2, t);
  w[0] = dd_mul(dd_mul(s, s), s);
  w[1] = dd_add_f(dd_sub(dd_mul_f(t3, 3.0f), dd_mul_f(t2, 6.0f)), 4.0f);
  w[3] = t3;
  w[2] = dd_add_f(dd_neg(dd_add(dd_add(w[0], w[1]), w[3])), 6.0f);
}

// the same weights for two positions at once (t.h, t.l: the lanes' high and low words), each
// lane bit for bit bspline6_dd's
__device__ __forceinline__ void bspline6_dd2(pair::D2 t, pair::D2 w[4]) {
  using namespace pair;
  const u64 one = pk(1.0f, 1.0f);
  // dd_add_f(a, b) = fast_two_sum(s.hi, s.lo + a.lo) with s = two_sum(a.hi, b)
  auto add_f = [](D2 a, u64 b) {
    const D2 s = two_sum2(a.h, b);
    return fast_two_sum2(s.h, add2(s.l, a.l));
  };
  // dd_mul_f(a, b) = fast_two_sum(p, fma(a.lo, b, fma(a.hi, b, -p))) with p = a.hi b
  auto mul_f = [](D2 a, u64 b) {
    const u64 p = mul2(a.h, b);
    u64 e = fma2(a.h, b, neg2(p));
    e = fma2(a.l, b, e);
    return fast_two_sum2(p, e);
  };
  const D2 s = add_f(d2_neg(t), one);
  const D2 t2 = d2_mul(t, t), t3 = d2_mul(t2, t);
  w[0] = d2_mul(d2_mul(s, s), s);
  w[1] = add_f(d2_sub(mul_f(t3, pk(3.0f, 3.0f)), mul_f(t2, pk(6.0f, 6.0f))), pk(4.0f, 4.0f));
  w[3] = t3;
  w[2] = add_f(d2_neg(d2_add(d2_add(w[0], w[1]), w[3])), pk(6.0f, 6.0f));
}

// floor of a dd position p (|p| < 2^23): integer part k and fraction t in [0, 1) as dd.
// p.hi - floor(p.hi) is not exact for -1 < p.hi < 0 (the result needs more bits than
// p.hi), so the subtraction is an error-free dd add.
__device__ __forceinline__ int dd_floor(dd p, dd* t) {
  float fl = floorf(p.hi);
  dd fr = dd_add_f(p, -fl);
  if (fr.hi < 0.0f) {
    fl -= 1.0f;
    fr = dd_add_f(fr, 1.0f);
  } else if (fr.hi >= 1.0f) {
    fl += 1.0f;
    fr = dd_add_f(fr, -1.0f);
  }
  *t = fr;
  return (int)fl;
}

__global__ void __launch_bounds__(RTX * RTY / RPT, 3)
    k_residual_dd(const float2* __restrict__ fdd, const float2* __restrict__ cdd,
                  const double* __restrict__ ua, const double* __restrict__ ub, int sel, int N,
                  int M, ResidConstsDD K, double* __restrict__ Fraw, float* __restrict__ coef,
                  double* partials, DevScalars* sc, Bat bat) {
  __shared__ dd tile[RTY + 4][RTX + 4];
  __shared__ dd dyt[RTY][RTX + 4];  // unscaled y-difference of u (halo 2 in x)
  fdd = badv(fdd, bat);
  cdd = badv(cdd, bat);
  ua = badv(ua, bat);
  ub = badv(ub, bat);
  Fraw = badv(Fraw, bat);
  coef = badv(coef, bat);
  partials = badv(partials, bat);
  sc = badv(sc, bat);
  if (bskip(sc, bat)) return;
  const double* __restrict__ u = (ub && ((sc->upar ^ sel) & 1)) ? ub : ua;
  const int bx = blockIdx.x * RTX, by = blockIdx.y * RTY;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < (RTY + 4) * (RTX + 4); idx += blockDim.x) {
    const int r = idx / (RTX + 4), cc = idx - r * (RTX + 4);
    int gi = by + r - 2, gj = bx + cc - 2;
    while (gi < 0) gi += N;
    while (gi >= N) gi -= N;
    while (gj < 0) gj += M;
    while (gj >= M) gj -= M;
    tile[r][cc] = dd_from_double(u[(size_t)gi * M + gj]);
  }
  __syncthreads();
  for (int idx = tid; idx < RTY * (RTX + 4); idx += blockDim.x) {
    const int r = idx / (RTX + 4), cc = idx - r * (RTX + 4);
    // (u[+2] - u[-2]) is subtracted from 8 (u[+1] - u[-1]), all in y
    dyt[r][cc] = dd_sub(dd_scale2(dd_sub(tile[r + 3][cc], tile[r + 1][cc]), 8.0f),
                        dd_sub(tile[r + 4][cc], tile[r][cc]));
  }
  __syncthreads();
  // partials: sum fn (dd), max Fraw, min Fraw (dd), min det (dd), non-finite count
  dd sum_fn = dd{0.f, 0.f}, fmax_ = dd{-INFINITY, 0.f}, fmin_ = dd{INFINITY, 0.f},
     dmin = dd{INFINITY, 0.f};
  float nonfinite = 0.f;
  float simp[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  const int tx = tid % RTX, ty0 = tid / RTX;
  const int j = bx + tx;
  const size_t P = (size_t)N * M;
  const float wx = ((j & 1) ? 4.0f : 2.0f) * K.w3M;
#pragma unroll 1
  for (int rr = 0; rr < RPT; ++rr) {
    const int ty = ty0 + rr * (RTY / RPT);
    const int i = by + ty;
    if (i >= N || j >= M) continue;
    const int r = ty + 2, q = tx + 2;
    const dd c0 = tile[r][q];
    const dd xp1 = tile[r][q + 1], xm1 = tile[r][q - 1], xp2 = tile[r][q + 2],
             xm2 = tile[r][q - 2];
    const dd ux =
        dd_mul(dd_sub(dd_scale2(dd_sub(xp1, xm1), 8.0f), dd_sub(xp2, xm2)), K.Mh);
    const dd uy = dd_mul(dyt[ty][q], K.Nh);
    // 16 (u[+1] + u[-1]) - (u[+2] + u[-2]) - 30 u
    const dd uxx = dd_mul(dd_sub(dd_sub(dd_scale2(dd_add(xp1, xm1), 16.0f), dd_add(xp2, xm2)),
                                 dd_mul_f(c0, 30.0f)),
                          K.Mh2);
    const dd yp1 = tile[r + 1][q], ym1 = tile[r - 1][q], yp2 = tile[r + 2][q],
             ym2 = tile[r - 2][q];
    const dd uyy = dd_mul(dd_sub(dd_sub(dd_scale2(dd_add(yp1, ym1), 16.0f), dd_add(yp2, ym2)),
                                 dd_mul_f(c0, 30.0f)),
                          K.Nh2);
    const dd uxy = dd_mul(dd_sub(dd_scale2(dd_sub(dyt[ty][q + 1], dyt[ty][q - 1]), 8.0f),
                                 dd_sub(dyt[ty][q + 2], dyt[ty][q - 2])),
                          K.MNh);
    // displaced point in grid units and the periodic cubic B-spline value there
    dd tx_, ty_;
    const int fj = dd_floor(dd_add_f(dd_mul_f(ux, K.M), (float)j), &tx_);
    const int fi = dd_floor(dd_add_f(dd_mul_f(uy, K.N), (float)i), &ty_);
    const int j0 = wrapi(fj, M), i0 = wrapi(fi, N);
    int jj[4], ii[4];
    jj[0] = j0 == 0 ? M - 1 : j0 - 1;
    jj[1] = j0;
    jj[2] = wrap_near(j0 + 1, M);
    jj[3] = wrap_near(j0 + 2, M);
    ii[0] = i0 == 0 ? N - 1 : i0 - 1;
    ii[1] = i0;
    ii[2] = wrap_near(i0 + 1, N);
    ii[3] = wrap_near(i0 + 2, N);
    dd G;
    float Gx, Gy;
    if (K.interp == 2) {  // nearest node (round half up on the fraction)
      const bool upx = tx_.hi > 0.5f || (tx_.hi == 0.5f && tx_.lo >= 0.0f);
      const bool upy = ty_.hi > 0.5f || (ty_.hi == 0.5f && ty_.lo >= 0.0f);
      const int jn = wrapi(fj + (upx ? 1 : 0), M);
      const int in = wrapi(fi + (upy ? 1 : 0), N);
      const size_t q = (size_t)in * M + jn;
      G = ldd(cdd, q);
      Gx = __ldg(K.gx + q);
      Gy = __ldg(K.gy + q);
    } else if (K.interp == 1) {  // bilinear on the cell (i0, j0) .. (i0 + 1, j0 + 1)
      const dd sx = dd_add_f(dd{-tx_.hi, -tx_.lo}, 1.0f), sy = dd_add_f(dd{-ty_.hi, -ty_.lo}, 1.0f);
      const size_t q00 = (size_t)ii[1] * M + jj[1], q01 = (size_t)ii[1] * M + jj[2];
      const size_t q10 = (size_t)ii[2] * M + jj[1], q11 = (size_t)ii[2] * M + jj[2];
      const dd r0 = dd_fma(ldd(cdd, q01), tx_, dd_mul(ldd(cdd, q00), sx));
      const dd r1 = dd_fma(ldd(cdd, q11), tx_, dd_mul(ldd(cdd, q10), sx));
      G = dd_fma(r1, ty_, dd_mul(r0, sy));
      const float ax = tx_.hi, ay = ty_.hi;
      const float w00 = (1.f - ax) * (1.f - ay), w01 = ax * (1.f - ay), w10 = (1.f - ax) * ay,
                  w11 = ax * ay;
      Gx = w00 * __ldg(K.gx + q00) + w01 * __ldg(K.gx + q01) + w10 * __ldg(K.gx + q10) +
           w11 * __ldg(K.gx + q11);
      Gy = w00 * __ldg(K.gy + q00) + w01 * __ldg(K.gy + q01) + w10 * __ldg(K.gy + q10) +
           w11 * __ldg(K.gy + q11);
    } else {
      // packed pairs (dd2.cuh): the x and y value weights in the two lanes of one call, then
      // the 16-tap gather over row pairs (b, b + 2), each lane a row's double-float sum in the
      // scalar order; the two lanes' partial sums of G (rows 0, 1 and rows 2, 3) are added last
      using namespace pair;
      dd wxs[4], wys[4];
      bspline6_dd(tx_, wxs);
      bspline6_dd(ty_, wys);
      D2 wv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) wv[a] = D2{pk(wxs[a].hi, wys[a].hi), pk(wxs[a].lo, wys[a].lo)};
      // gradient weights in FP32 (Jacobian only)
      float wxf[4], dwx[4], wyf[4], dwy[4];
      bspline_w<float>(tx_.hi, wxf, dwx);
      bspline_w<float>(ty_.hi, wyf, dwy);
      D2 G36p{0ull, 0ull};
      u64 gxp = 0ull, gyp = 0ull;
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const size_t ra = (size_t)ii[b] * M, rb = (size_t)ii[b + 2] * M;
        D2 sv{0ull, 0ull};
        u64 svf = 0ull, sdf = 0ull;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const float2 ca = __ldg(cdd + ra + jj[a]), cb = __ldg(cdd + rb + jj[a]);
          const D2 cv{pk(ca.x, cb.x), pk(ca.y, cb.y)};
          float xh, xl, yh, yl;  // the x weight, broadcast to both lanes
          upk(wv[a].h, xh, yh);
          upk(wv[a].l, xl, yl);
          sv = d2_add(d2_mul(cv, D2{pk(xh, xh), pk(xl, xl)}), sv);
          svf = fma2(cv.h, pk(wxf[a], wxf[a]), svf);
          sdf = fma2(cv.h, pk(dwx[a], dwx[a]), sdf);
        }
        float xh0, yh0, xl0, yl0, xh2, yh2, xl2, yl2;  // the y weights of rows b and b + 2
        upk(wv[b].h, xh0, yh0);
        upk(wv[b].l, xl0, yl0);
        upk(wv[b + 2].h, xh2, yh2);
        upk(wv[b + 2].l, xl2, yl2);
        const D2 wyp{pk(yh0, yh2), pk(yl0, yl2)};
        G36p = d2_add(d2_mul(sv, wyp), G36p);
        gxp = fma2(sdf, pk(wyf[b], wyf[b + 2]), gxp);
        gyp = fma2(svf, pk(dwy[b], dwy[b + 2]), gyp);
      }
      dd g01, g23;
      upk(G36p.h, g01.hi, g23.hi);
      upk(G36p.l, g01.lo, g23.lo);
      const dd G36 = dd_add(g01, g23);
      float gx01, gx23, gy01, gy23;
      upk(gxp, gx01, gx23);
      upk(gyp, gy01, gy23);
      G = dd_mul(G36, K.inv36);
      Gx = (gx01 + gx23) * K.M;
      Gy = (gy01 + gy23) * K.N;
    }
    const dd det = dd_sub(dd_mul(dd_add_f(uxx, 1.0f), dd_add_f(uyy, 1.0f)), dd_mul(uxy, uxy));
    const dd fn = dd_mul(G, det);
    const size_t p = (size_t)i * M + j;
    const dd fr = dd_sub(ldd(fdd, p), fn);
    Fraw[p] = dd_to_double(fr);
    // coefficients of the linearisation (Jacobian only), FP32
    const float Gt = G.hi, dett = det.hi;
    const float a11 = Gt * (1.0f + uyy.hi), a12 = -Gt * uxy.hi, a22 = Gt * (1.0f + uxx.hi);
    const float b1 = K.nob ? 0.0f : dett * Gx, b2 = K.nob ? 0.0f : dett * Gy;
    coef[p] = a11;
    coef[P + p] = a12;
    coef[2 * P + p] = a22;
    coef[3 * P + p] = b1;
    coef[4 * P + p] = b2;
    const float w = ((i & 1) ? 4.0f : 2.0f) * K.w3N * wx;
    simp[0] += w * a11;
    simp[1] += w * a12;
    simp[2] += w * a22;
    simp[3] += w * b1;
    simp[4] += w * b2;
    if (isfinite(fn.hi) && isfinite(fn.lo)) {
      sum_fn = dd_add(sum_fn, fn);
      if (dd_gt(fr, fmax_)) fmax_ = fr;
      if (dd_gt(fmin_, fr)) fmin_ = fr;
    } else {
      nonfinite += 1.0f;
    }
    if (dd_gt(dmin, det)) dmin = det;
  }
  // grid reductions in double-float (sum f_n, the five Simpson sums, max F, min F, min det,
  // the non-finite count)
  dd r[10] = {sum_fn,
              dd{simp[0], 0.f},
              dd{simp[1], 0.f},
              dd{simp[2], 0.f},
              dd{simp[3], 0.f},
              dd{simp[4], 0.f},
              fmax_,
              fmin_,
              dmin,
              dd{nonfinite, 0.f}};
  const int kind[10] = {0, 0, 0, 0, 0, 0, 1, 2, 2, 0};
  if (!grid_reduce_dd<10>(r, kind, partials, &sc->ticket[TK_RESID])) return;
  if (threadIdx.x == 0) {
    double v[10];
    for (int a = 0; a < 10; ++a) v[a] = (double)r[a].hi + (double)r[a].lo;
    const double Pd = (double)N * (double)M;
    const double mean_fn = v[0] / Pd;
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

// split FP64 values into (hi, lo) float pairs
__global__ void k_split_dd(const double* __restrict__ in, float2* __restrict__ out, long n,
                           Bat bat) {
  in = badv(in, bat);
  out = badv(out, bat);
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n;
       k += (long)gridDim.x * blockDim.x) {
    const dd v = dd_from_double(in[k]);
    out[k] = make_float2(v.hi, v.lo);
  }
}

cudaError_t launch_split_dd(const double* in, float2* out, long n, cudaStream_t st, Bat bat) {
  long nb = (n + 255) / 256;
  if (nb > 4096) nb = 4096;
  if (nb < 1) nb = 1;
  k_split_dd<<<bgrid(dim3((int)nb), bat), 256, 0, st>>>(in, out, n, bat);
  return cudaGetLastError();
}

static dd host_dd(double v) {
  dd r;
  r.hi = (float)v;
  r.lo = (float)(v - (double)r.hi);
  return r;
}

cudaError_t launch_residual_dd(const float2* fdd, const float2* cdd, const double* ua, int N,
                               int M, double* Fraw, float* coef, double* partials,
                               DevScalars* sc, cudaStream_t st, const double* ub, int sel,
                               int simplified, Bat bat, Interp ip) {
  dim3 grid((M + RTX - 1) / RTX, (N + RTY - 1) / RTY);
  ResidConstsDD K;
  K.Mh = host_dd((double)M / 12.0);
  K.Nh = host_dd((double)N / 12.0);
  K.Mh2 = host_dd((double)M * (double)M / 12.0);
  K.Nh2 = host_dd((double)N * (double)N / 12.0);
  K.MNh = host_dd((double)M * (double)N / 144.0);
  K.inv36 = host_dd(1.0 / 36.0);
  K.M = (float)M;
  K.N = (float)N;
  K.w3M = (float)(1.0 / (3.0 * (double)M));
  K.w3N = (float)(1.0 / (3.0 * (double)N));
  K.nob = simplified ? 1 : 0;
  K.interp = ip.mode;
  K.gx = ip.gx32;
  K.gy = ip.gy32;
  if (ip.mode && !(ip.gx32 && ip.gy32)) return cudaErrorInvalidValue;
  k_residual_dd<<<bgrid(grid, bat), RTX * RTY / RPT, 0, st>>>(fdd, cdd, ua, ub, sel, N, M, K,
                                                                Fraw, coef, partials, sc, bat);
  return cudaGetLastError();
}

int residual_partial_blocks(int N, int M) {
  return ((M + RTX - 1) / RTX) * ((N + RTY - 1) / RTY);
}

template <typename T>
cudaError_t launch_residual(const double* f, const double* c, const double* ua, int N, int M,
                            double* Fraw, T* coef, double* partials, DevScalars* sc,
                            cudaStream_t st, const double* ub, int sel, const float* c32,
                            int simplified, Interp ip) {
  dim3 grid((M + RTX - 1) / RTX, (N + RTY - 1) / RTY);
  ResidConsts K;
  K.Mh = (double)M / 12.0;
  K.Nh = (double)N / 12.0;
  K.Mh2 = (double)M * (double)M / 12.0;
  K.Nh2 = (double)N * (double)N / 12.0;
  K.MNh = K.Mh * K.Nh;
  K.w3M = 1.0 / (3.0 * (double)M);
  K.w3N = 1.0 / (3.0 * (double)N);
  K.nob = simplified ? 1 : 0;
  K.interp = ip.mode;
  K.gx = ip.gx;
  K.gy = ip.gy;
  if (ip.mode && !(ip.gx && ip.gy)) return cudaErrorInvalidValue;
  if (sizeof(T) == 4 && !c32) return cudaErrorInvalidValue;
  k_residual<T><<<grid, RTX * RTY / RPT, 0, st>>>(f, c, c32, ua, ub, sel, N, M, K, Fraw, coef,
                                                  partials, sc);
  return cudaGetLastError();
}

// sum of (Fraw + shift)^2 -> res_l2sum
__global__ void k_residual_l2(const double* __restrict__ Fraw, long P, double* partials,
                              DevScalars* sc, Bat bat) {
  Fraw = badv(Fraw, bat);
  partials = badv(partials, bat);
  sc = badv(sc, bat);
  if (bskip(sc, bat)) return;
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
                               DevScalars* sc, cudaStream_t st, Bat bat) {
  k_residual_l2<<<bgrid(dim3(reduce_blocks()), bat), 256, 0, st>>>(Fraw, (long)N * M, partials,
                                                                   sc, bat);
  return cudaGetLastError();
}

__global__ void k_shifted(const double* __restrict__ Fraw, double* __restrict__ F, long P,
                          const DevScalars* __restrict__ sc) {
  const double s = sc->shift;
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x)
    F[p] = Fraw[p] + s;
}

// in-place form (F += shift): one pointer, so no aliasing of restrict-qualified arguments
__global__ void k_shift_inplace(double* F, long P, const DevScalars* __restrict__ sc) {
  const double s = sc->shift;
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x)
    F[p] += s;
}

cudaError_t launch_shifted_residual(const double* Fraw, double* F, int N, int M,
                                    const DevScalars* sc, cudaStream_t st) {
  if (Fraw == F)
    k_shift_inplace<<<reduce_blocks(), 256, 0, st>>>(F, (long)N * M, sc);
  else
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
                             DevScalars* sc, T* __restrict__ sigma, Bat bat) {
  Fraw = badv(Fraw, bat);
  w = badv(w, bat);
  V0 = badv(V0, bat);
  partials = badv(partials, bat);
  sc = badv(sc, bat);
  sigma = badv(sigma, bat);
  if (bskip(sc, bat)) return;
  const double s = sc->shift, inv_tau = 1.0 / sc->tau;
  double v[1] = {0.0};
  const int kind[1] = {0};
  T acc = (T)0;
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x) {
    if (sigma) sigma[p] = (T)0;
    T bt;
    if constexpr (sizeof(T) == 4) {
      // the shifted residual in FP64 (one add), the rest in the vector precision
      float b = __double2float_rn(Fraw[p] + s) * (float)inv_tau;  // h = (f - f~_n) / tau
      if (restart) b -= w[p];
      bt = b;
    } else {
      double b = (Fraw[p] + s) * inv_tau;
      if (restart) b -= (double)w[p];
      bt = (T)b;
    }
    V0[p] = bt;
    acc += bt * bt;
  }
  if constexpr (sizeof(T) == 4) {
    float a[1] = {acc};
    if (!grid_sum_f<1>(a, partials, &sc->ticket[TK_INIT])) return;
    v[0] = (double)a[0];
  } else {
    v[0] = (double)acc;
    block_reduce<1>(v, kind);
    if (!publish_partials<1>(v, partials, &sc->ticket[TK_INIT])) return;
    reduce_partials<1>(v, kind, partials, gridDim.x);
  }
  if (threadIdx.x == 0) {
    const double beta = sqrt(v[0]);
    if (!restart) {
      // a new Newton step: the last residual evaluated was the current iterate's
      for (int a = 0; a < 5; ++a) sc->abar_n[a] = sc->abar[a];
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

// 16-byte vector access to the Krylov vectors (float4 / double2): when P is a multiple of
// the width every vector V_i = V + i P stays 16-byte aligned and the loops run over whole
// vectors (the loop over q below), else element by element (the tail loop covers all).
template <typename T> struct Vec16;
template <> struct Vec16<float> {
  using type = float4;
  static constexpr int W = 4;
};
template <> struct Vec16<double> {
  using type = double2;
  static constexpr int W = 2;
};
template <typename T>
__device__ __forceinline__ void vld(const T* __restrict__ base, long q, T (&x)[Vec16<T>::W]) {
  const typename Vec16<T>::type v = reinterpret_cast<const typename Vec16<T>::type*>(base)[q];
  memcpy(x, &v, sizeof(v));
}
template <typename T>
__device__ __forceinline__ void vst(T* __restrict__ base, long q, const T (&x)[Vec16<T>::W]) {
  typename Vec16<T>::type v;
  memcpy(&v, x, sizeof(v));
  reinterpret_cast<typename Vec16<T>::type*>(base)[q] = v;
}
// number of whole vectors of the 16-byte loops (0: element loop only)
__device__ __forceinline__ long nvec(long P, int W) { return P % W == 0 ? P / W : 0; }

// Close Arnoldi step j (one thread): H(j+1, j) = hn, the previous Givens rotations and a new
// one on column j, the residual estimate |g_(j+1)|, convergence / end of cycle, v_(j+1) =
// w / hn, and the conditional handle of step j + 1.  weak: hn came out below the resolution
// of the Pythagorean norm; the cycle ends without a convergence claim (the restart
// recomputes the residual explicitly).
__device__ void arnoldi_close(DevScalars* sc, int j, double hn, bool weak) {
  double* H = sc->H;
  const int m = sc->m;
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
  if (weak) {
    sc->cycle_done = 1;
  } else if (fabs(sc->gv[j + 1]) <= sc->eta * sc->bnorm || hn == 0.0) {
    sc->converged = 1;
    sc->cycle_done = 1;
  } else {
    sc->scale[j + 1] = 1.0 / hn;
    if (j + 1 == m) sc->cycle_done = 1;
  }
  sc->j = j + 1;
  // the handle of step j + 1 (the tail WHILE of the captured cycle for j + 1 >= its plain
  // steps, including j + 1 = m, where the cycle is done and the loop ends)
  if (sc->graph && j + 1 < OTGB_MAXM && sc->h_step[j + 1])
    cudaGraphSetConditional(sc->h_step[j + 1], sc->cycle_done ? 0u : 1u);
}

// Per-thread partial sums are kept in the vector precision T (a thread covers a few vectors
// of 16 bytes); partials are combined across threads and blocks in FP64.
template <typename T, int J>
__device__ __forceinline__ void dots_j(const T* __restrict__ V, const T* __restrict__ w, long P,
                                       double* partials, DevScalars* sc, int pass,
                                       bool split) {
  constexpr int W = Vec16<T>::W;
  T acc[J + 1];  // V_i . w (i < J) and w . w
#pragma unroll
  for (int i = 0; i <= J; ++i) acc[i] = (T)0;
  const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const long nth = (long)gridDim.x * blockDim.x, PV = nvec(P, W);
  for (long q = tid; q < PV; q += nth) {
    T wv[W];
    vld<T>(w, q, wv);
#pragma unroll
    for (int i = 0; i < J; ++i) {
      T x[W];
      vld<T>(V + (size_t)i * P, q, x);
#pragma unroll
      for (int k = 0; k < W; ++k) acc[i] += x[k] * wv[k];
    }
#pragma unroll
    for (int k = 0; k < W; ++k) acc[J] += wv[k] * wv[k];
  }
  for (long p = PV * W + tid; p < P; p += nth) {
    const T wp = w[p];
#pragma unroll
    for (int i = 0; i < J; ++i) acc[i] += V[(size_t)i * P + p] * wp;
    acc[J] += wp * wp;
  }
  double v[J + 1];
  if constexpr (sizeof(T) == 4) {
    if (split && pass == 0 && !sc->reorth) {
      // single-reduction step in FP32 (split): the block's sums go to its partials and the
      // update kernel finishes the step (every block of it sums the partials in the same
      // order; its block 0 closes the step) -- no last-block pass and no serial close here
      block_sum_f<J + 1>(acc);
      if (threadIdx.x == 0) {
        float* pf = reinterpret_cast<float*>(partials);
#pragma unroll
        for (int a = 0; a <= J; ++a) pf[(size_t)blockIdx.x * (J + 1) + a] = acc[a];
        if (blockIdx.x == 0) sc->jd = J - 1;
      }
      return;
    }
    if (!grid_sum_f<J + 1>(acc, partials, &sc->ticket[TK_DOTS])) return;
#pragma unroll
    for (int i = 0; i <= J; ++i) v[i] = (double)acc[i];
  } else {
    int kind[J + 1];
#pragma unroll
    for (int i = 0; i <= J; ++i) {
      v[i] = (double)acc[i];
      kind[i] = 0;
    }
    block_reduce<J + 1>(v, kind);
    if (!publish_partials<J + 1>(v, partials, &sc->ticket[TK_DOTS])) return;
    reduce_partials<J + 1>(v, kind, partials, gridDim.x);
  }
  if (threadIdx.x == 0) {
    const int m = sc->m, j = J - 1;
    if (pass == 0 && !sc->reorth) {
      // one reduction per Arnoldi step: with v_i orthonormal, ||w - sum h_i v_i||^2 =
      // ||w||^2 - sum h_i^2 (Pythagoras), so the norm and the Givens rotation finish here
      // and the update of w is a plain elementwise pass (mode 3) that ends no reduction.
      // The difference loses accuracy when w lies almost in span(v_0..v_j); below 1e-6
      // ||w||^2 (the FP32 sums' resolution) the cycle ends and the restart's explicit
      // residual decides.
      double h[J], hs = 0.0;
#pragma unroll
      for (int i = 0; i < J; ++i) h[i] = sc->scale[i] * v[i];
#pragma unroll
      for (int i = 0; i < J; ++i) {
        sc->hcol[i] = h[i];
        hs += h[i] * h[i];
      }
      const double ww = v[J], hn2 = ww - hs;
      const bool weak = !(hn2 > 1e-6 * ww);
      arnoldi_close_j<J>(sc, h, weak ? 0.0 : sqrt(hn2), weak);
    } else if (pass == 0) {
#pragma unroll
      for (int i = 0; i < J; ++i) sc->H[i * m + j] = sc->scale[i] * v[i];
    } else {
#pragma unroll
      for (int i = 0; i < J; ++i) {
        sc->h2[i] = sc->scale[i] * v[i];
        sc->H[i * m + j] += sc->h2[i];
      }
    }
    sc->ticket[TK_DOTS] = 0;
  }
}

template <typename T>
__global__ void k_gmres_dots(const T* __restrict__ V, const T* __restrict__ w, long P,
                             double* partials, DevScalars* sc, int pass, Bat bat) {
  V = badv(V, bat);
  w = badv(w, bat);
  partials = badv(partials, bat);
  sc = badv(sc, bat);
  if (bskip(sc, bat) || sc->cycle_done) return;
  if (pass) w = V + (size_t)(sc->j + 1) * P;
  // the split step (close in the update) serves single problems; a plan set's classes keep
  // the close in the multi-dot's last block (measured faster for their small per-pair grids)
  const bool split = !bat.on;
  switch (sc->j) {
#define OTGB_DOTS_CASE(k) \
  case k:                 \
    dots_j<T, k + 1>(V, w, P, partials, sc, pass, split); break;
    OTGB_DOTS_CASE(0) OTGB_DOTS_CASE(1) OTGB_DOTS_CASE(2) OTGB_DOTS_CASE(3)
    OTGB_DOTS_CASE(4) OTGB_DOTS_CASE(5) OTGB_DOTS_CASE(6) OTGB_DOTS_CASE(7)
    OTGB_DOTS_CASE(8) OTGB_DOTS_CASE(9) OTGB_DOTS_CASE(10) OTGB_DOTS_CASE(11)
    OTGB_DOTS_CASE(12) OTGB_DOTS_CASE(13) OTGB_DOTS_CASE(14)
#undef OTGB_DOTS_CASE
  }
}

template <typename T, int J>
__device__ __forceinline__ void update_j(T* __restrict__ V, const T* __restrict__ w, long P,
                                         double* partials, DevScalars* sc, int mode,
                                         bool split) {
  const int j = J - 1, m = sc->m;
  T coefs[J];
  double hv[J], hn = 0.0, inv_hn = 0.0;
  bool weak = false;
  if (sizeof(T) == 4 && mode == 3 && split) {
    float cf[J];
    finish_multidot_f32<J>(partials, gridDim.x, sc, hv, hn, inv_hn, weak, cf);
#pragma unroll
    for (int i = 0; i < J; ++i) coefs[i] = (T)cf[i];
  } else {
#pragma unroll
    for (int i = 0; i < J; ++i)
      coefs[i] = (T)((mode == 2 ? sc->h2[i] : (mode == 3 ? sc->hcol[i] : sc->H[i * m + j])) *
                     sc->scale[i]);
  }
  T* Vn = V + (size_t)(j + 1) * P;
  const T* src = (mode == 2) ? Vn : w;
  T acc = (T)0;
  constexpr int W = Vec16<T>::W;
  // FP32 mode 3: block 0 closes the step (one thread's serial FP64 work and round trips)
  // while the other blocks form v_(j+1); otherwise every block takes part
  const bool closer = sizeof(T) == 4 && mode == 3 && split && gridDim.x > 1;
  if (closer && blockIdx.x == 0) {
    if (threadIdx.x == 0) {
#pragma unroll
      for (int i = 0; i < J; ++i) sc->hcol[i] = hv[i];
      arnoldi_close_j<J, true>(sc, hv, hn, weak, inv_hn);
    }
    return;
  }
  const long bid = closer ? blockIdx.x - 1 : blockIdx.x, nbk = closer ? gridDim.x - 1 : gridDim.x;
  const long tid = bid * (long)blockDim.x + threadIdx.x;
  const long nth = nbk * blockDim.x, PV = nvec(P, W);
  for (long q = tid; q < PV; q += nth) {
    T x[W];
    vld<T>(src, q, x);
#pragma unroll
    for (int i = 0; i < J; ++i) {
      T y[W];
      vld<T>(V + (size_t)i * P, q, y);
#pragma unroll
      for (int k = 0; k < W; ++k) x[k] -= coefs[i] * y[k];
    }
    vst<T>(Vn, q, x);
#pragma unroll
    for (int k = 0; k < W; ++k) acc += x[k] * x[k];
  }
  for (long p = PV * W + tid; p < P; p += nth) {
    T x = src[p];
#pragma unroll
    for (int i = 0; i < J; ++i) x -= coefs[i] * V[(size_t)i * P + p];
    Vn[p] = x;
    acc += x * x;
  }
  // mode 1: first of two passes, the norm follows the second; mode 3: the step was closed
  // by block 0 above (FP32) or by the multi-dot (FP64)
  if (mode == 1 || mode == 3) {
    if (sizeof(T) == 4 && mode == 3 && split && !closer && blockIdx.x == 0 &&
        threadIdx.x == 0) {
#pragma unroll
      for (int i = 0; i < J; ++i) sc->hcol[i] = hv[i];
      arnoldi_close_j<J, true>(sc, hv, hn, weak, inv_hn);
    }
    return;
  }
  double v[1] = {(double)acc};
  if constexpr (sizeof(T) == 4) {
    float a[1] = {acc};
    if (!grid_sum_f<1>(a, partials, &sc->ticket[TK_UPDATE])) return;
    v[0] = (double)a[0];
  } else {
    const int kind[1] = {0};
    block_reduce<1>(v, kind);
    if (!publish_partials<1>(v, partials, &sc->ticket[TK_UPDATE])) return;
    reduce_partials<1>(v, kind, partials, gridDim.x);
  }
  if (threadIdx.x == 0) {
    arnoldi_close(sc, j, sqrt(v[0]), false);
    sc->ticket[TK_UPDATE] = 0;
  }
}

template <typename T>
__global__ void k_gmres_update(T* __restrict__ V, const T* __restrict__ w, long P,
                               double* partials, DevScalars* sc, int mode, Bat bat) {
  V = badv(V, bat);
  w = badv(w, bat);
  partials = badv(partials, bat);
  sc = badv(sc, bat);
  if (bskip(sc, bat) || sc->cycle_done) return;
  // mode 3 follows the multi-dot of step jd (FP32, single problem: the update closes the
  // step itself and advances sc->j, so it reads the step from jd; FP64 and plan-set classes:
  // the multi-dot closed it and advanced sc->j)
  const bool split = sizeof(T) == 4 && !bat.on;
  switch (mode == 3 ? (split ? sc->jd : sc->j - 1) : sc->j) {
#define OTGB_UPD_CASE(k) \
  case k:                \
    update_j<T, k + 1>(V, w, P, partials, sc, mode, split); break;
    OTGB_UPD_CASE(0) OTGB_UPD_CASE(1) OTGB_UPD_CASE(2) OTGB_UPD_CASE(3)
    OTGB_UPD_CASE(4) OTGB_UPD_CASE(5) OTGB_UPD_CASE(6) OTGB_UPD_CASE(7)
    OTGB_UPD_CASE(8) OTGB_UPD_CASE(9) OTGB_UPD_CASE(10) OTGB_UPD_CASE(11)
    OTGB_UPD_CASE(12) OTGB_UPD_CASE(13) OTGB_UPD_CASE(14)
#undef OTGB_UPD_CASE
  }
}

// y = R^{-1} g by back substitution: the 32 threads stage R and g in shared memory (one
// round of independent loads), thread 0 solves there
__global__ void k_gmres_finish(DevScalars* sc, Bat bat) {
  __shared__ double R[OTGB_MAXM * OTGB_MAXM], g[OTGB_MAXM], y[OTGB_MAXM];
  sc = badv(sc, bat);
  if (blockIdx.x != 0 || bskip(sc, bat)) return;
  const int n = sc->jend, m = sc->m;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) R[e] = sc->H[(e / n) * m + e % n];
  for (int e = threadIdx.x; e < n; e += blockDim.x) g[e] = sc->gv[e];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = n - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < n; ++k) s -= R[i * n + k] * y[k];
      y[i] = s / R[i * n + i];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += blockDim.x) sc->y[e] = y[e];
}

cudaError_t launch_gmres_finish(DevScalars* sc, cudaStream_t st, Bat bat) {
  k_gmres_finish<<<bgrid(dim3(1), bat), 32, 0, st>>>(sc, bat);
  return cudaGetLastError();
}

// sigma += sum_i y_i scale_i V_i
template <typename T, int J>
__device__ __forceinline__ void combine_j(const T* __restrict__ V, T* __restrict__ sigma, long P,
                                          const DevScalars* __restrict__ sc) {
  T coefs[J];
#pragma unroll
  for (int i = 0; i < J; ++i) coefs[i] = (T)(sc->y[i] * sc->scale[i]);
  constexpr int W = Vec16<T>::W;
  const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const long nth = (long)gridDim.x * blockDim.x, PV = nvec(P, W);
  for (long q = tid; q < PV; q += nth) {
    T x[W];
    vld<T>(sigma, q, x);
#pragma unroll
    for (int i = 0; i < J; ++i) {
      T y[W];
      vld<T>(V + (size_t)i * P, q, y);
#pragma unroll
      for (int k = 0; k < W; ++k) x[k] += coefs[i] * y[k];
    }
    vst<T>(sigma, q, x);
  }
  for (long p = PV * W + tid; p < P; p += nth) {
    T x = sigma[p];
#pragma unroll
    for (int i = 0; i < J; ++i) x += coefs[i] * V[(size_t)i * P + p];
    sigma[p] = x;
  }
}

template <typename T>
__global__ void k_gmres_combine(const T* __restrict__ V, T* __restrict__ sigma, long P,
                                const DevScalars* __restrict__ sc, Bat bat) {
  V = badv(V, bat);
  sigma = badv(sigma, bat);
  sc = badv(sc, bat);
  if (bskip(sc, bat)) return;
  switch (sc->jend) {
#define OTGB_CMB_CASE(k) \
  case k:                \
    combine_j<T, k>(V, sigma, P, sc); break;
    OTGB_CMB_CASE(1) OTGB_CMB_CASE(2) OTGB_CMB_CASE(3) OTGB_CMB_CASE(4)
    OTGB_CMB_CASE(5) OTGB_CMB_CASE(6) OTGB_CMB_CASE(7) OTGB_CMB_CASE(8)
    OTGB_CMB_CASE(9) OTGB_CMB_CASE(10) OTGB_CMB_CASE(11) OTGB_CMB_CASE(12)
    OTGB_CMB_CASE(13) OTGB_CMB_CASE(14) OTGB_CMB_CASE(15)
#undef OTGB_CMB_CASE
    default: break;
  }
}

template <typename T>
cudaError_t launch_gmres_init(const double* Fraw, const T* w, T* V0, long P, int restart,
                              double* partials, DevScalars* sc, int nblocks, cudaStream_t st,
                              T* sigma, Bat bat) {
  k_gmres_init<T><<<bgrid(dim3(nblocks), bat), 256, 0, st>>>(Fraw, w, V0, P, restart, partials,
                                                             sc, sigma, bat);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_gmres_dots(const T* V, const T* w, long P, double* partials, DevScalars* sc,
                              int nblocks, cudaStream_t st, int pass, Bat bat) {
  k_gmres_dots<T><<<bgrid(dim3(nblocks), bat), 256, 0, st>>>(V, w, P, partials, sc, pass, bat);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_gmres_update(T* V, const T* w, long P, double* partials, DevScalars* sc,
                                int nblocks, cudaStream_t st, int mode, Bat bat) {
  k_gmres_update<T><<<bgrid(dim3(nblocks), bat), 256, 0, st>>>(V, w, P, partials, sc, mode,
                                                               bat);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_gmres_combine(const T* V, T* sigma, long P, const DevScalars* sc,
                                 int nblocks, cudaStream_t st, Bat bat) {
  k_gmres_combine<T><<<bgrid(dim3(nblocks), bat), 256, 0, st>>>(V, sigma, P, sc, bat);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Device-resident Newton control (Eq. linma with the convexity safeguard), one thread.
// Mirrors the host loop: stop tests before each solve, step halving on an inadmissible
// candidate, s doubled (capped at 1) after an accepted step.
// ---------------------------------------------------------------------------------------
#define OT_STATUS_OK 0
#define OT_STATUS_EINVAL (-1)
#define OT_STATUS_ENOCONV (-2)
#define OT_STATUS_EDIVERGED (-3)

__device__ __forceinline__ void set_cond(const DevScalars* sc, unsigned long long h,
                                         unsigned int v) {
  if (sc->graph && h) cudaGraphSetConditional(h, v);
}

// One control operation on one problem's scalars.  handles = 0: a batched solve, whose
// conditional handles are set once for all pairs by k_ctl_batch (and whose Arnoldi steps are
// not conditional); the return value is what the operation's handle would receive.
__device__ int ctl_apply(int op, DevScalars* sc, int add, bool handles) {
  sc->kcount += add;
  int cont = 0;
  switch (op) {
    case CTL_NEWTON: {
      // tau schedule: the damping drops to 1 for good once max|F| < tau_switch
      if (sc->tau_switch > 0.0 && sc->res_inf < sc->tau_switch) sc->tau = 1.0;
      if (sc->in_bad) {
        sc->status = OT_STATUS_EINVAL;
      } else if (!sc->admissible) {
        sc->status = OT_STATUS_EDIVERGED;
      } else if (sc->res_inf < sc->tol) {
        sc->status = OT_STATUS_OK;
      } else if (sc->newton_n >= sc->max_newton) {
        sc->status = OT_STATUS_ENOCONV;
      } else {
        sc->status = OT_STATUS_OK;
        cont = 1;
      }
      sc->active = cont;
      if (handles) set_cond(sc, sc->h_newton, cont);
      break;
    }
    case CTL_ACCEPT: {
      const double s = sc->step_s;
      if (!sc->safeguard || sc->admissible || s < 0x1p-30) {
        sc->upar ^= 1;
        sc->newton_n += 1;
        sc->step_s = (2.0 * s < 1.0) ? 2.0 * s : 1.0;
      } else {
        sc->step_s = 0.5 * s;
        sc->halvings += 1;
        cont = 1;
      }
      sc->halve = cont;
      if (handles) set_cond(sc, sc->h_halve, cont);
      break;
    }
    case CTL_PRE_CYCLE:
      cont = sc->converged ? 0 : 1;
      sc->in_cycle = cont;
      if (handles) set_cond(sc, sc->h_cycle, cont);
      break;
    case CTL_CYCLE_BEGIN:
      if (handles) {
        for (int k = 1; k < sc->m; ++k) set_cond(sc, sc->h_step[k], 0);
        set_cond(sc, sc->h_step[0], sc->converged ? 0u : 1u);
      }
      break;
    case CTL_CYCLE_END: {
      // the unconditional Arnoldi steps a short cycle left also launched (and skipped)
      if (handles && sc->jend < sc->steps_uncond)
        sc->kcount += (long long)sc->step_kernels * (sc->steps_uncond - sc->jend);
      cont = (!sc->converged && sc->cycles < sc->max_restarts) ? 1 : 0;
      sc->in_cycle = cont;
      if (handles) {
        set_cond(sc, sc->h_cycle, cont);
        set_cond(sc, sc->h_restart, cont);
        if (cont) sc->kcount += 4;  // restart residual: 3 matvec passes + init
      }
      break;
    }
    case CTL_FORCING:
      // Eisenstat & Walker (1996), choice 2 with gamma = 0.9, alpha = 2: eta = gamma
      // (|F_k| / |F_k-1|)^2, kept >= gamma eta_prev^2 when that exceeds 0.1, at most eta_max;
      // and no tighter than needed to reach the Newton tolerance (0.5 tol / |F_k|)
      if (sc->forcing) {
        const double r = sc->res_inf, rp = sc->res_prev;
        double e = sc->eta_max;
        if (rp > 0.0) {
          const double q = r / rp;
          e = 0.9 * q * q;
          const double sg = 0.9 * sc->eta * sc->eta;
          if (sg > 0.1) e = fmax(e, sg);
          e = fmin(e, sc->eta_max);
        }
        e = fmax(e, fmin(sc->eta_max, 0.5 * sc->tol / r));
        e = fmax(e, 1e-6);
        sc->eta = e;
        sc->res_prev = r;
      }
      break;
    case CTL_GMRES_DONE:
      // Arnoldi steps: 3 matvec passes + dots + update (+ dots + update when reorthogonal.;
      // the fused update carries the next step's first matvec pass)
      if (handles) sc->kcount += (long long)sc->step_kernels * sc->iters;
      sc->gmres_iters_total += sc->iters;
      sc->gmres_cycles_total += sc->cycles;
      break;
  }
  return cont;
}

__global__ void k_ctl(int op, DevScalars* sc, int add) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  ctl_apply(op, sc, add, true);
}

// The same operation for every pair of a batched solve the mask selects (one thread per
// pair), then the operation's conditional handle set to "any pair continues".  Kernel
// launches are counted on pair 0 (the launches are shared by the pairs).
__global__ void k_ctl_batch(int op, DevScalars* sc, int add, Bat bat) {
  int cont = 0;
  const int b = threadIdx.x;
  if (b < bat.n) {
    DevScalars* s = reinterpret_cast<DevScalars*>(reinterpret_cast<uintptr_t>(sc) +
                                                  (size_t)b * bat.slab);
    if (!bskip(s, bat)) cont = ctl_apply(op, s, b == 0 ? add : 0, false);
  }
  const int any = __syncthreads_or(cont);
  if (threadIdx.x == 0) {
    switch (op) {
      case CTL_NEWTON: set_cond(sc, sc->h_newton, any); break;
      case CTL_ACCEPT: set_cond(sc, sc->h_halve, any); break;
      case CTL_PRE_CYCLE: set_cond(sc, sc->h_cycle, any); break;
      case CTL_CYCLE_END:
        set_cond(sc, sc->h_cycle, any);
        set_cond(sc, sc->h_restart, any);
        if (any) sc->kcount += 4;
        break;
    }
  }
}

cudaError_t launch_ctl(int op, DevScalars* sc, cudaStream_t st, int add, Bat bat) {
  if (bat.on) {
    if (bat.n > 1024) return cudaErrorInvalidValue;
    k_ctl_batch<<<1, (bat.n + 31) / 32 * 32, 0, st>>>(op, sc, add, bat);
  } else {
    k_ctl<<<1, 32, 0, st>>>(op, sc, add);
  }
  return cudaGetLastError();
}

__global__ void k_sum_sel(UPair up, long P, double* partials, DevScalars* sc, double* mean_out,
                          Bat bat) {
  up.a = badv(up.a, bat);
  up.b = badv(up.b, bat);
  partials = badv(partials, bat);
  sc = badv(sc, bat);
  mean_out = badv(mean_out, bat);
  if (bskip(sc, bat)) return;
  const double* __restrict__ u = (sc->upar & 1) ? up.b : up.a;
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

__global__ void k_sub_sel(UPair up, double* __restrict__ out, long P,
                          const DevScalars* __restrict__ sc, const double* __restrict__ mean,
                          Bat bat) {
  up.a = badv(up.a, bat);
  up.b = badv(up.b, bat);
  out = badv(out, bat);
  sc = badv(sc, bat);
  mean = badv(mean, bat);
  if (bskip(sc, bat)) return;
  const double* __restrict__ u = (sc->upar & 1) ? up.b : up.a;
  const double m = *mean;
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x)
    out[p] = u[p] - m;
}

cudaError_t launch_final_gauge(UPair u, double* out, int N, int M, double* partials,
                               DevScalars* sc, double* mean_out, cudaStream_t st, Bat bat) {
  const dim3 nb = bgrid(dim3(reduce_blocks()), bat);
  k_sum_sel<<<nb, 256, 0, st>>>(u, (long)N * M, partials, sc, mean_out, bat);
  k_sub_sel<<<nb, 256, 0, st>>>(u, out, (long)N * M, sc, mean_out, bat);
  return cudaGetLastError();
}

// grid gradient of g by the 4th-order centred differences (periodic), FP64 and FP32 copies:
// the nearest-node and bilinear interpolation modes interpolate it at the displaced points
__global__ void k_grad4(const double* __restrict__ g, int N, int M, double* __restrict__ gx,
                        double* __restrict__ gy, float* __restrict__ gx32,
                        float* __restrict__ gy32) {
  const long P = (long)N * M;
  const double sx = (double)M / 12.0, sy = (double)N / 12.0;
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x) {
    const int i = (int)(p / M), j = (int)(p - (long)i * M);
    const double* row = g + (size_t)i * M;
    const int jm1 = wrapi(j - 1, M), jm2 = wrapi(j - 2, M), jp1 = wrapi(j + 1, M),
              jp2 = wrapi(j + 2, M);
    const int im1 = wrapi(i - 1, N), im2 = wrapi(i - 2, N), ip1 = wrapi(i + 1, N),
              ip2 = wrapi(i + 2, N);
    const double a = (-row[jp2] + 8.0 * row[jp1] - 8.0 * row[jm1] + row[jm2]) * sx;
    const double b = (-g[(size_t)ip2 * M + j] + 8.0 * g[(size_t)ip1 * M + j] -
                      8.0 * g[(size_t)im1 * M + j] + g[(size_t)im2 * M + j]) * sy;
    gx[p] = a;
    gy[p] = b;
    gx32[p] = (float)a;
    gy32[p] = (float)b;
  }
}

cudaError_t launch_grad4(const double* g, int N, int M, double* gx, double* gy, float* gx32,
                         float* gy32, cudaStream_t st) {
  k_grad4<<<reduce_blocks(), 256, 0, st>>>(g, N, M, gx, gy, gx32, gy32);
  return cudaGetLastError();
}

// 2-norm and normalisation of a vector (the power iteration of the inverse operator)
__global__ void k_norm2(const double* __restrict__ x, long P, double* partials, DevScalars* sc) {
  double v[1] = {0.0};
  const int kind[1] = {0};
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x)
    v[0] += x[p] * x[p];
  block_reduce<1>(v, kind);
  if (!publish_partials<1>(v, partials, &sc->ticket[TK_NORM])) return;
  reduce_partials<1>(v, kind, partials, gridDim.x);
  if (threadIdx.x == 0) {
    sc->pw_norm = sqrt(v[0]);
    sc->ticket[TK_NORM] = 0;
  }
}

__global__ void k_scale_by_norm(double* __restrict__ x, long P, const DevScalars* __restrict__ sc) {
  const double n = sc->pw_norm;
  const double s = n > 0.0 ? 1.0 / n : 0.0;
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x)
    x[p] *= s;
}

// kernel timing: put an Arnoldi step back to step j of an open cycle, outside any graph
// (the step's close must not touch the conditional handles of the plan's solve graph, which
// may have been destroyed since)
__global__ void k_set_step(DevScalars* sc, int j) {
  sc->j = j;
  sc->jd = j;
  sc->cycle_done = 0;
  sc->graph = 0;
  sc->ticket[TK_DOTS] = 0;
}

cudaError_t launch_set_step(DevScalars* sc, int j, cudaStream_t st) {
  k_set_step<<<1, 1, 0, st>>>(sc, j);
  return cudaGetLastError();
}

cudaError_t launch_normalize(double* x, long P, double* partials, DevScalars* sc,
                             cudaStream_t st) {
  const int nb = reduce_blocks();
  k_norm2<<<nb, 256, 0, st>>>(x, P, partials, sc);
  k_scale_by_norm<<<nb, 256, 0, st>>>(x, P, sc);
  return cudaGetLastError();
}

// batched solve: copies between the pairs' slabs and the caller's per-pair planes
__global__ void k_gather(const double* const* __restrict__ tab, double* __restrict__ dst, long P,
                         Bat bat) {
  const double* __restrict__ src = tab[blockIdx.z];
  dst = badv(dst, bat);
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x)
    dst[p] = src[p];
}

__global__ void k_scatter(const double* __restrict__ src, double* const* __restrict__ tab,
                          long P, const DevScalars* __restrict__ sc, Bat bat) {
  sc = badv(sc, bat);
  if (bskip(sc, bat)) return;
  double* __restrict__ dst = tab[blockIdx.z];
  src = badv(src, bat);
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x)
    dst[p] = src[p];
}

cudaError_t launch_gather(const double* const* tab, double* dst, long P, Bat bat,
                          cudaStream_t st) {
  k_gather<<<bgrid(dim3(reduce_blocks()), bat), 256, 0, st>>>(tab, dst, P, bat);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const double* src, double* const* tab, long P, const DevScalars* sc,
                           Bat bat, cudaStream_t st) {
  k_scatter<<<bgrid(dim3(reduce_blocks()), bat), 256, 0, st>>>(src, tab, P, sc, bat);
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
                                          cudaStream_t, const double*, int, const float*, int,  \
                                          Interp);                                            \
  template cudaError_t launch_gmres_init<T>(const double*, const T*, T*, long, int, double*,  \
                                            DevScalars*, int, cudaStream_t, T*, Bat);         \
  template cudaError_t launch_gmres_dots<T>(const T*, const T*, long, double*, DevScalars*,   \
                                            int, cudaStream_t, int, Bat);                     \
  template cudaError_t launch_gmres_update<T>(T*, const T*, long, double*, DevScalars*, int,  \
                                              cudaStream_t, int, Bat);                        \
  template cudaError_t launch_gmres_combine<T>(const T*, T*, long, const DevScalars*, int,    \
                                               cudaStream_t, Bat);                            \
  template cudaError_t launch_convert<T>(const void*, int, void*, int, long, cudaStream_t);

OTGB_INST_NEWTON(float)
OTGB_INST_NEWTON(double)

}  // namespace otgb
