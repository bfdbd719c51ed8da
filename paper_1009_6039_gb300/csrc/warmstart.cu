// Learned warm start: the kernels of the network's input features, of its training (FP32)
// and of its inference (BF16 on the tcgen05 tensor cores with an FP32 accumulator in TMEM);
// also the transport outputs of Sec. 5.2, which share the tiled double-float stencils.
//
// The paper starts Newton from u0 = 0; the damped iteration only needs an admissible start,
// det(I + D^2 u0) > 0 (Theorem convproof).  The warm start is
//   h  = P(log f - log g)        P: mean-zero inverse of the 4th-order stencil Laplacian
//   x  = 16 features per point at h (below)
//   s  = MLP(x), 16 -> 128 -> 128 -> 128 -> 1, SiLU, trained to predict Lap_h(phi* - h)
//   u0 = alpha (h + P(G s)), G the Gaussian low-pass exp(-((k1/(M/4))^2 + (k2/(N/4))^2)/2),
//        alpha the largest of 1, 1/2, 1/4, 1/8 with det(I + alpha D^2 u0) > 0 everywhere,
//        else 0 (the zero start).
// Parameters: one flat FP32 vector W0[H,16], b0[H], W1[H,H], b1[H], W2[H,H], b2[H], w3[H], b3.
#include <math.h>
#include <stdint.h>

#include <cuda_bf16.h>

#include "dd.cuh"
#include "otgb_internal.cuh"

namespace otgb {

namespace {

constexpr int K = OTGB_WS_K, H = OTGB_WS_H;
constexpr float kFloor = 1e-3f;

// index a mod L for any int a (the displaced-point gather can leave the grid by many cells)
__device__ __forceinline__ int wrapi(int a, int L) {
  const int r = a % L;
  return r < 0 ? r + L : r;
}
// index i + d mod L for 0 <= i < L and |d| < L (stencil neighbours): no division
__device__ __forceinline__ int wrap_near(int a, int L) {
  return a < 0 ? a + L : (a >= L ? a - L : a);
}

// 4th-order centred stencils of a periodic FP64 field (spacing 1/M along j, 1/N along i),
// at grid points 0 <= i < N, 0 <= j < M
struct Stencil {
  const double* u;
  int N, M;
  __device__ double at(int i, int j) const {
    return u[(size_t)wrap_near(i, N) * M + wrap_near(j, M)];
  }
  __device__ double dx(int i, int j) const {
    return (-at(i, j + 2) + 8.0 * at(i, j + 1) - 8.0 * at(i, j - 1) + at(i, j - 2)) *
           (double)M / 12.0;
  }
  __device__ double dy(int i, int j) const {
    return (-at(i + 2, j) + 8.0 * at(i + 1, j) - 8.0 * at(i - 1, j) + at(i - 2, j)) *
           (double)N / 12.0;
  }
  __device__ double dxx(int i, int j) const {
    return (-at(i, j + 2) + 16.0 * at(i, j + 1) - 30.0 * at(i, j) + 16.0 * at(i, j - 1) -
            at(i, j - 2)) * (double)M * (double)M / 12.0;
  }
  __device__ double dyy(int i, int j) const {
    return (-at(i + 2, j) + 16.0 * at(i + 1, j) - 30.0 * at(i, j) + 16.0 * at(i - 1, j) -
            at(i - 2, j)) * (double)N * (double)N / 12.0;
  }
  __device__ double dxy(int i, int j) const {
    return (-dy(i, j + 2) + 8.0 * dy(i, j + 1) - 8.0 * dy(i, j - 1) + dy(i, j - 2)) *
           (double)M / 12.0;
  }
};

// log f - log g with FP32 logarithms (h only seeds the features and the warm start)
template <typename T>
__global__ void k_ws_source(const double* __restrict__ f, const double* __restrict__ g,
                            T* __restrict__ src, long P) {
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x)
    src[p] = (T)(logf((float)f[p]) - logf((float)g[p]));
}

// ---------------------------------------------------------------------------------------
// Tiled stencils in double-float arithmetic: a block of 256 threads owns a 32 x 32 tile of
// grid points (4 rows per thread) and stages the field with a halo of 2 (as dd) and its
// unscaled y-differences in shared memory.
// ---------------------------------------------------------------------------------------
constexpr int TW = 32, TRPT = 4;
struct TileDD {
  dd t[TW + 4][TW + 4];
  dd dy[TW][TW + 4];
};
struct StencilK {
  dd Mh, Nh, Mh2, Nh2, MNh;  // M/12, N/12, M^2/12, N^2/12, MN/144
};

__device__ void tile_load_dd(TileDD& T, const double* __restrict__ u, int N, int M, int by,
                             int bx) {
  for (int idx = threadIdx.x; idx < (TW + 4) * (TW + 4); idx += blockDim.x) {
    const int r = idx / (TW + 4), cc = idx - r * (TW + 4);
    const int gi = wrap_near(by + r - 2, N), gj = wrap_near(bx + cc - 2, M);
    T.t[r][cc] = dd_from_double(u[(size_t)gi * M + gj]);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < TW * (TW + 4); idx += blockDim.x) {
    const int r = idx / (TW + 4), cc = idx - r * (TW + 4);
    T.dy[r][cc] = dd_sub(dd_scale2(dd_sub(T.t[r + 3][cc], T.t[r + 1][cc]), 8.0f),
                         dd_sub(T.t[r + 4][cc], T.t[r][cc]));
  }
  __syncthreads();
}

// 4th-order stencils at tile point (ty, tx)
__device__ __forceinline__ void tile_stencils_dd(const TileDD& T, int ty, int tx,
                                                 const StencilK& K, dd* ux, dd* uy, dd* uxx,
                                                 dd* uyy, dd* uxy) {
  const int r = ty + 2, q = tx + 2;
  const dd c0 = T.t[r][q];
  const dd xp1 = T.t[r][q + 1], xm1 = T.t[r][q - 1], xp2 = T.t[r][q + 2], xm2 = T.t[r][q - 2];
  const dd yp1 = T.t[r + 1][q], ym1 = T.t[r - 1][q], yp2 = T.t[r + 2][q], ym2 = T.t[r - 2][q];
  const dd c30 = dd_mul_f(c0, 30.0f);
  *ux = dd_mul(dd_sub(dd_scale2(dd_sub(xp1, xm1), 8.0f), dd_sub(xp2, xm2)), K.Mh);
  *uy = dd_mul(T.dy[ty][q], K.Nh);
  *uxx = dd_mul(dd_sub(dd_sub(dd_scale2(dd_add(xp1, xm1), 16.0f), dd_add(xp2, xm2)), c30),
                K.Mh2);
  *uyy = dd_mul(dd_sub(dd_sub(dd_scale2(dd_add(yp1, ym1), 16.0f), dd_add(yp2, ym2)), c30),
                K.Nh2);
  *uxy = dd_mul(dd_sub(dd_scale2(dd_sub(T.dy[ty][q + 1], T.dy[ty][q - 1]), 8.0f),
                       dd_sub(T.dy[ty][q + 2], T.dy[ty][q - 2])),
                K.MNh);
}

// integer part and fraction (FP32) of the dd grid position p
__device__ __forceinline__ int dd_floor_frac(dd p, float* t) {
  float fl = floorf(p.hi);
  dd fr = dd_add_f(p, -fl);
  if (fr.hi < 0.0f) {
    fl -= 1.0f;
    fr = dd_add_f(fr, 1.0f);
  } else if (fr.hi >= 1.0f) {
    fl += 1.0f;
    fr = dd_add_f(fr, -1.0f);
  }
  *t = fminf(fr.hi, 0.99999994f);
  return (int)fl;
}

__device__ __forceinline__ void cubic_bspline_f(float t, float w[4], float dw[4]) {
  const float t2 = t * t, t3 = t2 * t, s = 1.0f - t;
  w[0] = s * s * s * (1.0f / 6.0f);
  w[1] = (3.0f * t3 - 6.0f * t2 + 4.0f) * (1.0f / 6.0f);
  w[2] = (-3.0f * t3 + 3.0f * t2 + 3.0f * t + 1.0f) * (1.0f / 6.0f);
  w[3] = t3 * (1.0f / 6.0f);
  dw[0] = -0.5f * s * s;
  dw[1] = 0.5f * (3.0f * t2 - 4.0f * t);
  dw[2] = 0.5f * (-3.0f * t2 + 2.0f * t + 1.0f);
  dw[3] = 0.5f * t2;
}

// features at the potential h: stencils of h and the displaced point in double-float, the
// interpolant of g (FP32 coefficients), its gradient and the logarithms in FP32:
//  [log f, log g, lg, r = log f - lg - ld, hxx + hyy, hxx - hyy, 2 hxy, hxx hyy - hxy^2,
//   10 hx, 10 hy, 0.1 Gx / Gc, 0.1 Gy / Gc, (Gx hx + Gy hy) / Gc, (hxx - hyy)^2 + 4 hxy^2,
//   r (hxx + hyy), 0],   Gc = max(G, floor), lg = log Gc, ld = log max(det, floor),
// G, Gx, Gy the interpolant of g at T = x + grad h, det = det(I + D^2 h).
__global__ void __launch_bounds__(256)
    k_ws_features(const double* __restrict__ f, const double* __restrict__ g,
                  const float* __restrict__ c32, const double* __restrict__ h, int N, int M,
                  StencilK K, float* __restrict__ X) {
  __shared__ TileDD T;
  const int bx = blockIdx.x * TW, by = blockIdx.y * TW;
  tile_load_dd(T, h, N, M, by, bx);
  const int tx = threadIdx.x % TW, ty0 = threadIdx.x / TW;
  const int j = bx + tx;
#pragma unroll 1
  for (int rr = 0; rr < TRPT; ++rr) {
    const int ty = ty0 + rr * (TW / TRPT);
    const int i = by + ty;
    if (i >= N || j >= M) continue;
    dd ux, uy, uxx, uyy, uxy;
    tile_stencils_dd(T, ty, tx, K, &ux, &uy, &uxx, &uyy, &uxy);
    float txf, tyf;
    const int fj = dd_floor_frac(dd_add_f(dd_mul_f(ux, (float)M), (float)j), &txf);
    const int fi = dd_floor_frac(dd_add_f(dd_mul_f(uy, (float)N), (float)i), &tyf);
    const int j0 = wrapi(fj, M), i0 = wrapi(fi, N);
    float wx[4], dwx[4], wy[4], dwy[4];
    cubic_bspline_f(txf, wx, dwx);
    cubic_bspline_f(tyf, wy, dwy);
    float G = 0.f, gx = 0.f, gy = 0.f;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float* row = c32 + (size_t)wrap_near(i0 - 1 + b, N) * M;
      float rv = 0.f, rd = 0.f;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float cv = __ldg(row + wrap_near(j0 - 1 + a, M));
        rv = fmaf(cv, wx[a], rv);
        rd = fmaf(cv, dwx[a], rd);
      }
      G = fmaf(rv, wy[b], G);
      gx = fmaf(rd, wy[b], gx);
      gy = fmaf(rv, dwy[b], gy);
    }
    const float Gx = gx * (float)M, Gy = gy * (float)N;
    const float hx = ux.hi, hy = uy.hi, hxx = uxx.hi, hyy = uyy.hi, hxy = uxy.hi;
    const float det = (1.0f + hxx) * (1.0f + hyy) - hxy * hxy;
    const float Gc = fmaxf(G, kFloor);
    const size_t p = (size_t)i * M + j;
    const float lf = logf((float)f[p]), lg = logf(Gc), ld = logf(fmaxf(det, kFloor));
    const float r = lf - lg - ld;
    float x[16];
    x[0] = lf;
    x[1] = logf((float)g[p]);
    x[2] = lg;
    x[3] = r;
    x[4] = hxx + hyy;
    x[5] = hxx - hyy;
    x[6] = 2.0f * hxy;
    x[7] = hxx * hyy - hxy * hxy;
    x[8] = 10.0f * hx;
    x[9] = 10.0f * hy;
    x[10] = 0.1f * Gx / Gc;
    x[11] = 0.1f * Gy / Gc;
    x[12] = (Gx * hx + Gy * hy) / Gc;
    x[13] = (hxx - hyy) * (hxx - hyy) + 4.0f * hxy * hxy;
    x[14] = r * (hxx + hyy);
    x[15] = 0.f;
    float4* o = reinterpret_cast<float4*>(X + p * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      o[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
  }
}

// training target s* = (D_xx + D_yy)(phi - h)
__global__ void k_ws_target(const double* __restrict__ phi, const double* __restrict__ h,
                            int N, int M, double* __restrict__ diff, float* __restrict__ t,
                            int stage) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= M) return;
  const size_t p = (size_t)i * M + j;
  if (stage == 0) {
    diff[p] = phi[p] - h[p];
  } else {
    const Stencil S{diff, N, M};
    t[p] = (float)(S.dxx(i, j) + S.dyy(i, j));
  }
}

__global__ void k_ws_widen(const float* __restrict__ s, double* __restrict__ out, long P) {
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x)
    out[p] = (double)s[p];
}

__global__ void k_ws_sum(const double* __restrict__ h, const double* __restrict__ t,
                         double* __restrict__ u, long P) {
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x)
    u[p] = h[p] + t[p];
}

// min over the grid of det(I + alpha D^2 u) for each alpha in {1, 1/2, 1/4, 1/8} (tiled
// double-float stencils; alpha scales exactly); the last block picks the largest admissible
// alpha (0 if none, or if the network reported an error) and writes it to *alpha.
__global__ void __launch_bounds__(256)
    k_ws_admissible(const double* __restrict__ u, int N, int M, StencilK K,
                    double* __restrict__ partials, unsigned int* ticket,
                    const int* __restrict__ err, double* alpha) {
  __shared__ TileDD T;
  __shared__ float red[4][8];
  __shared__ bool last;
  const int bx = blockIdx.x * TW, by = blockIdx.y * TW;
  tile_load_dd(T, u, N, M, by, bx);
  float mn[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
  const int tx = threadIdx.x % TW, ty0 = threadIdx.x / TW;
  const int j = bx + tx;
#pragma unroll 1
  for (int rr = 0; rr < TRPT; ++rr) {
    const int ty = ty0 + rr * (TW / TRPT);
    const int i = by + ty;
    if (i >= N || j >= M) continue;
    dd ux, uy, uxx, uyy, uxy;
    tile_stencils_dd(T, ty, tx, K, &ux, &uy, &uxx, &uyy, &uxy);
    float a = 1.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q, a *= 0.5f) {
      const dd d = dd_sub(dd_mul(dd_add_f(dd_scale2(uxx, a), 1.0f), dd_add_f(dd_scale2(uyy, a), 1.0f)),
                          dd_scale2(dd_mul(uxy, uxy), a * a));
      mn[q] = fminf(mn[q], d.hi);  // d.hi carries the sign (d.hi == 0 counts as not > 0)
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float v = mn[q];
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[q][wid] = v;
  }
  __syncthreads();
  const unsigned int nb = gridDim.x * gridDim.y;
  const unsigned int bid = blockIdx.y * gridDim.x + blockIdx.x;
  if (threadIdx.x == 0) {
    for (int q = 0; q < 4; ++q) {
      float v = INFINITY;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fminf(v, red[q][w]);
      partials[(size_t)bid * 4 + q] = (double)v;
    }
    __threadfence();
    last = atomicAdd(ticket, 1u) == nb - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last block: all its threads take the per-block minima (strided, then a block tree)
  float v4[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
  for (unsigned int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
    for (int q = 0; q < 4; ++q)
      v4[q] = fminf(v4[q], (float)((volatile const double*)partials)[(size_t)b * 4 + q]);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float v = v4[q];
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[q][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double a = 1.0, pick = 0.0;
  for (int q = 0; q < 4; ++q, a *= 0.5) {
    float v = INFINITY;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fminf(v, red[q][w]);
    if (v > 0.0f) {
      pick = a;
      break;
    }
  }
  if (err && *err) pick = 0.0;
  *alpha = pick;
  *ticket = 0u;
}

__global__ void k_ws_scale(double* __restrict__ u, long P, const double* __restrict__ alpha) {
  const double a = *alpha;
  // a = 0 is the zero start: written as such, so that a non-finite prediction (e.g. after a
  // network timeout) cannot leak into it through 0 * inf
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x)
    u[p] = (a == 0.0) ? 0.0 : u[p] * a;
}

// ---------------------------------------------------------------------------------------
// BF16 inference on the tensor cores (tcgen05).
//
// One CTA of 128 threads takes 128-row tiles of X: thread r owns row r, which is TMEM lane
// r of the accumulator (warp w reads lanes 32w..32w+31).  Per tile: X (converted to BF16)
// -> MMA with W0 (K = 16) -> TMEM -> SiLU -> BF16 activations in shared memory -> 8 MMAs
// with W1 (K = 128) -> ... -> W2 -> SiLU -> dot with w3 in FP32 -> s.  The biases b0, b1,
// b2 ride in the matrix products: one more K block per layer, whose B rows hold the bias
// split into two BF16 parts (hi = bf16(b), lo = bf16(b - hi), b to 2^-17 relative) against
// an A block of ones in its first two columns, so that the accumulator holds z = a W^T + b.
//
// Operands are K-major BF16 in the no-swizzle canonical layout: 8-row x 16-byte core
// matrices, the two core matrices of a 16-wide K block 128 bytes apart (LBO) and
// consecutive 8-row groups 256 bytes apart (SBO); each K block of a 128-row operand is a
// contiguous 4 KB.  Byte offset of element (r, k):
//   (k / 16) * 4096 + (r / 8) * 256 + ((k / 8) % 2) * 128 + (r % 8) * 16 + (k % 8) * 2.
// ---------------------------------------------------------------------------------------
__host__ __device__ constexpr int op_offset(int r, int k) {
  return (k >> 4) * 4096 + (r >> 3) * 256 + ((k >> 3) & 1) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// chains of the tensor-core network kernel: independent warpgroups, each with its own
// 128-row tile, activation buffer, TMEM accumulator (128 columns) and mbarrier
constexpr int WS_CH = 4;

// packed weights (operand layout, each layer's bias block after its weight K blocks)
constexpr int SM_W0 = 0;                       // W0 (K = 16) + bias block: 8 KB
constexpr int SM_W1 = SM_W0 + 8192;            // W1 (K = 128) + bias block: 36 KB
constexpr int SM_W2 = SM_W1 + 36864;           // W2 + bias block: 36 KB
constexpr int SM_ONES = SM_W2 + 36864;         // the A block of ones: 4 KB
constexpr int SM_A = SM_ONES + 4096;           // WS_CH x 32 KB activations / X tiles
constexpr int SM_BIAS = SM_A + WS_CH * 32768;  // w3 (128 FP32), b3
constexpr int SM_BAR = SM_BIAS + 128 * 4 + 16; // WS_CH mbarriers
constexpr int SM_TMEM = SM_BAR + 8 * WS_CH;
constexpr int SM_TOTAL = SM_TMEM + 8 + 128;    // + alignment slack
constexpr int PACKED_W_BYTES = SM_A - SM_W0;   // 86016: W0, W1, W2 with biases, ones

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: start, LBO, SBO (all >> 4), version 1 (bit 46),
// base offset 0, no swizzle
__device__ __forceinline__ uint64_t mdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, M = 128, N = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 3) << 17) |
                            ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// bounded wait for the mbarrier phase with parity `par`: at most 4096 tries, each of which
// suspends the thread for at most 10 us (the suspend-time hint) -- about 40 ms in all, where
// an MMA group takes microseconds; false if it gave up
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t par) {
  for (int it = 0; it < 4096; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred q;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(par), "r"(10000)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// TMEM load of 32 columns of this warp's 32 lanes (one FP32 value per column for this
// thread's lane) without its wait: the values arrive in r later, and tmem_wait_ld(r) is the
// point from which they may be read (its in-out operands keep every use of r behind it)
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.wait::ld.sync.aligned;"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
        "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]),
        "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]),
        "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]),
        "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]),
        "+r"(r[31])
      :
      : "memory");
}

// the load and its wait: 32 FP32 values of this thread's lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  tmem_ld32_async(taddr, r);
  tmem_wait_ld(r);
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// SiLU of four values (two packed pairs) with one reciprocal.  The readout of the
// tensor-core network is bound by instruction issue and the special-function unit (an
// exponential and a reciprocal per value): the elementwise steps run as packed FP32 pairs
// (FMUL2), and Montgomery's simultaneous inversion (1 / (d0 d1 d2 d3) and the partial
// products give every 1/d_i) leaves a quarter reciprocal per value, at a few ulp of extra
// error.  The packed weights and biases carry a factor 2^-30 (exact in BF16 and FP32), so
// the accumulator holds z' = 2^-30 z, and with d' = min(2^-30 (1 + e^-z), 1) -- one
// saturating FMA, which also caps the denominator so that the product of four stays finite
// and normal -- SiLU(z) = z / (1 + e^-z) = z' / d'.  Below z = -20.8 the cap makes the value
// -|z| 2^-30 instead of -|z| e^-|z|, both negligible against the O(1) activations they are
// summed with.
constexpr float kZScale = 0x1p-30f;  // z' = kZScale z
__device__ __forceinline__ float ex2_ftz(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_ftz(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// d' = saturate(e 2^-30 + 2^-30): 2^-30 (1 + e) capped at 1 (+inf -> 1)
__device__ __forceinline__ float den_sat(float e) {
  float y;
  asm("fma.rn.sat.f32 %0, %1, %2, %2;" : "=f"(y) : "f"(e), "f"(kZScale));
  return y;
}
__device__ __forceinline__ void silu_x4(float2& z01, float2& z23) {
  // t = -z log2(e) = z' (-log2(e) / kZScale)
  const float2 nl = make_float2(-1.4426950408889634f / kZScale, -1.4426950408889634f / kZScale);
  const float2 t01 = __fmul2_rn(z01, nl), t23 = __fmul2_rn(z23, nl);
  const float d0 = den_sat(ex2_ftz(t01.x)), d1 = den_sat(ex2_ftz(t01.y));
  const float d2 = den_sat(ex2_ftz(t23.x)), d3 = den_sat(ex2_ftz(t23.y));
  const float ab = d0 * d1, cd = d2 * d3;
  const float rp = rcp_ftz(ab * cd);
  const float iab = cd * rp, icd = ab * rp;
  z01 = __fmul2_rn(z01, make_float2(d1 * iab, d0 * iab));
  z23 = __fmul2_rn(z23, make_float2(d3 * icd, d2 * icd));
}

// SiLU of 32 accumulator values (the bias is already in them), in place
__device__ __forceinline__ void silu32(float (&v)[32]) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float2 z01 = make_float2(v[4 * q], v[4 * q + 1]);
    float2 z23 = make_float2(v[4 * q + 2], v[4 * q + 3]);
    silu_x4(z01, z23);
    v[4 * q] = z01.x;
    v[4 * q + 1] = z01.y;
    v[4 * q + 2] = z23.x;
    v[4 * q + 3] = z23.y;
  }
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// store 8 consecutive BF16 values of row r starting at column k0 (a multiple of 8)
__device__ __forceinline__ void st_row8(unsigned char* base, int r, int k0, const float* v) {
  uint4 q;
  q.x = pack_bf16(v[0], v[1]);
  q.y = pack_bf16(v[2], v[3]);
  q.z = pack_bf16(v[4], v[5]);
  q.w = pack_bf16(v[6], v[7]);
  *reinterpret_cast<uint4*>(base + op_offset(r, k0)) = q;
}

// wait for this chain's MMA group (all its threads poll with a suspend hint, bounded)
__device__ __forceinline__ bool chain_wait(uint32_t bar, uint32_t par) {
  const bool ok = bar_wait(bar, par);
  fence_after();
  return ok;
}

// barrier of one chain (warpgroup g: 128 threads, named barrier 1 + g)
__device__ __forceinline__ void chain_sync(int g) {
  asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory");
}

// the same barrier, returning whether every thread of the chain passed ok: the chain takes
// one decision after a bounded wait, even if its threads' waits ended differently
__device__ __forceinline__ bool chain_all(int g, bool ok) {
  uint32_t res;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, 128, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(res)
      : "r"((uint32_t)ok), "r"(1 + g)
      : "memory");
  return res != 0;
}

// one row of X (16 FP32 features; zeros past the last row)
__device__ __forceinline__ void load_x_row(const float* __restrict__ X, long row, long rows,
                                           float (&v)[16]) {
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = 0.f;
  if (row < rows) {
    const float4* xr = reinterpret_cast<const float4*>(X + row * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 a = __ldg(xr + q);
      v[4 * q] = a.x;
      v[4 * q + 1] = a.y;
      v[4 * q + 2] = a.z;
      v[4 * q + 3] = a.w;
    }
  }
}

// layer readout of this thread's row r (all 128 columns of the chain's accumulator, 32 at a
// time): SiLU -> BF16 A tile of the next layer
__device__ __forceinline__ void readout_row(uint32_t trow, unsigned char* sA, int r) {
#pragma unroll 1
  for (int col = 0; col < 128; col += 32) {
    float v[32];
    tmem_ld32(trow + col, v);
    silu32(v);
#pragma unroll
    for (int q = 0; q < 4; ++q) st_row8(sA, r, col + 8 * q, v + 8 * q);
  }
}

// One persistent CTA per SM holds the weights once and runs WS_CH independent chains, one
// per warpgroup: chain g takes 128-row tiles (thread r of the warpgroup owns row r, which
// is TMEM lane r, in accumulator columns 128 g ..), and per tile issues its three MMA
// groups from its first thread and reads each result back with its 128 threads.  The
// chains synchronise only within themselves (named barriers), so one chain's MMAs run
// while the others read out (the readout -- bias, SiLU, BF16 packing -- bounds the kernel).
// stall != 0 (a test of the failure path): chain 0 does not issue its first MMA group, so
// its wait runs out; the kernel then sets *err and the chain stops (after a bounded wait
// for anything it has in flight); the others finish, and the TMEM is freed at the end.
__global__ void __launch_bounds__(128 * WS_CH, 1)
    k_ws_mlp_tc(const unsigned char* __restrict__ wpack, const float* __restrict__ params,
                const float* __restrict__ X, long rows, float* __restrict__ out,
                int* __restrict__ err, int stall) {
  constexpr int NT = 128 * WS_CH;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* sm =
      (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  const int tid = threadIdx.x, warp = tid >> 5, g = warp >> 2, r = tid & 127;
  float* sb = reinterpret_cast<float*>(sm + SM_BIAS);
  const uint32_t bar = smem_u32(sm + SM_BAR + 8 * g);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + SM_TMEM);

  // weights with their bias blocks and the block of ones (pre-packed BF16 operand layout),
  // and w3, b3 in FP32, into shared memory
  {
    const uint4* src = reinterpret_cast<const uint4*>(wpack);
    uint4* dst = reinterpret_cast<uint4*>(sm + SM_W0);
    for (int q = tid; q < PACKED_W_BYTES / 16; q += NT) dst[q] = src[q];
    for (int q = tid; q < H; q += NT) sb[q] = params[H * K + 3 * H + 2 * H * H + q];  // w3
    if (tid == 0) sb[128] = params[H * K + 4 * H + 2 * H * H];                       // b3
  }
  if (warp == 0) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
            smem_u32(tmem_slot)),
        "r"(128 * WS_CH)
        : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (r == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = *tmem_slot;
  const uint32_t tacc = tbase + 128 * g;                              // this chain's columns
  const uint32_t trow = tacc + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's lanes
  unsigned char* sA = sm + SM_A + 32768 * g;
  const uint32_t aA = smem_u32(sA), aW0 = smem_u32(sm + SM_W0), aW1 = smem_u32(sm + SM_W1),
                 aW2 = smem_u32(sm + SM_W2), aOnes = smem_u32(sm + SM_ONES);
  uint32_t phase = 0;
  bool ok = true;
  bool inflight = false;
  const long ntiles = (rows + 127) / 128;
  const long tstride = (long)gridDim.x * WS_CH;
  // X row -> BF16 (K block 0 of the A operand): the first tile's here, every later tile's
  // under the previous tile's last matrix product (below)
  {
    const long row0 = ((long)blockIdx.x * WS_CH + g) * 128 + r;
    float v[16];
    load_x_row(X, row0, rows, v);
    st_row8(sA, r, 0, v);
    st_row8(sA, r, 8, v + 8);
  }
  for (long tile = (long)blockIdx.x * WS_CH + g; tile < ntiles && ok; tile += tstride) {
    const long row = tile * 128 + r;
    // the X row two tiles ahead towards L2 (its register load one tile ahead then finds it
    // there)
    {
      const long prow = row + 2 * tstride * 128;
      if (prow < rows) asm volatile("prefetch.global.L2 [%0];" ::"l"(X + prow * 16));
    }
    // layer 0: D = X W0^T + b0; layers 1 and 2: D = A W^T + b, K = 128 in eight K blocks of
    // 16, each layer closed by the bias block against the block of ones
#pragma unroll 1
    for (int layer = 0; layer <= 2; ++layer) {
      fence_async_smem();
      fence_before();
      chain_sync(g);
      if (r == 0 && !(stall && g == 0 && tile == (long)blockIdx.x * WS_CH)) {
        fence_after();
        if (layer == 0) {
          mma_bf16(tacc, mdesc(aA, 128, 256), mdesc(aW0, 128, 256), 0);
          mma_bf16(tacc, mdesc(aOnes, 128, 256), mdesc(aW0 + 4096, 128, 256), 1);
        } else {
          const uint32_t aW = layer == 1 ? aW1 : aW2;
#pragma unroll
          for (int kb = 0; kb < 8; ++kb)
            mma_bf16(tacc, mdesc(aA + kb * 4096, 128, 256), mdesc(aW + kb * 4096, 128, 256),
                     kb > 0 ? 1u : 0u);
          mma_bf16(tacc, mdesc(aOnes, 128, 256), mdesc(aW + 8 * 4096, 128, 256), 1);
        }
        mma_commit(bar);
      }
      inflight = true;
      // the next tile's X row, loaded while the last product of this tile runs
      float xn[16];
      if (layer == 2) load_x_row(X, row + tstride * 128, rows, xn);
      ok = chain_all(g, chain_wait(bar, phase));
      if (!ok) break;
      inflight = false;
      phase ^= 1;
      if (layer == 2) {  // the A tile is free again: the next tile's X into it
        st_row8(sA, r, 0, xn);
        st_row8(sA, r, 8, xn + 8);
      }
      if (layer < 2) {
        readout_row(trow, sA, r);
      } else {
        // last hidden layer: s = b3 + sum_j w3_j SiLU(z_j) in FP32 over the row (two packed
        // partial sums, even and odd j)
        float2 acc2 = make_float2(0.0f, 0.0f);
#pragma unroll 1
        for (int col = 0; col < 128; col += 32) {
          float v[32];
          tmem_ld32(trow + col, v);
          silu32(v);
          const float4* w4 = reinterpret_cast<const float4*>(sb + col);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 w = w4[q];
            acc2 = __ffma2_rn(make_float2(w.x, w.y), make_float2(v[4 * q], v[4 * q + 1]), acc2);
            acc2 = __ffma2_rn(make_float2(w.z, w.w), make_float2(v[4 * q + 2], v[4 * q + 3]),
                              acc2);
          }
        }
        if (row < rows) out[row] = sb[128] + (acc2.x + acc2.y);
      }
    }
  }
  if (!ok) {
    if (r == 0 && err) atomicExch(err, 1);
    // let an MMA group still in flight finish before its TMEM goes away (bounded; with
    // `stall` nothing is in flight and this wait runs out too)
    if (inflight) bar_wait(bar, phase);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                 "r"(128 * WS_CH)
                 : "memory");
}

// FP32 parameters -> the packed operands: W0, W1, W2 in the operand layout (rows = output
// units), each followed by its bias block (column K_l: bf16(b), column K_l + 1: the BF16
// remainder, zeros after), all times kZScale (a power of two: the BF16 values are the
// unscaled ones' times kZScale exactly); then the block of ones (columns 0 and 1 of every
// row)
__global__ void k_ws_pack(const float* __restrict__ params, unsigned char* __restrict__ wpack) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // one 8-element group
  const int n0 = H * (K + 16) / 8, n1 = H * (H + 16) / 8, n3 = 128 * 16 / 8;
  if (idx >= n0 + 2 * n1 + n3) return;
  float v[8];
  if (idx >= n0 + 2 * n1) {  // the block of ones
    const int g = idx - n0 - 2 * n1, row = g / 2, k0 = (g % 2) * 8;
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = (k0 + q < 2) ? 1.0f : 0.0f;
    st_row8(wpack + SM_ONES, row, k0, v);
    return;
  }
  int layer, g = idx;
  if (g < n0) {
    layer = 0;
  } else if (g < n0 + n1) {
    layer = 1;
    g -= n0;
  } else {
    layer = 2;
    g -= n0 + n1;
  }
  const int kd = layer == 0 ? K : H;  // weight columns; the bias block follows
  const int row = g / ((kd + 16) / 8), k0 = (g % ((kd + 16) / 8)) * 8;
  const float* w = params + (layer == 0 ? 0 : (layer == 1 ? H * K + H : H * K + 2 * H + H * H));
  if (k0 < kd) {
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = w[row * kd + k0 + q] * kZScale;
  } else {
    const float b = w[H * kd + row] * kZScale;  // the layer's bias follows its weights
    const float hi = __bfloat162float(__float2bfloat16_rn(b));
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = 0.0f;
    if (k0 == kd) {
      v[0] = hi;
      v[1] = b - hi;
    }
  }
  unsigned char* base = wpack + (layer == 0 ? SM_W0 : (layer == 1 ? SM_W1 : SM_W2));
  st_row8(base, row, k0, v);
}

// ---------------------------------------------------------------------------------------
// Training (FP32 on the CUDA cores: a few GFLOP per step, run offline).
// C[m, n] = sum_k A(m, k) B(k, n) over a 64 x 64 tile per block, 4 x 4 per thread,
// with A(m, k) = TA ? A[k lda + m] : A[m lda + k] and B(k, n) = TB ? B[n ldb + k] : B[k ldb + n].
// blockIdx.z selects a slice [z kchunk, (z + 1) kchunk) of k (partial sums to C + z Mr ldc).
// Epilogues: 0 plain; 1 Z = acc + bias[n], C2 = SiLU(Z); 2 C = acc SiLU'(zp[m, n]).
// ---------------------------------------------------------------------------------------
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256)
    k_gemm(int Mr, int Nc, int Kd, const float* __restrict__ A, int lda,
           const float* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
           const float* __restrict__ bias, float* __restrict__ C2, const float* __restrict__ zp,
           int kchunk) {
  __shared__ float As[16][64 + 4], Bs[16][64 + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int kbeg = blockIdx.z * kchunk, kend = min(Kd, kbeg + kchunk);
  float acc[4][4] = {};
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
    for (int q = threadIdx.x; q < 16 * 64; q += 256) {
      const int kk = TA ? q / 64 : q % 16, mm = TA ? q % 64 : q / 16;
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < Mr && k < kend) ? (TA ? A[(long)k * lda + m] : A[(long)m * lda + k]) : 0.f;
      const int kb = TB ? q % 16 : q / 64, nn = TB ? q / 16 : q % 64;
      const int n = n0 + nn, k2 = k0 + kb;
      Bs[kb][nn] = (n < Nc && k2 < kend) ? (TB ? B[(long)n * ldb + k2] : B[(long)k2 * ldb + n]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[kk][ty * 4 + q];
        b[q] = Bs[kk][tx * 4 + q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
  float* Cz = C + (long)blockIdx.z * Mr * ldc;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int m = m0 + ty * 4 + p;
    if (m >= Mr) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int n = n0 + tx * 4 + q;
      if (n >= Nc) continue;
      const long o = (long)m * ldc + n;
      float v = acc[p][q];
      if (EPI == 1) {
        v += bias[n];
        Cz[o] = v;
        C2[o] = v / (1.0f + expf(-v));
      } else if (EPI == 2) {
        const float z = zp[o], s = 1.0f / (1.0f + expf(-z));
        Cz[o] = v * s * (1.0f + z * (1.0f - s));
      } else {
        Cz[o] = v;
      }
    }
  }
}

// sum of S partial planes of n values each (fixed order) into out
__global__ void k_sum_partials(const float* __restrict__ part, int S, long n,
                               float* __restrict__ out) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n;
       q += (long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < S; ++z) s += part[(long)z * n + q];
    out[q] = s;
  }
}

// column sums of a (rows x cols) matrix over row chunks of `chunk` rows: part[z, col]
__global__ void k_colsum(const float* __restrict__ A, int rows, int cols, int chunk,
                         float* __restrict__ part) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= cols) return;
  const int r0 = blockIdx.y * chunk, r1 = min(rows, r0 + chunk);
  float s = 0.f;
  for (int rr = r0; rr < r1; ++rr) s += A[(long)rr * cols + col];
  part[(long)blockIdx.y * cols + col] = s;
}

__global__ void k_gather_rows(const float* __restrict__ X, const float* __restrict__ t,
                              const long long* __restrict__ idx, int B, float* __restrict__ Xb,
                              float* __restrict__ tb) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= B * 4) return;
  const int b = q >> 2, part = q & 3;
  const long long r = idx[b];
  reinterpret_cast<float4*>(Xb)[(long)b * 4 + part] =
      reinterpret_cast<const float4*>(X)[r * 4 + part];
  if (part == 0) tb[b] = t[r];
}

// output layer: y = A2 w3 + b3, e = y - t, dy = 2 e / B, dZ2 = dy w3 SiLU'(Z2); loss partials
__global__ void k_ws_out(const float* __restrict__ A2, const float* __restrict__ Z2,
                         const float* __restrict__ params, const float* __restrict__ tb, int B,
                         float* __restrict__ dy, float* __restrict__ dZ2,
                         double* __restrict__ loss_part) {
  const int b = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  const float* w3 = params + H * K + 3 * H + 2 * H * H;
  const float b3 = params[H * K + 4 * H + 2 * H * H];
  double e2 = 0.0;
  if (b < B) {
    float s = 0.f;
    for (int j = lane; j < H; j += 32) s = fmaf(A2[(long)b * H + j], w3[j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float e = s + b3 - tb[b];
    const float d = 2.0f * e / (float)B;
    if (lane == 0) dy[b] = d;
    for (int j = lane; j < H; j += 32) {
      const float z = Z2[(long)b * H + j], sg = 1.0f / (1.0f + expf(-z));
      dZ2[(long)b * H + j] = d * w3[j] * sg * (1.0f + z * (1.0f - sg));
    }
    e2 = (double)e * (double)e;
  }
  __shared__ double red[8];
  if (lane == 0) red[threadIdx.x >> 5] = e2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    loss_part[blockIdx.x] = s;
  }
}

__global__ void k_sum_f64(const double* __restrict__ part, int n, double scale,
                          double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int q = 0; q < n; ++q) s += part[q];
  *out = s * scale;
}

__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, long n, float lr, float b1, float b2,
                       float c1, float c2, float eps) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n;
       q += (long)gridDim.x * blockDim.x) {
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.0f - b1) * gq;
    const float vq = b2 * v[q] + (1.0f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    p[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
  }
}

inline dim3 grid2(int N, int M) { return dim3((M + 127) / 128, N); }
inline int nblk(long P, int t = 256) {
  long b = (P + t - 1) / t;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

// ---------------------------------------------------------------------------------------
// Transport outputs (Sec. 5.2): the distance d(f, g) = int |x - T(x)|^2 f dx =
// int |grad u|^2 f dx, T = x + grad u, as the grid mean of |grad u|^2 f (the periodic
// trapezoid rule), and the divergence of the displacement, div = u_xx + u_yy, with the
// residual's 4th-order stencils on the same double-float tiles.  Per-block (hi, lo) partial
// sums; the last block to take a ticket adds them in block order with all its threads.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ dd warp_sum_dd(dd v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = dd_add(v, dd{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
  return v;
}

__global__ void __launch_bounds__(256)
    k_transport(const double* __restrict__ f, const double* __restrict__ u, int N, int M,
                StencilK K, double* __restrict__ div, float2* __restrict__ partials,
                unsigned int* ticket, double* dist) {
  __shared__ TileDD T;
  __shared__ float2 red[8];
  __shared__ bool last;
  const int bx = blockIdx.x * TW, by = blockIdx.y * TW;
  tile_load_dd(T, u, N, M, by, bx);
  const int tx = threadIdx.x % TW, ty0 = threadIdx.x / TW;
  const int j = bx + tx;
  dd acc = dd{0.f, 0.f};
#pragma unroll 1
  for (int rr = 0; rr < TRPT; ++rr) {
    const int ty = ty0 + rr * (TW / TRPT);
    const int i = by + ty;
    if (i >= N || j >= M) continue;
    dd ux, uy, uxx, uyy, uxy;
    tile_stencils_dd(T, ty, tx, K, &ux, &uy, &uxx, &uyy, &uxy);
    const size_t p = (size_t)i * M + j;
    const dd g2 = dd_add(dd_mul(ux, ux), dd_mul(uy, uy));
    acc = dd_add(acc, dd_mul(g2, dd_from_double(f[p])));
    if (div) div[p] = dd_to_double(dd_add(uxx, uyy));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  acc = warp_sum_dd(acc);
  if (lane == 0) red[wid] = make_float2(acc.hi, acc.lo);
  __syncthreads();
  const unsigned int nb = gridDim.x * gridDim.y;
  if (threadIdx.x == 0) {
    dd b = dd{0.f, 0.f};
    for (int w = 0; w < nw; ++w) b = dd_add(b, dd{red[w].x, red[w].y});
    partials[blockIdx.y * gridDim.x + blockIdx.x] = make_float2(b.hi, b.lo);
    __threadfence();
    last = atomicAdd(ticket, 1u) == nb - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  dd s = dd{0.f, 0.f};
  for (unsigned int b = threadIdx.x; b < nb; b += blockDim.x) {
    const volatile float2* q = (const volatile float2*)partials + b;
    s = dd_add(s, dd{q->x, q->y});
  }
  s = warp_sum_dd(s);
  if (lane == 0) red[wid] = make_float2(s.hi, s.lo);
  __syncthreads();
  if (threadIdx.x == 0) {
    dd t = dd{0.f, 0.f};
    for (int w = 0; w < nw; ++w) t = dd_add(t, dd{red[w].x, red[w].y});
    *dist = dd_to_double(t) / ((double)N * (double)M);
    *ticket = 0u;
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
cudaError_t launch_ws_source(const double* f, const double* g, double* src, long P,
                             cudaStream_t st) {
  k_ws_source<double><<<nblk(P), 256, 0, st>>>(f, g, src, P);
  return cudaGetLastError();
}

cudaError_t launch_ws_source32(const double* f, const double* g, float* src, long P,
                               cudaStream_t st) {
  k_ws_source<float><<<nblk(P), 256, 0, st>>>(f, g, src, P);
  return cudaGetLastError();
}

static dd host_dd(double v) {
  dd r;
  r.hi = (float)v;
  r.lo = (float)(v - (double)r.hi);
  return r;
}

static StencilK stencil_consts(int N, int M) {
  StencilK K;
  K.Mh = host_dd((double)M / 12.0);
  K.Nh = host_dd((double)N / 12.0);
  K.Mh2 = host_dd((double)M * (double)M / 12.0);
  K.Nh2 = host_dd((double)N * (double)N / 12.0);
  K.MNh = host_dd((double)M * (double)N / 144.0);
  return K;
}

static dim3 tiles(int N, int M) { return dim3((M + TW - 1) / TW, (N + TW - 1) / TW); }

cudaError_t launch_ws_features(const double* f, const double* g, const float* c32,
                               const double* h, int N, int M, float* X, cudaStream_t st) {
  k_ws_features<<<tiles(N, M), 256, 0, st>>>(f, g, c32, h, N, M, stencil_consts(N, M), X);
  return cudaGetLastError();
}

cudaError_t launch_ws_target(const double* phi, const double* h, int N, int M, double* scratch,
                             float* t, cudaStream_t st) {
  k_ws_target<<<grid2(N, M), 128, 0, st>>>(phi, h, N, M, scratch, t, 0);
  k_ws_target<<<grid2(N, M), 128, 0, st>>>(phi, h, N, M, scratch, t, 1);
  return cudaGetLastError();
}

cudaError_t launch_ws_widen(const float* s, double* out, long P, cudaStream_t st) {
  k_ws_widen<<<nblk(P), 256, 0, st>>>(s, out, P);
  return cudaGetLastError();
}

cudaError_t launch_ws_sum(const double* h, const double* t, double* u, long P, cudaStream_t st) {
  k_ws_sum<<<nblk(P), 256, 0, st>>>(h, t, u, P);
  return cudaGetLastError();
}

int ws_admissible_blocks(int N, int M) { return ((M + TW - 1) / TW) * ((N + TW - 1) / TW); }

cudaError_t launch_ws_admissible(double* u, int N, int M, double* partials,
                                 unsigned int* ticket, const int* err, double* alpha,
                                 cudaStream_t st) {
  k_ws_admissible<<<tiles(N, M), 256, 0, st>>>(u, N, M, stencil_consts(N, M), partials, ticket,
                                               err, alpha);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long P = (long)N * M;
  k_ws_scale<<<nblk(P), 256, 0, st>>>(u, P, alpha);
  return cudaGetLastError();
}

cudaError_t launch_transport(const double* f, const double* u, int N, int M, double* div,
                             double* partials, unsigned int* ticket, double* dist,
                             cudaStream_t st) {
  k_transport<<<tiles(N, M), 256, 0, st>>>(f, u, N, M, stencil_consts(N, M), div,
                                           reinterpret_cast<float2*>(partials), ticket, dist);
  return cudaGetLastError();
}

size_t ws_packed_bytes() { return PACKED_W_BYTES; }

cudaError_t launch_ws_pack(const float* params, unsigned char* wpack, cudaStream_t st) {
  const int n = (H * (K + 16) + 2 * H * (H + 16) + 128 * 16) / 8;
  k_ws_pack<<<(n + 255) / 256, 256, 0, st>>>(params, wpack);
  return cudaGetLastError();
}

cudaError_t launch_ws_mlp(const unsigned char* wpack, const float* params, const float* X,
                          long rows, float* out, int* err, int sms, cudaStream_t st,
                          int stall) {
  if (rows <= 0) return cudaSuccess;
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_ws_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SM_TOTAL);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  // one CTA per SM (its shared memory and the 512 TMEM columns of its four chains fill it)
  const long tiles = (rows + 127) / 128;
  const long ctas = (tiles + WS_CH - 1) / WS_CH;
  const long grid = ctas < (long)sms ? ctas : (long)sms;
  k_ws_mlp_tc<<<(unsigned)grid, 128 * WS_CH, SM_TOTAL, st>>>(wpack, params, X, rows, out, err,
                                                            stall);
  return cudaGetLastError();
}

// one training step's kernels (gradient only; the trainer adds Adam)
cudaError_t launch_ws_grad(const float* params, const float* X, const float* t,
                           const long long* idx, int B, WsTrainBuffers& tb, cudaStream_t st) {
  const long HH = (long)H * H;
  const long oW0 = 0, ob0 = H * K, oW1 = ob0 + H, ob1 = oW1 + HH, oW2 = ob1 + H, ob2 = oW2 + HH,
             ow3 = ob2 + H, ob3 = ow3 + H;
  k_gather_rows<<<(B * 4 + 255) / 256, 256, 0, st>>>(X, t, idx, B, tb.Xb, tb.tb);
  const dim3 gf(H / 64, (B + 63) / 64, 1);
  // forward
  k_gemm<false, true, 1><<<gf, 256, 0, st>>>(B, H, K, tb.Xb, K, params + oW0, K, tb.Z0, H,
                                             params + ob0, tb.A0, nullptr, K);
  k_gemm<false, true, 1><<<gf, 256, 0, st>>>(B, H, H, tb.A0, H, params + oW1, H, tb.Z1, H,
                                             params + ob1, tb.A1, nullptr, H);
  k_gemm<false, true, 1><<<gf, 256, 0, st>>>(B, H, H, tb.A1, H, params + oW2, H, tb.Z2, H,
                                             params + ob2, tb.A2, nullptr, H);
  const int nout = (B + 7) / 8;
  k_ws_out<<<nout, 256, 0, st>>>(tb.A2, tb.Z2, params, tb.tb, B, tb.dy, tb.dZ2, tb.loss_part);
  k_sum_f64<<<1, 32, 0, st>>>(tb.loss_part, nout, 1.0 / (double)B, tb.loss);
  // backward: weight gradients over row chunks, data gradients through the layers
  const int chunk = WS_ROW_CHUNK, S = (B + chunk - 1) / chunk;
  float* g = tb.grad;
  auto wgrad = [&](const float* dZ, const float* Ain, int kin, long ow, long ob) {
    const dim3 gw((kin + 63) / 64, H / 64, S);
    k_gemm<true, false, 0><<<gw, 256, 0, st>>>(H, kin, B, dZ, H, Ain, kin, tb.part, kin,
                                               nullptr, nullptr, nullptr, chunk);
    k_sum_partials<<<nblk((long)H * kin), 256, 0, st>>>(tb.part, S, (long)H * kin, g + ow);
    k_colsum<<<dim3((H + 127) / 128, S), 128, 0, st>>>(dZ, B, H, chunk, tb.part);
    k_sum_partials<<<1, 128, 0, st>>>(tb.part, S, H, g + ob);
  };
  // w3, b3: column sums of A2 dy and of dy
  {
    const dim3 gw(1, H / 64, S);
    k_gemm<true, false, 0><<<gw, 256, 0, st>>>(H, 1, B, tb.A2, H, tb.dy, 1, tb.part, 1, nullptr,
                                               nullptr, nullptr, chunk);
    k_sum_partials<<<1, 128, 0, st>>>(tb.part, S, H, g + ow3);
    k_colsum<<<dim3(1, S), 128, 0, st>>>(tb.dy, B, 1, chunk, tb.part);
    k_sum_partials<<<1, 32, 0, st>>>(tb.part, S, 1, g + ob3);
  }
  wgrad(tb.dZ2, tb.A1, H, oW2, ob2);
  k_gemm<false, false, 2><<<gf, 256, 0, st>>>(B, H, H, tb.dZ2, H, params + oW2, H, tb.dZ1, H,
                                              nullptr, nullptr, tb.Z1, H);
  wgrad(tb.dZ1, tb.A0, H, oW1, ob1);
  k_gemm<false, false, 2><<<gf, 256, 0, st>>>(B, H, H, tb.dZ1, H, params + oW1, H, tb.dZ2, H,
                                              nullptr, nullptr, tb.Z0, H);
  wgrad(tb.dZ2, tb.Xb, K, oW0, ob0);
  return cudaGetLastError();
}

cudaError_t launch_ws_adam(float* p, float* m, float* v, const float* g, long n, float lr,
                           int t, cudaStream_t st) {
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - pow(b1, t)), c2 = (float)(1.0 - pow(b2, t));
  k_adam<<<nblk(n), 256, 0, st>>>(p, m, v, g, n, lr, (float)b1, (float)b2, c1, c2, 1e-8f);
  return cudaGetLastError();
}

}  // namespace otgb
