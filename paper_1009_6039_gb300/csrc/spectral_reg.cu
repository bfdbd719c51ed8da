// Register-resident FP32 passes of the preconditioned matvec w = L Lbar^{-1} sigma of
// Strain's method (Sec. 4.2), for power-of-two transform lengths 64..1024.
//
// A transform of length L = 32 T runs in T threads of one warp, each holding 32 elements in
// registers, as two register DFTs with one shared-memory exchange between them (a "two-level"
// transform; the internal twiddles of the 32-point DFT are compile-time constants, the
// exchange twiddles W_L^{t k} come from per-plan tables laid out for contiguous loads):
//
//   forward  (A then B)   thread t holds x[t + T m], m < 32   -> DFT-32 over m,
//                         times W_L^{t ka}, exchange, DFT-T over t
//                         -> thread t holds X[ka + 32 kb], ka = t + T j (j < 32/T), kb < T
//   inverse  (B then A)   the reverse order and sign: from the spectrum distributed as above
//                         to x[t + T m]
//
// The half spectrum of the matvec is stored TRANSPOSED (M/2 x N: entry (k1, k2) at
// k1 * N + k2, the packed DC/Nyquist pair in k1 = 0 as in the standard layout), so the
// column pass reads and writes whole columns contiguously and the row passes exchange it
// through shared-memory tiles of RB rows:
//
//   k_mvT_r2c      sigma rows -> packed half spectrum (transposed)
//   k_mvT_col      per column: forward column FFT, S = rho-bar sigma-hat / (N M), inverse
//                  column FFTs of S (Nyquist channel of column 0 premultiplied by
//                  d11(M/2)), (i s1(k2)) S and s2(k2) S
//   k_mvT_combine  per row: the five complex-to-real transforms (d_xx Q0, d_x Q0, d_x Q1,
//                  Q1, Q2) weighted by a11, b1, 2 a12, b2, a22 and summed into w
#include "spectral.cuh"

namespace otgb {
namespace {

// cos(2 pi j / 32) for j = 0..8
__host__ __device__ constexpr float kcos32(int j) {
  return j == 0   ? 1.0f
         : j == 1 ? 0.98078528040323044913f
         : j == 2 ? 0.92387953251128675613f
         : j == 3 ? 0.83146961230254523708f
         : j == 4 ? 0.70710678118654752440f
         : j == 5 ? 0.55557023301960222474f
         : j == 6 ? 0.38268343236508977173f
         : j == 7 ? 0.19509032201612826785f
                  : 0.0f;
}
// cos and sin of 2 pi j / 32 for any integer j
__host__ __device__ constexpr float cos32_0(int r) {  // r in 0..31
  return r <= 8 ? kcos32(r) : r <= 16 ? -kcos32(16 - r) : r <= 24 ? -kcos32(r - 16)
                                                                   : kcos32(32 - r);
}
__host__ __device__ constexpr float cos32(int j) { return cos32_0(((j % 32) + 32) % 32); }
__host__ __device__ constexpr float sin32(int j) { return cos32(8 - j); }

// z * exp(SIGN 2 pi i j / 32); j is a compile-time constant after unrolling
template <int SIGN>
__device__ __forceinline__ float2 rot32(float2 z, int j) {
  j &= 31;
  if (j == 0) return z;
  if (j == 16) return make_float2(-z.x, -z.y);
  if (j == 8) return mul_si<float, SIGN>(z);
  if (j == 24) return mul_si<float, -SIGN>(z);
  const float c = cos32(j), s = (float)SIGN * sin32(j);
  return make_float2(z.x * c - z.y * s, z.x * s + z.y * c);
}

// In-register DFT of size R (natural order in and out), kernel exp(SIGN 2 pi i n k / R).
// R = 16, 32 as 4 x (R/4): DFT-(R/4) over n = a + 4 b for each a, twiddle W_R^{a kb},
// DFT-4 over a; output index kb + (R/4) ka.
template <int R, int SIGN> struct RDft {
  static_assert(R == 16 || R == 32, "RDft: R = 2, 4, 8, 16 or 32");
  static constexpr int A = 4, B = R / 4;
  __device__ __forceinline__ static void run(float2* v);
};
template <int SIGN> struct RDft<1, SIGN> {
  __device__ __forceinline__ static void run(float2*) {}
};
template <int SIGN> struct RDft<2, SIGN> {
  __device__ __forceinline__ static void run(float2* v) { Bfly<float, 2, SIGN>::run(v); }
};
template <int SIGN> struct RDft<4, SIGN> {
  __device__ __forceinline__ static void run(float2* v) { Bfly<float, 4, SIGN>::run(v); }
};
template <int SIGN> struct RDft<8, SIGN> {
  __device__ __forceinline__ static void run(float2* v) { Bfly<float, 8, SIGN>::run(v); }
};
template <int R, int SIGN>
__device__ __forceinline__ void RDft<R, SIGN>::run(float2* v) {
  float2 tmp[R];
#pragma unroll
  for (int a = 0; a < A; ++a) {
    float2 u[B];
#pragma unroll
    for (int b = 0; b < B; ++b) u[b] = v[a + A * b];
    RDft<B, SIGN>::run(u);
#pragma unroll
    for (int kb = 0; kb < B; ++kb) tmp[a + A * kb] = rot32<SIGN>(u[kb], a * kb * (32 / R));
  }
#pragma unroll
  for (int kb = 0; kb < B; ++kb) {
    float2 u[A];
#pragma unroll
    for (int a = 0; a < A; ++a) u[a] = tmp[a + A * kb];
    RDft<A, SIGN>::run(u);
#pragma unroll
    for (int ka = 0; ka < A; ++ka) v[kb + B * ka] = u[ka];
  }
}

// exchange buffer of one transform: T rows of 32 (+1 padding) elements
template <int L> __host__ __device__ constexpr int xbuf_len() { return (L / 32) * 33; }

// Forward two-level transform of length L (kernel exp(-2 pi i n k / L)).
// In: thread t (< T) holds x[t + T m] at v[m].  Out: X[ka + 32 kb] at v[j T + kb] for
// ka = t + T j.  twA[ka T + t] = W_L^{t ka}.  All 32 lanes of the warp must call it.
template <int L>
__device__ __forceinline__ void fft2l_fwd(float2 (&v)[32], float2* sbuf, int t,
                                          const float2* __restrict__ twA) {
  constexpr int T = L / 32;
  RDft<32, -1>::run(v);
#pragma unroll
  for (int ka = 1; ka < 32; ++ka) v[ka] = cmul<float>(v[ka], twA[ka * T + t]);
#pragma unroll
  for (int ka = 0; ka < 32; ++ka) sbuf[t * 33 + ka] = v[ka];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 32 / T; ++j) {
    const int ka = t + T * j;
    float2 u[T];
#pragma unroll
    for (int tt = 0; tt < T; ++tt) u[tt] = sbuf[tt * 33 + ka];
    RDft<T, -1>::run(u);
#pragma unroll
    for (int kb = 0; kb < T; ++kb) v[j * T + kb] = u[kb];
  }
  __syncwarp();
}

// Inverse two-level transform (kernel exp(+2 pi i n k / L), unnormalised): the reverse of
// fft2l_fwd.  In: X[ka + 32 kb] at v[j T + kb], ka = t + T j.  Out: x[t + T m] at v[m].
// twB[tt * 32 + ka] = W_L^{tt ka} (conjugated here).
template <int L>
__device__ __forceinline__ void fft2l_inv(float2 (&v)[32], float2* sbuf, int t,
                                          const float2* __restrict__ twB) {
  constexpr int T = L / 32;
#pragma unroll
  for (int j = 0; j < 32 / T; ++j) {
    const int ka = t + T * j;
    float2 u[T];
#pragma unroll
    for (int kb = 0; kb < T; ++kb) u[kb] = v[j * T + kb];
    RDft<T, +1>::run(u);
#pragma unroll
    for (int tt = 0; tt < T; ++tt) {
      const float2 w = twB[tt * 32 + ka];
      sbuf[tt * 33 + ka] =
          make_float2(u[tt].x * w.x + u[tt].y * w.y, u[tt].y * w.x - u[tt].x * w.y);
    }
  }
  __syncwarp();
#pragma unroll
  for (int ka = 0; ka < 32; ++ka) v[ka] = sbuf[t * 33 + ka];
  __syncwarp();
  RDft<32, +1>::run(v);
}

// rows per block of the row passes, columns per block of the column pass
template <int L> __host__ __device__ constexpr int mv_rows() {
  return (L / 32) >= 16 ? 4 : 64 / (L / 32);
}

// ---------------------------------------------------------------------------------------
// Row pass: sigma (N x M real, M = 2L) -> packed half spectrum, transposed (specT[k][row]).
// The real row is read as L complex z[n] = x[2n] + i x[2n+1]; after the length-L transform
// X_k = E_k + W_M^k O_k with E_k = (Z_k + conj Z_{L-k}) / 2, O_k = -i (Z_k - conj Z_{L-k}) / 2,
// and X_0 packed as (Z_0.x + Z_0.y) + i (Z_0.x - Z_0.y) = X(0) + i X(M/2).
// ---------------------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(128)
    k_mvT_r2c(const float* __restrict__ xbase, size_t x_stride, const int* __restrict__ jptr,
              const double* __restrict__ scale, float2* __restrict__ specT, int N,
              const float2* __restrict__ twA, const float2* __restrict__ twM,
              const int* __restrict__ skip) {
  if (skip && *skip) return;
  constexpr int T = L / 32, RB = mv_rows<L>(), M = 2 * L, SB = xbuf_len<L>(), NB = L + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  const int g = threadIdx.x / T, t = threadIdx.x - g * T;
  const int row0 = blockIdx.x * RB, row = row0 + g;
  const bool active = row < N;
  float2* sbuf = sm + g * SB;
  float2* nat = sm + RB * SB + g * NB;
  const int jv = jptr ? *jptr : 0;
  const float* x = xbase + (size_t)jv * x_stride;
  const float sc = scale ? (float)scale[jv] : 1.f;
  const float2* xr = reinterpret_cast<const float2*>(x + (size_t)(active ? row : 0) * M);
  float2 v[32];
#pragma unroll
  for (int m = 0; m < 32; ++m) {
    const float2 z = active ? xr[t + T * m] : make_float2(0.f, 0.f);
    v[m] = make_float2(z.x * sc, z.y * sc);
  }
  fft2l_fwd<L>(v, sbuf, t, twA);
#pragma unroll
  for (int j = 0; j < 32 / T; ++j)
#pragma unroll
    for (int kb = 0; kb < T; ++kb) nat[t + T * j + 32 * kb] = v[j * T + kb];
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const int k = t + T * i;
    const float2 zk = nat[k], zm = nat[(L - k) & (L - 1)];
    if (k == 0) {
      v[i] = make_float2(zk.x + zk.y, zk.x - zk.y);
    } else {
      const float2 Ev = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      const float2 Ov = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
      v[i] = cadd<float>(Ev, cmul<float>(twM[k], Ov));
    }
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 32; ++i) nat[t + T * i] = v[i];
  __syncthreads();
  // transposed store: RB consecutive rows of each frequency k1 are contiguous
  for (int idx = threadIdx.x; idx < L * RB; idx += blockDim.x) {
    const int k = idx / RB, r = idx - k * RB;
    if (row0 + r < N) specT[(size_t)k * N + row0 + r] = sm[RB * SB + r * NB + k];
  }
}

// ---------------------------------------------------------------------------------------
// Column pass (column length NL = N): CB columns per block, three groups of T = NL/32
// threads per column (one warp per group and column set).  Group 0 runs the forward column
// transform and forms S = rho-bar sigma-hat / (N M) in shared memory; after one block
// barrier group p runs inverse transform p (Q0 = S, Q1 = (i s1(k2)) S, Q2 = s2(k2) S), so
// the three inverse transforms of a column run at the same time.
// ---------------------------------------------------------------------------------------
template <int NL> __host__ __device__ constexpr int mv_cols() { return 32 / (NL / 32); }

template <int NL>
__global__ void __launch_bounds__(96)
    k_mvT_col(const float2* __restrict__ specT, float2* __restrict__ o0,
              float2* __restrict__ o1, float2* __restrict__ o2, int M, float inv_nm,
              const float2* __restrict__ twA, const float2* __restrict__ twB,
              const DevScalars* __restrict__ sc, const int* __restrict__ skip,
              const float2* __restrict__ symx, const float2* __restrict__ symy) {
  if (skip && *skip) return;
  constexpr int T = NL / 32, CB = mv_cols<NL>(), SB = xbuf_len<NL>();
  static_assert(SB >= NL && CB * T == 32, "one warp per group; a column fits the buffer");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  const int Lc = M / 2;
  const int grp = threadIdx.x >> 5, rem = threadIdx.x & 31;
  const int c = rem / T, t = rem - c * T;
  const int col = blockIdx.x * CB + c;
  const bool active = col < Lc;
  float2* sbuf = sm + (grp * CB + c) * SB;
  float2* sS = sm + 3 * CB * SB + c * NL;  // S of this column (natural order k2)
  float2* s0buf = sm + CB * (3 * SB + NL);  // Q0 of column 0 (its Nyquist channel premultiplied)
  if (grp == 0) {
    const float2* src = specT + (size_t)(active ? col : 0) * NL;
    float2 v[32];
#pragma unroll
    for (int m = 0; m < 32; ++m) v[m] = active ? src[t + T * m] : make_float2(0.f, 0.f);
    fft2l_fwd<NL>(v, sbuf, t, twA);
    // thread t holds sigma-hat(k1 = col, k2 = k) at v[j T + kb], k = t + T j + 32 kb.
    // Column 0 carries the two real columns k1 = 0 and k1 = M/2 as A + i B: unpacking needs
    // the entry at N - k, which another thread holds (every column exchanges, so that all
    // lanes of the warp take the same path).
#pragma unroll
    for (int j = 0; j < 32 / T; ++j)
#pragma unroll
      for (int kb = 0; kb < T; ++kb) sbuf[t + T * j + 32 * kb] = v[j * T + kb];
    __syncwarp();
    float ab[5];
#pragma unroll
    for (int a = 0; a < 5; ++a) ab[a] = (float)sc->abar[a];
    const float2 sxc = symx[active ? col : 0];
    const float2 sx0 = symx[0], sxn = symx[M / 2];
    const float d11n = sxn.y;
#pragma unroll
    for (int j = 0; j < 32 / T; ++j) {
#pragma unroll
      for (int kb = 0; kb < T; ++kb) {
        const int k = t + T * j + 32 * kb;
        const float2 z = v[j * T + kb];
        const float2 sy = symy[k];
        if (col == 0) {
          const float2 q = sbuf[(NL - k) & (NL - 1)];
          float2 A = make_float2(0.5f * (z.x + q.x), 0.5f * (z.y - q.y));
          float2 B = make_float2(0.5f * (z.y + q.y), -0.5f * (z.x - q.x));
          A = cmul<float>(rho_bar<float>(ab, sx0, sy), A);
          B = cmul<float>(rho_bar<float>(ab, sxn, sy), B);
          const float2 Bn = cscale<float>(B, d11n);
          s0buf[k] = cscale<float>(make_float2(A.x - Bn.y, A.y + Bn.x), inv_nm);
          sS[k] = cscale<float>(make_float2(A.x - B.y, A.y + B.x), inv_nm);
        } else {
          sS[k] = cscale<float>(cmul<float>(rho_bar<float>(ab, sxc, sy), z), inv_nm);
        }
      }
    }
  }
  __syncthreads();
  // inverse transform p = grp of this column; each thread reads the entries of S it would
  // hold in the transform's input distribution
  float2 u[32];
#pragma unroll
  for (int j = 0; j < 32 / T; ++j) {
#pragma unroll
    for (int kb = 0; kb < T; ++kb) {
      const int k = t + T * j + 32 * kb;
      const float2 s = sS[k];
      if (grp == 0) {
        u[j * T + kb] = (col == 0) ? s0buf[k] : s;
      } else {
        const float2 sy = symy[k];
        u[j * T + kb] =
            (grp == 1) ? make_float2(-sy.x * s.y, sy.x * s.x) : cscale<float>(s, sy.y);
      }
    }
  }
  fft2l_inv<NL>(u, sbuf, t, twB);
  if (active) {
    float2* dst = (grp == 0 ? o0 : (grp == 1 ? o1 : o2)) + (size_t)col * NL;
#pragma unroll
    for (int m = 0; m < 32; ++m) dst[t + T * m] = u[m];
  }
}

// ---------------------------------------------------------------------------------------
// Row combine: the five complex-to-real row transforms of the transposed Q0, Q1, Q2 and
// w = a11 d_xx + b1 d_x (on Q0) + 2 a12 d_x + b2 (on Q1) + a22 (on Q2).  The complex-to-real
// step of a packed row: Z_k = (X_k + conj X_{L-k}) + i (X_k - conj X_{L-k}) conj(W_M^k)
// (Z_0 = (X_0.x + X_0.y) + i (X_0.x - X_0.y)); the inverse length-L transform of Z gives the
// real pairs (y[2n], y[2n+1]).  RB = 32/T rows per block and five groups (one warp each),
// one per term: the five transforms of a row run at the same time, each group leaves its
// weighted term in its exchange buffer, and the block sums them.
// ---------------------------------------------------------------------------------------
template <int L> __host__ __device__ constexpr int mv_rows5() { return 32 / (L / 32); }

template <int L>
__global__ void __launch_bounds__(160)
    k_mvT_combine(const float2* __restrict__ q0T, const float2* __restrict__ q1T,
                  const float2* __restrict__ q2T, const float* __restrict__ coef,
                  float* __restrict__ out, int N, const float2* __restrict__ twB,
                  const float2* __restrict__ twM, const int* __restrict__ skip,
                  const float2* __restrict__ symx) {
  if (skip && *skip) return;
  constexpr int T = L / 32, RB = mv_rows5<L>(), M = 2 * L, SB = xbuf_len<L>(), NB = L + 1;
  static_assert(RB * T == 32 && SB >= L, "one warp per term group; a row fits the buffer");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);
  const int term = threadIdx.x >> 5, rem = threadIdx.x & 31;
  const int g = rem / T, t = rem - g * T;
  const int row0 = blockIdx.x * RB, row = row0 + g;
  const bool active = row < N;
  float2* qs = sm;                                   // [plane][row][NB]
  float2* sbuf = sm + 3 * RB * NB + (term * RB + g) * SB;
  for (int idx = threadIdx.x; idx < 3 * L * RB; idx += blockDim.x) {
    const int p = idx / (L * RB), r0 = idx - p * (L * RB);
    const int k = r0 / RB, r = r0 - k * RB;
    const float2* q = p == 0 ? q0T : (p == 1 ? q1T : q2T);
    qs[(p * RB + r) * NB + k] =
        (row0 + r < N) ? q[(size_t)k * N + row0 + r] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  // term: source plane, row symbol kind (0: 1, 1: d/dx, 2: d2/dx2), coefficient plane
  const int plane = term < 2 ? 0 : (term < 4 ? 1 : 2);
  const int kind = term == 0 ? 2 : ((term == 1 || term == 2) ? 1 : 0);
  const int cidx = term == 0 ? 0 : (term == 1 ? 3 : (term == 2 ? 1 : (term == 3 ? 4 : 2)));
  const float mult = term == 2 ? 2.f : 1.f;
  const float2* qr = qs + (plane * RB + g) * NB;
  float2 v[32];
#pragma unroll
  for (int j = 0; j < 32 / T; ++j) {
#pragma unroll
    for (int kb = 0; kb < T; ++kb) {
      const int k = t + T * j + 32 * kb;
      const float2 X = row_symbol_apply<float>(qr[k], k, kind, symx);
      float2 Z;
      if (k == 0) {
        Z = make_float2(X.x + X.y, X.x - X.y);
      } else {
        const float2 Xm = row_symbol_apply<float>(qr[L - k], L - k, kind, symx);
        const float2 Ev = make_float2(X.x + Xm.x, X.y - Xm.y);
        const float2 dv = make_float2(X.x - Xm.x, X.y + Xm.y);
        const float2 Ov = cmul<float>(dv, cconj<float>(twM[k]));
        Z = make_float2(Ev.x - Ov.y, Ev.y + Ov.x);
      }
      v[j * T + kb] = Z;
    }
  }
  fft2l_inv<L>(v, sbuf, t, twB);
  // the weighted term into this group's exchange buffer (free after the transform)
  const size_t P = (size_t)N * M;
  const float2* cr =
      reinterpret_cast<const float2*>(coef + (size_t)cidx * P + (size_t)(active ? row : 0) * M);
#pragma unroll
  for (int m = 0; m < 32; ++m) {
    const float2 a = active ? cr[t + T * m] : make_float2(0.f, 0.f);
    sbuf[t + T * m] = make_float2(mult * a.x * v[m].x, mult * a.y * v[m].y);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < RB * L; idx += blockDim.x) {
    const int r = idx / L, n = idx - r * L;
    if (row0 + r >= N) continue;
    float2 sum = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const float2 y = sm[3 * RB * NB + (q * RB + r) * SB + n];
      sum.x += y.x;
      sum.y += y.y;
    }
    reinterpret_cast<float2*>(out + (size_t)(row0 + r) * M)[n] = sum;
  }
}

// ---------------------------------------------------------------------------------------
template <int L>
cudaError_t r2c_L(const float* x, size_t xs, const int* jptr, const double* scale,
                  float2* specT, int N, const SpecTables& tb, const int* skip,
                  cudaStream_t st) {
  constexpr int T = L / 32, RB = mv_rows<L>();
  const size_t sm = (size_t)RB * (xbuf_len<L>() + L + 1) * sizeof(float2);
  cudaError_t e = prepare_launch(k_mvT_r2c<L>, RB * T, sm);
  if (e != cudaSuccess) return e;
  k_mvT_r2c<L><<<(N + RB - 1) / RB, RB * T, sm, st>>>(
      x, xs, jptr, scale, specT, N, (const float2*)tb.t2rA, (const float2*)tb.twM, skip);
  return cudaGetLastError();
}

template <int NL>
cudaError_t col_L(const float2* specT, float2* o0, float2* o1, float2* o2, int M,
                  const SpecTables& tb, const DevScalars* sc, const int* skip,
                  cudaStream_t st) {
  constexpr int CB = mv_cols<NL>();
  const int Lc = M / 2;
  const size_t sm = ((size_t)CB * (3 * xbuf_len<NL>() + NL) + NL) * sizeof(float2);
  cudaError_t e = prepare_launch(k_mvT_col<NL>, 96, sm);
  if (e != cudaSuccess) return e;
  k_mvT_col<NL><<<(Lc + CB - 1) / CB, 96, sm, st>>>(
      specT, o0, o1, o2, M, (float)(1.0 / ((double)NL * (double)M)), (const float2*)tb.t2cA,
      (const float2*)tb.t2cB, sc, skip, (const float2*)tb.symx, (const float2*)tb.symy);
  return cudaGetLastError();
}

template <int L>
cudaError_t combine_L(const float2* q0T, const float2* q1T, const float2* q2T,
                      const float* coef, float* out, int N, const SpecTables& tb,
                      const int* skip, cudaStream_t st) {
  constexpr int RB = mv_rows5<L>();
  const size_t sm = (size_t)RB * (3 * (L + 1) + 5 * xbuf_len<L>()) * sizeof(float2);
  cudaError_t e = prepare_launch(k_mvT_combine<L>, 160, sm);
  if (e != cudaSuccess) return e;
  k_mvT_combine<L><<<(N + RB - 1) / RB, 160, sm, st>>>(
      q0T, q1T, q2T, coef, out, N, (const float2*)tb.t2rB, (const float2*)tb.twM, skip,
      (const float2*)tb.symx);
  return cudaGetLastError();
}

bool reg_len(int L) { return L >= 64 && L <= 1024 && (L & (L - 1)) == 0; }

}  // namespace

bool mvT_supported(int N, int M) { return reg_len(N) && reg_len(M / 2); }

cudaError_t launch_mvT_r2c(const float* x, size_t xs, const int* jptr, const double* scale,
                           float2* specT, int N, int M, const SpecTables& tb,
                           const int* skip, cudaStream_t st) {
  switch (M / 2) {
    case 64: return r2c_L<64>(x, xs, jptr, scale, specT, N, tb, skip, st);
    case 128: return r2c_L<128>(x, xs, jptr, scale, specT, N, tb, skip, st);
    case 256: return r2c_L<256>(x, xs, jptr, scale, specT, N, tb, skip, st);
    case 512: return r2c_L<512>(x, xs, jptr, scale, specT, N, tb, skip, st);
    case 1024: return r2c_L<1024>(x, xs, jptr, scale, specT, N, tb, skip, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_mvT_col(const float2* specT, float2* o0, float2* o1, float2* o2, int N,
                           int M, const SpecTables& tb, const DevScalars* sc,
                           const int* skip, cudaStream_t st) {
  switch (N) {
    case 64: return col_L<64>(specT, o0, o1, o2, M, tb, sc, skip, st);
    case 128: return col_L<128>(specT, o0, o1, o2, M, tb, sc, skip, st);
    case 256: return col_L<256>(specT, o0, o1, o2, M, tb, sc, skip, st);
    case 512: return col_L<512>(specT, o0, o1, o2, M, tb, sc, skip, st);
    case 1024: return col_L<1024>(specT, o0, o1, o2, M, tb, sc, skip, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_mvT_combine(const float2* q0T, const float2* q1T, const float2* q2T,
                               const float* coef, float* out, int N, int M,
                               const SpecTables& tb, const int* skip, cudaStream_t st) {
  switch (M / 2) {
    case 64: return combine_L<64>(q0T, q1T, q2T, coef, out, N, tb, skip, st);
    case 128: return combine_L<128>(q0T, q1T, q2T, coef, out, N, tb, skip, st);
    case 256: return combine_L<256>(q0T, q1T, q2T, coef, out, N, tb, skip, st);
    case 512: return combine_L<512>(q0T, q1T, q2T, coef, out, N, tb, skip, st);
    case 1024: return combine_L<1024>(q0T, q1T, q2T, coef, out, N, tb, skip, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace otgb
