// Finite-difference comparison path (Sec. 4.1): the linear equation of each Newton step,
// L theta = a11 theta_xx + 2 a12 theta_xy + a22 theta_yy + b1 theta_x + b2 theta_y = h,
// discretised with second-order centred differences into A, made square and invertible by
// adding the extra equation sum theta = 0 to every row (A~ = A + 1 1^T), and solved from
// theta = 0 by biconjugate gradients without preconditioning.
//
// One BiCG iteration is three kernels, each skipping itself once the iteration has stopped
// (so the host can launch fixed-size chunks and read the state once per chunk):
//   k_bicg_matvec  q = A~ p, q* = A~^T p*, den = (q, p*)           -> alpha = rho / den
//   k_bicg_update  x += alpha p, r -= alpha q, r* -= alpha q*,
//                  rho' = (r, r*), ||r||^2                          -> stop test, beta
//   k_bicg_dir     p = r + beta p, p* = r* + beta p*, sum p, sum p* (for the next A~ p)
// The transpose is applied in divergence form: A^T y = D_xx(a11 y) + D_xy(2 a12 y) +
// D_yy(a22 y) - D_x(b1 y) - D_y(b2 y) (the second differences are symmetric, the centred
// first differences antisymmetric).  All arithmetic is FP64 (the paper's comparison path;
// the Fourier method is the fast one).  Grid: row-major N x M, x along the row index j
// (spacing 1/M), y along i (spacing 1/N), periodic.
#include <math.h>

#include "otgb_internal.cuh"
#include "reduce.cuh"

namespace otgb {

namespace {

struct Nbr {
  long c, xm, xp, ym, yp, pp, pm, mp, mm;  // centre, +-x, +-y, (y, x) diagonals
};

__device__ __forceinline__ Nbr neighbours(long p, int N, int M) {
  const int i = (int)(p / M), j = (int)(p - (long)i * M);
  const int jm = j == 0 ? M - 1 : j - 1, jp = j == M - 1 ? 0 : j + 1;
  const int im = i == 0 ? N - 1 : i - 1, ip = i == N - 1 ? 0 : i + 1;
  const long ri = (long)i * M, rm = (long)im * M, rp = (long)ip * M;
  return Nbr{p, ri + jm, ri + jp, rm + j, rp + j, rp + jp, rp + jm, rm + jp, rm + jm};
}

// b = h when given, else (F_raw + shift) / tau: the Newton step's right-hand side
__global__ void k_bicg_init(const double* __restrict__ Fraw, const double* __restrict__ h,
                            double* __restrict__ x, double* __restrict__ r,
                            double* __restrict__ rs, double* __restrict__ pv,
                            double* __restrict__ ps, long P, double* partials,
                            DevScalars* sc, int max_iters) {
  const double shift = sc->shift, inv_tau = 1.0 / sc->tau;
  double v[2] = {0.0, 0.0};
  const int kind[2] = {0, 0};
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x) {
    const double b = h ? h[p] : (Fraw[p] + shift) * inv_tau;
    x[p] = 0.0;
    r[p] = b;
    rs[p] = b;
    pv[p] = b;
    ps[p] = b;
    v[0] += b;
    v[1] += b * b;
  }
  block_reduce<2>(v, kind);
  if (!publish_partials<2>(v, partials, &sc->ticket[TK_BICG])) return;
  reduce_partials<2>(v, kind, partials, gridDim.x);
  if (threadIdx.x == 0) {
    sc->bicg_sp = v[0];
    sc->bicg_sps = v[0];
    sc->bicg_b2 = v[1];
    sc->bicg_r2 = v[1];
    sc->bicg_rho = v[1];
    sc->bicg_iters = 0;
    sc->bicg_max = max_iters;
    sc->bicg_done = v[1] == 0.0 ? 1 : 0;
    sc->bicg_status = v[1] == 0.0 ? 0 : 1;
    sc->ticket[TK_BICG] = 0;
  }
}

__global__ void k_bicg_matvec(const double* __restrict__ coef, const double* __restrict__ pv,
                              const double* __restrict__ ps, double* __restrict__ q,
                              double* __restrict__ qs, int N, int M, double* partials,
                              DevScalars* sc) {
  if (sc->bicg_done) return;
  const long P = (long)N * M;
  const double* __restrict__ a11 = coef;
  const double* __restrict__ a12 = coef + P;
  const double* __restrict__ a22 = coef + 2 * P;
  const double* __restrict__ b1 = coef + 3 * P;
  const double* __restrict__ b2 = coef + 4 * P;
  const double mm2 = (double)M * M, nn2 = (double)N * N, hx = 0.5 * M, hy = 0.5 * N;
  const double xy = 0.25 * (double)N * M;
  const double sp = sc->bicg_sp, sps = sc->bicg_sps;
  double v[1] = {0.0};
  const int kind[1] = {0};
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x) {
    const Nbr n = neighbours(p, N, M);
    // A p with the coefficients of this row
    const double pc = pv[n.c];
    const double pxx = (pv[n.xp] - 2.0 * pc + pv[n.xm]) * mm2;
    const double pyy = (pv[n.yp] - 2.0 * pc + pv[n.ym]) * nn2;
    const double pxy = (pv[n.pp] - pv[n.pm] - pv[n.mp] + pv[n.mm]) * xy;
    const double px = (pv[n.xp] - pv[n.xm]) * hx;
    const double py = (pv[n.yp] - pv[n.ym]) * hy;
    const double qv = a11[n.c] * pxx + 2.0 * a12[n.c] * pxy + a22[n.c] * pyy + b1[n.c] * px +
                      b2[n.c] * py + sp;
    // A^T p* in divergence form: the differences of (coefficient x p*)
    const double sc_ = ps[n.c];
    const double txx =
        (a11[n.xp] * ps[n.xp] - 2.0 * a11[n.c] * sc_ + a11[n.xm] * ps[n.xm]) * mm2;
    const double tyy =
        (a22[n.yp] * ps[n.yp] - 2.0 * a22[n.c] * sc_ + a22[n.ym] * ps[n.ym]) * nn2;
    const double txy = 2.0 *
                       (a12[n.pp] * ps[n.pp] - a12[n.pm] * ps[n.pm] - a12[n.mp] * ps[n.mp] +
                        a12[n.mm] * ps[n.mm]) *
                       xy;
    const double tx = (b1[n.xp] * ps[n.xp] - b1[n.xm] * ps[n.xm]) * hx;
    const double ty = (b2[n.yp] * ps[n.yp] - b2[n.ym] * ps[n.ym]) * hy;
    q[p] = qv;
    qs[p] = txx + txy + tyy - tx - ty + sps;
    v[0] += qv * sc_;
  }
  block_reduce<1>(v, kind);
  if (!publish_partials<1>(v, partials, &sc->ticket[TK_BICG])) return;
  reduce_partials<1>(v, kind, partials, gridDim.x);
  if (threadIdx.x == 0) {
    if (v[0] == 0.0) {
      sc->bicg_done = 1;
      sc->bicg_status = 2;  // breakdown
    } else {
      sc->bicg_alpha = sc->bicg_rho / v[0];
    }
    sc->ticket[TK_BICG] = 0;
  }
}

__global__ void k_bicg_update(double* __restrict__ x, double* __restrict__ r,
                              double* __restrict__ rs, const double* __restrict__ pv,
                              const double* __restrict__ q, const double* __restrict__ qs,
                              long P, double* partials, DevScalars* sc) {
  if (sc->bicg_done) return;
  const double alpha = sc->bicg_alpha;
  double v[2] = {0.0, 0.0};
  const int kind[2] = {0, 0};
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x) {
    x[p] += alpha * pv[p];
    const double rn = r[p] - alpha * q[p];
    const double rsn = rs[p] - alpha * qs[p];
    r[p] = rn;
    rs[p] = rsn;
    v[0] += rn * rsn;
    v[1] += rn * rn;
  }
  block_reduce<2>(v, kind);
  if (!publish_partials<2>(v, partials, &sc->ticket[TK_BICG])) return;
  reduce_partials<2>(v, kind, partials, gridDim.x);
  if (threadIdx.x == 0) {
    const int it = sc->bicg_iters + 1;
    sc->bicg_iters = it;
    sc->bicg_r2 = v[1];
    if (v[1] <= sc->eta * sc->eta * sc->bicg_b2) {
      sc->bicg_done = 1;
      sc->bicg_status = 0;
    } else if (it >= sc->bicg_max) {
      sc->bicg_done = 1;
      sc->bicg_status = 1;
    } else if (v[0] == 0.0) {
      sc->bicg_done = 1;
      sc->bicg_status = 2;
    } else {
      sc->bicg_beta = v[0] / sc->bicg_rho;
      sc->bicg_rho = v[0];
    }
    sc->ticket[TK_BICG] = 0;
  }
}

__global__ void k_bicg_dir(const double* __restrict__ r, const double* __restrict__ rs,
                           double* __restrict__ pv, double* __restrict__ ps, long P,
                           double* partials, DevScalars* sc) {
  if (sc->bicg_done) return;
  const double beta = sc->bicg_beta;
  double v[2] = {0.0, 0.0};
  const int kind[2] = {0, 0};
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x) {
    const double a = r[p] + beta * pv[p];
    const double b = rs[p] + beta * ps[p];
    pv[p] = a;
    ps[p] = b;
    v[0] += a;
    v[1] += b;
  }
  block_reduce<2>(v, kind);
  if (!publish_partials<2>(v, partials, &sc->ticket[TK_BICG])) return;
  reduce_partials<2>(v, kind, partials, gridDim.x);
  if (threadIdx.x == 0) {
    sc->bicg_sp = v[0];
    sc->bicg_sps = v[1];
    sc->ticket[TK_BICG] = 0;
  }
}

// y = A~ x (transpose = 0) or A~^T x (1), with sum x from a first pass
__global__ void k_fd_sum(const double* __restrict__ x, long P, double* partials,
                         DevScalars* sc) {
  double v[1] = {0.0};
  const int kind[1] = {0};
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x)
    v[0] += x[p];
  block_reduce<1>(v, kind);
  if (!publish_partials<1>(v, partials, &sc->ticket[TK_BICG])) return;
  reduce_partials<1>(v, kind, partials, gridDim.x);
  if (threadIdx.x == 0) {
    sc->bicg_sp = v[0];
    sc->bicg_sps = v[0];
    sc->ticket[TK_BICG] = 0;
  }
}

// u_out = u_in + s theta
__global__ void k_axpy_to(const double* __restrict__ u_in, const double* __restrict__ th,
                          double s, double* __restrict__ u_out, long P) {
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P;
       p += (long)gridDim.x * blockDim.x)
    u_out[p] = u_in[p] + s * th[p];
}

int fd_blocks() {
  static int nb = 0;
  if (nb == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    nb = (sms > 0 ? sms : 148) * 4;
  }
  return nb;
}

}  // namespace

cudaError_t launch_bicg_init(const double* Fraw, const double* h, FdBufs b, long P,
                             double* partials, DevScalars* sc, int max_iters,
                             cudaStream_t st) {
  k_bicg_init<<<fd_blocks(), 256, 0, st>>>(Fraw, h, b.x, b.r, b.rs, b.p, b.ps, P, partials,
                                           sc, max_iters);
  return cudaGetLastError();
}

cudaError_t launch_bicg_iteration(const double* coef, FdBufs b, int N, int M,
                                  double* partials, DevScalars* sc, cudaStream_t st) {
  const long P = (long)N * M;
  const int nb = fd_blocks();
  k_bicg_matvec<<<nb, 256, 0, st>>>(coef, b.p, b.ps, b.q, b.qs, N, M, partials, sc);
  k_bicg_update<<<nb, 256, 0, st>>>(b.x, b.r, b.rs, b.p, b.q, b.qs, P, partials, sc);
  k_bicg_dir<<<nb, 256, 0, st>>>(b.r, b.rs, b.p, b.ps, P, partials, sc);
  return cudaGetLastError();
}

cudaError_t launch_fd_apply(const double* coef, const double* x, int transpose, double* y,
                            double* tmp, int N, int M, double* partials, DevScalars* sc,
                            cudaStream_t st) {
  const long P = (long)N * M;
  const int nb = fd_blocks();
  // the matvec kernel forms A~ p and A~^T p* together: pass x as both and keep the one
  // asked for (the other goes to tmp); with bicg_done cleared and rho = 0
  k_fd_sum<<<nb, 256, 0, st>>>(x, P, partials, sc);
  k_bicg_matvec<<<nb, 256, 0, st>>>(coef, x, x, transpose ? tmp : y, transpose ? y : tmp, N,
                                    M, partials, sc);
  return cudaGetLastError();
}

cudaError_t launch_axpy_to(const double* u_in, const double* th, double s, double* u_out,
                           long P, cudaStream_t st) {
  k_axpy_to<<<fd_blocks(), 256, 0, st>>>(u_in, th, s, u_out, P);
  return cudaGetLastError();
}

}  // namespace otgb
