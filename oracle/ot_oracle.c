/*
 * ot_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for the damped-Newton
 * Monge-Ampere solver of periodic L2 optimal transport (Saumier, Agueh & Khouider,
 * "An efficient numerical algorithm for the L2 optimal transport problem with
 * applications to image processing", arXiv:1009.6039).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  The CUDA product path never calls it and
 * shares no code, header, table or constant generator with it.
 *
 * Every routine follows the paper's steps in the paper's order, with no blocking, fusion
 * or reordering:
 *   - Sec. 3.1, Eq. (ma2)         : M(u) = g(x + grad u) det(I + D^2 u)
 *   - Sec. 3.1, Eq. (linearmaeq)  : D_u M . theta = g Tr(Adj(I+D^2u) D^2 theta)
 *                                    + det(I+D^2u) grad g . grad theta
 *   - Sec. 3.1, Eq. (linma)       : damped Newton, u_{n+1} = u_n + theta_n,
 *                                    D_{u_n}M theta_n = (f - f_n)/tau, int theta_n = 0
 *   - Sec. 4 (intro)              : N x M periodic grid, 4th-order centred differences for
 *                                    grad u and D^2 u, interpolation of g, Eq. (translation)
 *   - Sec. 4.2, Eq. (fouriersystem): Strain's split L Lbar^{-1} sigma = h, Lbar theta = sigma;
 *                                    symbol rho-bar(k); alpha_ij, beta_i by inverse FFTs;
 *                                    restarted GMRES(m); averages by Simpson's rule
 *   - Sec. 4.1                    : the comparison path: second-order centred differences
 *                                    of theta, the augmented system A~ = A + 1 1^T, BiCG
 *
 * Readings where the paper is silent (each listed in the design notes of the repository):
 *   - stencils: D1 = (-u[+2] + 8u[+1] - 8u[-1] + u[-2]) / (12h),
 *               D2 = (-u[+2] + 16u[+1] - 30u + 16u[-1] - u[-2]) / (12h^2),
 *               mixed u_xy = D1_x applied to D1_y (tensor product);
 *   - g at displaced points: periodic cubic B-spline interpolant of the grid g (prefilter by
 *     a cyclic tridiagonal solve per axis), grad g = exact gradient of that interpolant;
 *     the displaced point in grid units is (j + M u_x, i + N u_y), cell = floor, wrapped;
 *   - Nyquist: first-derivative symbols vanish at k = L/2, second-derivative symbols are
 *     -(2 pi k)^2 there, mixed symbols are the product of first-derivative symbols;
 *   - Simpson on a periodic grid: weights (2/3, 4/3, 2/3, ...)/L per axis (L even);
 *   - GMRES: zero initial guess, modified Gram-Schmidt Arnoldi, Givens rotations, stop
 *     when the estimated residual norm <= eta * ||h||_2, explicit residual at restart;
 *   - Newton stop: max |f - f~_n| < tol evaluated before each solve;
 *   - inputs: Eq. (translation) applied to f and g on entry (Sec. 5.2 does this to images).
 *
 * Grid convention: row-major u[i*M + j]; i = 0..N-1 is the y index (y = i/N),
 * j = 0..M-1 is the x index (x = j/M).  x1 = x, x2 = y in the paper's notation.
 *
 * Parity unpinned: none of the exported functions -- each is pinned by a test against a
 * closed form, an invariant, a special case or a brute-force / library computation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "ot_oracle.h"

#define TWO_PI 6.283185307179586476925286766559

/* ------------------------------------------------------------------------------------ */
/* Fourier transforms (used by Sec. 4.2)                                                   */
/* ------------------------------------------------------------------------------------ */

/* exp(sign * 2 pi i * t / L) with exact reduction of t modulo L. */
static void unit_root(long t, long L, int sign, double *c, double *s) {
  long r = t % L;
  if (r < 0) r += L;
  double a = TWO_PI * (double)r / (double)L;
  *c = cos(a);
  *s = sign * sin(a);
}

static int smallest_factor(int L) {
  for (int p = 2; p * p <= L; ++p)
    if (L % p == 0) return p;
  return L;
}

/* Table of the L-th roots of unity exp(sign 2 pi i t / L), t = 0..L-1. */
static void root_table(int L, int sign, double *tr, double *ti) {
  for (int t = 0; t < L; ++t) unit_root(t, L, sign, &tr[t], &ti[t]);
}

/* Recursive decimation in time on the smallest prime factor p of the current length Lc:
 *   X[k + q m] = sum_{r<p} W_Lc^{r (k + q m)} Y_r[k],  m = Lc/p,
 * where Y_r is the length-m transform of the r-th decimated subsequence.  A prime length
 * is a direct O(Lc^2) sum.  W_Lc^t = tab[(t mod Lc) * tstep] with tab the roots of the
 * top-level length Lc * tstep.  out must not alias in. */
static void fft_rec(const double *in_re, const double *in_im, long stride, int Lc,
                    const double *tr, const double *ti, long tstep, double *out_re,
                    double *out_im) {
  if (Lc == 1) {
    out_re[0] = in_re[0];
    out_im[0] = in_im[0];
    return;
  }
  int p = smallest_factor(Lc);
  if (p == Lc) {
    for (int k = 0; k < Lc; ++k) {
      double sr = 0.0, si = 0.0;
      for (int n = 0; n < Lc; ++n) {
        long t = ((long)k * n % Lc) * tstep;
        double xr = in_re[n * stride], xi = in_im[n * stride];
        sr += xr * tr[t] - xi * ti[t];
        si += xr * ti[t] + xi * tr[t];
      }
      out_re[k] = sr;
      out_im[k] = si;
    }
    return;
  }
  int m = Lc / p;
  double *y_re = (double *)malloc(sizeof(double) * Lc);
  double *y_im = (double *)malloc(sizeof(double) * Lc);
  for (int r = 0; r < p; ++r)
    fft_rec(in_re + r * stride, in_im + r * stride, stride * p, m, tr, ti, tstep * p,
            y_re + r * m, y_im + r * m);
  for (int k = 0; k < m; ++k) {
    for (int q = 0; q < p; ++q) {
      long kk = k + (long)q * m;
      double sr = 0.0, si = 0.0;
      for (int r = 0; r < p; ++r) {
        long t = ((long)r * kk % Lc) * tstep;
        double yr = y_re[r * m + k], yi = y_im[r * m + k];
        sr += yr * tr[t] - yi * ti[t];
        si += yr * ti[t] + yi * tr[t];
      }
      out_re[kk] = sr;
      out_im[kk] = si;
    }
  }
  free(y_re);
  free(y_im);
}

/* Unnormalised 1-D DFT of a strided sequence with a given root table, into out. */
static void fft_strided(const double *re, const double *im, long stride, int L,
                        const double *tr, const double *ti, double *o_re, double *o_im) {
  fft_rec(re, im, stride, L, tr, ti, 1, o_re, o_im);
}

/* Unnormalised 1-D DFT, in place: X_k = sum_n x_n exp(sign 2 pi i k n / L),
 * sign = -1 forward, +1 inverse. */
int orc_fft1(double *re, double *im, int L, int sign) {
  if (L <= 0 || (sign != 1 && sign != -1)) return -1;
  double *tr = (double *)malloc(sizeof(double) * L);
  double *ti = (double *)malloc(sizeof(double) * L);
  double *o_re = (double *)malloc(sizeof(double) * L);
  double *o_im = (double *)malloc(sizeof(double) * L);
  root_table(L, sign, tr, ti);
  fft_strided(re, im, 1, L, tr, ti, o_re, o_im);
  memcpy(re, o_re, sizeof(double) * L);
  memcpy(im, o_im, sizeof(double) * L);
  free(tr);
  free(ti);
  free(o_re);
  free(o_im);
  return 0;
}

/* Unnormalised 2-D DFT of an N x M row-major complex array, in place: 1-D transforms of
 * every row (length M), then of every column (length N). */
int orc_fft2(double *re, double *im, int N, int M, int sign) {
  if (N <= 0 || M <= 0 || (sign != 1 && sign != -1)) return -1;
  int Lmax = N > M ? N : M;
  double *tr = (double *)malloc(sizeof(double) * Lmax);
  double *ti = (double *)malloc(sizeof(double) * Lmax);
  double *o_re = (double *)malloc(sizeof(double) * Lmax);
  double *o_im = (double *)malloc(sizeof(double) * Lmax);
  root_table(M, sign, tr, ti);
  for (int i = 0; i < N; ++i) {
    fft_strided(re + (long)i * M, im + (long)i * M, 1, M, tr, ti, o_re, o_im);
    memcpy(re + (long)i * M, o_re, sizeof(double) * M);
    memcpy(im + (long)i * M, o_im, sizeof(double) * M);
  }
  root_table(N, sign, tr, ti);
  for (int j = 0; j < M; ++j) {
    fft_strided(re + j, im + j, M, N, tr, ti, o_re, o_im);
    for (int i = 0; i < N; ++i) {
      re[(long)i * M + j] = o_re[i];
      im[(long)i * M + j] = o_im[i];
    }
  }
  free(tr);
  free(ti);
  free(o_re);
  free(o_im);
  return 0;
}

/* Brute-force 2-D DFT (O(P^2)), the definition written out:
 * X[k2][k1] = sum_{n2,n1} x[n2][n1] exp(sign 2 pi i (k1 n1 / M + k2 n2 / N)). */
int orc_dft2(const double *re, const double *im, int N, int M, int sign, double *o_re,
             double *o_im) {
  if (N <= 0 || M <= 0) return -1;
  long NM = (long)N * M;
  for (int k2 = 0; k2 < N; ++k2)
    for (int k1 = 0; k1 < M; ++k1) {
      double sr = 0.0, si = 0.0;
      for (int n2 = 0; n2 < N; ++n2)
        for (int n1 = 0; n1 < M; ++n1) {
          /* phase = (k1 n1 mod M) / M + (k2 n2 mod N) / N, as an exact fraction of NM */
          long t = ((long)((long)k1 * n1 % M)) * N + ((long)((long)k2 * n2 % N)) * M;
          double c, s;
          unit_root(t, NM, sign, &c, &s);
          double xr = re[(long)n2 * M + n1], xi = im[(long)n2 * M + n1];
          sr += xr * c - xi * s;
          si += xr * s + xi * c;
        }
      o_re[(long)k2 * M + k1] = sr;
      o_im[(long)k2 * M + k1] = si;
    }
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Fourth-order centred differences (Sec. 4, intro)                                        */
/* ------------------------------------------------------------------------------------ */

static inline long wrap(long a, long L) {
  long r = a % L;
  return r < 0 ? r + L : r;
}

/* d/dx along j (spacing 1/M) of a periodic row-major field at (i, j). */
static double d1x(const double *u, int N, int M, int i, int j) {
  (void)N;
  const double *row = u + (long)i * M;
  double s = -row[wrap(j + 2, M)] + 8.0 * row[wrap(j + 1, M)] - 8.0 * row[wrap(j - 1, M)] +
             row[wrap(j - 2, M)];
  return s * (double)M / 12.0;
}

static double d1y(const double *u, int N, int M, int i, int j) {
  double s = -u[wrap(i + 2, N) * M + j] + 8.0 * u[wrap(i + 1, N) * M + j] -
             8.0 * u[wrap(i - 1, N) * M + j] + u[wrap(i - 2, N) * M + j];
  return s * (double)N / 12.0;
}

static double d2x(const double *u, int N, int M, int i, int j) {
  (void)N;
  const double *row = u + (long)i * M;
  double s = -row[wrap(j + 2, M)] + 16.0 * row[wrap(j + 1, M)] - 30.0 * row[j] +
             16.0 * row[wrap(j - 1, M)] - row[wrap(j - 2, M)];
  return s * (double)M * (double)M / 12.0;
}

static double d2y(const double *u, int N, int M, int i, int j) {
  double s = -u[wrap(i + 2, N) * M + j] + 16.0 * u[wrap(i + 1, N) * M + j] -
             30.0 * u[(long)i * M + j] + 16.0 * u[wrap(i - 1, N) * M + j] -
             u[wrap(i - 2, N) * M + j];
  return s * (double)N * (double)N / 12.0;
}

/* Mixed derivative: the x-stencil applied to the y-derivative at the four x-neighbours. */
static double dxy(const double *u, int N, int M, int i, int j) {
  double a = d1y(u, N, M, i, (int)wrap(j + 2, M));
  double b = d1y(u, N, M, i, (int)wrap(j + 1, M));
  double c = d1y(u, N, M, i, (int)wrap(j - 1, M));
  double d = d1y(u, N, M, i, (int)wrap(j - 2, M));
  return (-a + 8.0 * b - 8.0 * c + d) * (double)M / 12.0;
}

void orc_derivatives(const double *u, int N, int M, double *ux, double *uy, double *uxx,
                     double *uyy, double *uxy) {
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < M; ++j) {
      long p = (long)i * M + j;
      if (ux) ux[p] = d1x(u, N, M, i, j);
      if (uy) uy[p] = d1y(u, N, M, i, j);
      if (uxx) uxx[p] = d2x(u, N, M, i, j);
      if (uyy) uyy[p] = d2y(u, N, M, i, j);
      if (uxy) uxy[p] = dxy(u, N, M, i, j);
    }
}

/* ------------------------------------------------------------------------------------ */
/* Periodic cubic B-spline interpolation of g (Sec. 4: g at x + grad u by interpolation)  */
/* ------------------------------------------------------------------------------------ */

/* Solve the cyclic tridiagonal system (1/6) c[k-1] + (4/6) c[k] + (1/6) c[k+1] = r[k]
 * (indices mod n, n >= 3) by the Sherman-Morrison formula: split off the two corner
 * entries as a rank-one update of a plain tridiagonal matrix solved by the Thomas
 * algorithm.  r is overwritten with c. */
static void cyclic_tridiag_solve(double *r, int n) {
  const double lo = 1.0 / 6.0, di = 4.0 / 6.0, up = 1.0 / 6.0;
  const double corner_bl = 1.0 / 6.0; /* A[n-1][0] */
  const double corner_tr = 1.0 / 6.0; /* A[0][n-1] */
  double gamma = -di;
  double *bb = (double *)malloc(sizeof(double) * n);
  double *x = (double *)malloc(sizeof(double) * n);
  double *z = (double *)malloc(sizeof(double) * n);
  double *uvec = (double *)malloc(sizeof(double) * n);
  double *cp = (double *)malloc(sizeof(double) * n);
  for (int k = 0; k < n; ++k) bb[k] = di;
  bb[0] = di - gamma;
  bb[n - 1] = di - corner_bl * corner_tr / gamma;
  for (int k = 0; k < n; ++k) uvec[k] = 0.0;
  uvec[0] = gamma;
  uvec[n - 1] = corner_bl;
  /* Thomas algorithm on (lo, bb, up) for two right-hand sides */
  double *rhs[2] = {r, uvec};
  double *sol[2] = {x, z};
  for (int s = 0; s < 2; ++s) {
    double *d = rhs[s], *o = sol[s];
    double den = bb[0];
    cp[0] = up / den;
    o[0] = d[0] / den;
    for (int k = 1; k < n; ++k) {
      den = bb[k] - lo * cp[k - 1];
      cp[k] = up / den;
      o[k] = (d[k] - lo * o[k - 1]) / den;
    }
    for (int k = n - 2; k >= 0; --k) o[k] -= cp[k] * o[k + 1];
  }
  double vx = x[0] + corner_tr / gamma * x[n - 1];
  double vz = z[0] + corner_tr / gamma * z[n - 1];
  double fac = vx / (1.0 + vz);
  for (int k = 0; k < n; ++k) r[k] = x[k] - fac * z[k];
  free(bb);
  free(x);
  free(z);
  free(uvec);
  free(cp);
}

/* Coefficients c of the periodic tensor-product cubic B-spline interpolant of grid data g:
 * sum_{a,b} c[i+b][j+a] B(a) B(b) = g[i][j] with B(0) = 4/6, B(+-1) = 1/6. */
int orc_bspline_coeffs(const double *g, int N, int M, double *c) {
  if (N < 3 || M < 3) return -1;
  memcpy(c, g, sizeof(double) * (long)N * M);
  for (int i = 0; i < N; ++i) cyclic_tridiag_solve(c + (long)i * M, M);
  double *col = (double *)malloc(sizeof(double) * N);
  for (int j = 0; j < M; ++j) {
    for (int i = 0; i < N; ++i) col[i] = c[(long)i * M + j];
    cyclic_tridiag_solve(col, N);
    for (int i = 0; i < N; ++i) c[(long)i * M + j] = col[i];
  }
  free(col);
  return 0;
}

/* Uniform cubic B-spline weights for the taps at offsets -1, 0, 1, 2 from the cell origin,
 * fraction t in [0, 1), and their derivatives in t. */
static void bspline_weights(double t, double w[4], double dw[4]) {
  double s = 1.0 - t;
  w[0] = s * s * s / 6.0;
  w[1] = (3.0 * t * t * t - 6.0 * t * t + 4.0) / 6.0;
  w[2] = (-3.0 * t * t * t + 3.0 * t * t + 3.0 * t + 1.0) / 6.0;
  w[3] = t * t * t / 6.0;
  dw[0] = -s * s / 2.0;
  dw[1] = (3.0 * t * t - 4.0 * t) / 2.0;
  dw[2] = (-3.0 * t * t + 2.0 * t + 1.0) / 2.0;
  dw[3] = t * t / 2.0;
}

/* Interpolant and its gradient at a point given in grid units (gx_pos along j, gy_pos
 * along i): value = sum c[i0+b][j0+a] w_a(fx) w_b(fy), a, b in {-1, 0, 1, 2}. */
void orc_bspline_eval_grid(const double *c, int N, int M, double gx_pos, double gy_pos,
                           double *val, double *dgdx, double *dgdy) {
  double fj = floor(gx_pos), fi = floor(gy_pos);
  double tx = gx_pos - fj, ty = gy_pos - fi;
  long j0 = (long)fj, i0 = (long)fi;
  double wx[4], dwx[4], wy[4], dwy[4];
  bspline_weights(tx, wx, dwx);
  bspline_weights(ty, wy, dwy);
  double v = 0.0, gx = 0.0, gy = 0.0;
  for (int b = 0; b < 4; ++b) {
    long ii = wrap(i0 + b - 1, N);
    for (int a = 0; a < 4; ++a) {
      long jj = wrap(j0 + a - 1, M);
      double cv = c[ii * M + jj];
      v += cv * wx[a] * wy[b];
      gx += cv * dwx[a] * wy[b];
      gy += cv * wx[a] * dwy[b];
    }
  }
  *val = v;
  *dgdx = gx * (double)M;
  *dgdy = gy * (double)N;
}

/* Same, at a point of the unit torus (x along j, y along i). */
void orc_bspline_eval(const double *c, int N, int M, double x, double y, double *val,
                      double *dgdx, double *dgdy) {
  orc_bspline_eval_grid(c, N, M, x * (double)M, y * (double)N, val, dgdx, dgdy);
}

/* ------------------------------------------------------------------------------------ */
/* Nonlinear residual and linearised coefficients (Eq. ma2, Eq. linearmaeq, Eq. translation) */
/* ------------------------------------------------------------------------------------ */

/* For the iterate u:
 *   f_n = G(x + grad u) det(I + D^2 u)                                  (Eq. ma2)
 *   f~_n = f_n - mean(f_n) + 1                                          (Eq. translation)
 *   F = f - f~_n
 *   coefficients of D_u M (Eq. linearmaeq) with Adj(I + D^2 u) = [[1+u_yy, -u_xy],
 *   [-u_xy, 1+u_xx]]:  a11 = G (1+u_yy), a12 = -G u_xy, a22 = G (1+u_xx),
 *                      b1 = det dG/dx, b2 = det dG/dy.
 * coef (optional) holds 5 planes in the order a11, a12, a22, b1, b2.
 * scal (optional): [0] mean f_n, [1] max|F|, [2] sqrt(mean F^2), [3] min det,
 *                  [4] count of non-finite f_n. */
/* simplified operator (Sec. 3.3 remark): g(x + grad u) Tr(Adj(I + D^2 u) D^2 theta), i.e. the
 * coefficients b1 = b2 = 0; F itself is unchanged */
static int g_simplified = 0;
void orc_set_simplified(int on) { g_simplified = on ? 1 : 0; }

/* Interpolation of g at the displaced points (Sec. 4 intro: closest-neighbour interpolation
 * used for the images of Sec. 5.2, linear interpolation named as the alternative and used
 * in Sec. 5.3): 0 = the periodic cubic B-spline interpolant of the coefficients c (default),
 * 1 = bilinear, 2 = nearest node.  In modes 1 and 2, c holds the grid values of g itself
 * (no prefilter), G(T) interpolates them and grad G(T) interpolates, by the same rule, the
 * grid gradient of g by the 4th-order centred differences. */
static int g_interp = 0;
void orc_set_interp(int mode) { g_interp = (mode == 1 || mode == 2) ? mode : 0; }
int orc_get_interp(void) { return g_interp; }

static void interp_eval_grid(const double *c, const double *gxg, const double *gyg, int N,
                             int M, double gx_pos, double gy_pos, double *val, double *dgdx,
                             double *dgdy) {
  if (g_interp == 2) { /* nearest node: round half up */
    long jn = wrap((long)floor(gx_pos + 0.5), M), in = wrap((long)floor(gy_pos + 0.5), N);
    long q = in * M + jn;
    *val = c[q];
    *dgdx = gxg[q];
    *dgdy = gyg[q];
    return;
  }
  /* bilinear on the cell (i0, j0) .. (i0 + 1, j0 + 1) */
  double fj = floor(gx_pos), fi = floor(gy_pos);
  double tx = gx_pos - fj, ty = gy_pos - fi;
  long j0 = wrap((long)fj, M), i0 = wrap((long)fi, N);
  long j1 = wrap(j0 + 1, M), i1 = wrap(i0 + 1, N);
  double w[4] = {(1.0 - tx) * (1.0 - ty), tx * (1.0 - ty), (1.0 - tx) * ty, tx * ty};
  long q[4] = {i0 * M + j0, i0 * M + j1, i1 * M + j0, i1 * M + j1};
  double v = 0.0, a = 0.0, b = 0.0;
  for (int k = 0; k < 4; ++k) {
    v += w[k] * c[q[k]];
    a += w[k] * gxg[q[k]];
    b += w[k] * gyg[q[k]];
  }
  *val = v;
  *dgdx = a;
  *dgdy = b;
}

int orc_residual(const double *f, const double *c, const double *u, int N, int M, double *F,
                 double *coef, double *scal) {
  long P = (long)N * M;
  double *fn = (double *)malloc(sizeof(double) * P);
  double *gxg = NULL, *gyg = NULL;
  if (g_interp) { /* grid gradient of g (c holds g in these modes) */
    gxg = (double *)malloc(sizeof(double) * P);
    gyg = (double *)malloc(sizeof(double) * P);
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < M; ++j) {
        gxg[(long)i * M + j] = d1x(c, N, M, i, j);
        gyg[(long)i * M + j] = d1y(c, N, M, i, j);
      }
  }
  double sum_fn = 0.0, min_det = INFINITY;
  long nonfinite = 0;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < M; ++j) {
      long p = (long)i * M + j;
      double ux = d1x(u, N, M, i, j), uy = d1y(u, N, M, i, j);
      double uxx = d2x(u, N, M, i, j), uyy = d2y(u, N, M, i, j);
      double uxy = dxy(u, N, M, i, j);
      double G, Gx, Gy;
      if (g_interp)
        interp_eval_grid(c, gxg, gyg, N, M, (double)j + (double)M * ux,
                         (double)i + (double)N * uy, &G, &Gx, &Gy);
      else
        orc_bspline_eval_grid(c, N, M, (double)j + (double)M * ux, (double)i + (double)N * uy,
                              &G, &Gx, &Gy);
      double det = (1.0 + uxx) * (1.0 + uyy) - uxy * uxy;
      fn[p] = G * det;
      if (!isfinite(fn[p])) nonfinite++;
      sum_fn += fn[p];
      if (det < min_det) min_det = det;
      if (coef) {
        coef[0 * P + p] = G * (1.0 + uyy);
        coef[1 * P + p] = -G * uxy;
        coef[2 * P + p] = G * (1.0 + uxx);
        coef[3 * P + p] = g_simplified ? 0.0 : det * Gx;
        coef[4 * P + p] = g_simplified ? 0.0 : det * Gy;
      }
    }
  double mean_fn = sum_fn / (double)P;
  double rinf = 0.0, r2 = 0.0;
  for (long p = 0; p < P; ++p) {
    double ft = fn[p] - mean_fn + 1.0;
    double r = f[p] - ft;
    if (F) F[p] = r;
    if (fabs(r) > rinf) rinf = fabs(r);
    r2 += r * r;
  }
  if (scal) {
    scal[0] = mean_fn;
    scal[1] = rinf;
    scal[2] = sqrt(r2 / (double)P);
    scal[3] = min_det;
    scal[4] = (double)nonfinite;
  }
  free(fn);
  free(gxg);
  free(gyg);
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Simpson averages of the coefficients (Sec. 4.2, last paragraph)                          */
/* ------------------------------------------------------------------------------------ */

/* Composite Simpson rule on [0,1]^2 with the periodic node x_L identified with x_0:
 * per-axis weights (2/3 at even index, 4/3 at odd index) / L.  L must be even. */
double orc_simpson_mean(const double *a, int N, int M) {
  double s = 0.0;
  for (int i = 0; i < N; ++i) {
    double wy = ((i % 2) == 0 ? 2.0 : 4.0) / (3.0 * (double)N);
    for (int j = 0; j < M; ++j) {
      double wx = ((j % 2) == 0 ? 2.0 : 4.0) / (3.0 * (double)M);
      s += wy * wx * a[(long)i * M + j];
    }
  }
  return s;
}

/* ------------------------------------------------------------------------------------ */
/* Strain's preconditioned operator (Sec. 4.2, Eq. fouriersystem and rho-bar)              */
/* ------------------------------------------------------------------------------------ */

/* signed frequency of DFT index n of length L, and whether it is the Nyquist index */
static long signed_freq(int n, int L, int *is_nyq) {
  *is_nyq = (L % 2 == 0) && (n == L / 2);
  return n <= L / 2 ? n : (long)n - L;
}

/* Symbols of the derivatives in the linear operator: 0 (default) the paper's spectral
 * symbols 2 pi i k and -(2 pi k)^2 (Sec. 4.2); 1 the Fourier symbols of the 4th-order
 * stencils of the residual (reading R1), which make L the exact linearisation of the
 * discrete F. */
static int g_fd = 0;
void orc_set_fd_symbols(int on) { g_fd = on ? 1 : 0; }

/* first-derivative symbol (purely imaginary): returns its imaginary part.  Spectral:
 * 2 pi k, 0 at Nyquist; stencil: (8 sin t - sin 2t) / (6 h), t = 2 pi k / L, h = 1/L. */
static double sym1(long k, int L, int nyq, int fd) {
  if (fd) {
    double t = TWO_PI * (double)k / (double)L;
    return (8.0 * sin(t) - sin(2.0 * t)) / 6.0 * (double)L;
  }
  return nyq ? 0.0 : TWO_PI * (double)k;
}

/* second-derivative symbol (real).  Spectral: -(2 pi k)^2, kept at Nyquist; stencil:
 * (-2 cos 2t + 32 cos t - 30) / (12 h^2). */
static double sym2(long k, int L, int fd) {
  if (fd) {
    double t = TWO_PI * (double)k / (double)L;
    return (-2.0 * cos(2.0 * t) + 32.0 * cos(t) - 30.0) / 12.0 * (double)L * (double)L;
  }
  return -(TWO_PI * (double)k) * (TWO_PI * (double)k);
}

/* symbol of d_p d_q at frequency (k1, k2) (p, q in {1, 2}, 1 = x along M, 2 = y along N)
 * as a complex number (re, im).  Same-axis pairs use the second-derivative symbol; the
 * mixed pair is the product of the two first-derivative symbols. */
static void sym_pq(int p, int q, long k1, int n1, int M, long k2, int n2, int N, int fd,
                   double *re, double *im) {
  if (p == q) {
    *re = (p == 1) ? sym2(k1, M, fd) : sym2(k2, N, fd);
    *im = 0.0;
  } else {
    /* (i s1)(i s2) = -s1 s2 */
    *re = -sym1(k1, M, n1, fd) * sym1(k2, N, n2, fd);
    *im = 0.0;
  }
}

static void sym_p(int p, long k1, int n1, int M, long k2, int n2, int N, int fd, double *re,
                  double *im) {
  *re = 0.0;
  *im = (p == 1) ? sym1(k1, M, n1, fd) : sym1(k2, N, n2, fd);
}

/* rho-bar(k) = 1 / (sum_ij abar_ij d_i d_j + sum_i bbar_i d_i) with the symbols above,
 * 0 where the denominator vanishes.  abar = {a11, a12, a22, b1, b2} (a21 = a12). */
static void rho_bar_nm(const double abar[5], long k1, int n1, int M, long k2, int n2, int N,
                       int fd, double *re, double *im) {
  double A[2][2] = {{abar[0], abar[1]}, {abar[1], abar[2]}};
  double B[2] = {abar[3], abar[4]};
  double dr = 0.0, di = 0.0;
  for (int p = 1; p <= 2; ++p)
    for (int q = 1; q <= 2; ++q) {
      double sr, si;
      sym_pq(p, q, k1, n1, M, k2, n2, N, fd, &sr, &si);
      dr += A[p - 1][q - 1] * sr;
      di += A[p - 1][q - 1] * si;
    }
  for (int p = 1; p <= 2; ++p) {
    double sr, si;
    sym_p(p, k1, n1, M, k2, n2, N, fd, &sr, &si);
    dr += B[p - 1] * sr;
    di += B[p - 1] * si;
  }
  double den = dr * dr + di * di;
  if (den == 0.0) {
    *re = 0.0;
    *im = 0.0;
  } else {
    *re = dr / den;
    *im = -di / den;
  }
}

/* w = L Lbar^{-1} sigma:
 *   sigma-hat = FFT(sigma); S = rho-bar sigma-hat;
 *   alpha_pq = IFFT(sym_pq S), beta_p = IFFT(sym_p S)   (all d(d+1) = 6 of them);
 *   w = sum_pq a_pq alpha_pq + sum_p b_p beta_p.
 * coef: 5 planes a11, a12, a22, b1, b2 (a21 = a12). */
void orc_apply_op(const double *coef, const double abar[5], const double *sigma, int N, int M,
                  double *w) {
  long P = (long)N * M;
  double *s_re = (double *)malloc(sizeof(double) * P);
  double *s_im = (double *)malloc(sizeof(double) * P);
  double *t_re = (double *)malloc(sizeof(double) * P);
  double *t_im = (double *)malloc(sizeof(double) * P);
  for (long p = 0; p < P; ++p) {
    s_re[p] = sigma[p];
    s_im[p] = 0.0;
  }
  orc_fft2(s_re, s_im, N, M, -1);
  for (int i = 0; i < N; ++i) {
    int n2;
    long k2 = signed_freq(i, N, &n2);
    for (int j = 0; j < M; ++j) {
      int n1;
      long k1 = signed_freq(j, M, &n1);
      double rr, ri;
      rho_bar_nm(abar, k1, n1, M, k2, n2, N, g_fd, &rr, &ri);
      long p = (long)i * M + j;
      double a = s_re[p], b = s_im[p];
      s_re[p] = rr * a - ri * b;
      s_im[p] = rr * b + ri * a;
    }
  }
  for (long p = 0; p < P; ++p) w[p] = 0.0;
  const double *a_pq[2][2] = {{coef, coef + P}, {coef + P, coef + 2 * P}};
  const double *b_p[2] = {coef + 3 * P, coef + 4 * P};
  double inv = 1.0 / (double)P;
  for (int term = 0; term < 6; ++term) {
    int p, q = 0, second = term < 4;
    if (second) {
      p = term / 2 + 1;
      q = term % 2 + 1;
    } else {
      p = term - 3;
    }
    for (int i = 0; i < N; ++i) {
      int n2;
      long k2 = signed_freq(i, N, &n2);
      for (int j = 0; j < M; ++j) {
        int n1;
        long k1 = signed_freq(j, M, &n1);
        double sr, si;
        if (second)
          sym_pq(p, q, k1, n1, M, k2, n2, N, g_fd, &sr, &si);
        else
          sym_p(p, k1, n1, M, k2, n2, N, g_fd, &sr, &si);
        long idx = (long)i * M + j;
        t_re[idx] = sr * s_re[idx] - si * s_im[idx];
        t_im[idx] = sr * s_im[idx] + si * s_re[idx];
      }
    }
    orc_fft2(t_re, t_im, N, M, +1);
    const double *cf = second ? a_pq[p - 1][q - 1] : b_p[p - 1];
    for (long idx = 0; idx < P; ++idx) w[idx] += cf[idx] * (t_re[idx] * inv);
  }
  free(s_re);
  free(s_im);
  free(t_re);
  free(t_im);
}

/* theta = Lbar^{-1} sigma = sum_{k != 0} rho-bar(k) sigma-hat(k) e^{2 pi i k.x}
 * (Sec. 4.2, recovery of theta; one forward and one inverse FFT). */
void orc_apply_lbar_inv(const double abar[5], const double *sigma, int N, int M,
                        double *theta) {
  long P = (long)N * M;
  double *s_re = (double *)malloc(sizeof(double) * P);
  double *s_im = (double *)malloc(sizeof(double) * P);
  for (long p = 0; p < P; ++p) {
    s_re[p] = sigma[p];
    s_im[p] = 0.0;
  }
  orc_fft2(s_re, s_im, N, M, -1);
  for (int i = 0; i < N; ++i) {
    int n2;
    long k2 = signed_freq(i, N, &n2);
    for (int j = 0; j < M; ++j) {
      int n1;
      long k1 = signed_freq(j, M, &n1);
      double rr, ri;
      rho_bar_nm(abar, k1, n1, M, k2, n2, N, g_fd, &rr, &ri);
      long p = (long)i * M + j;
      double a = s_re[p], b = s_im[p];
      s_re[p] = rr * a - ri * b;
      s_im[p] = rr * b + ri * a;
    }
  }
  orc_fft2(s_re, s_im, N, M, +1);
  for (long p = 0; p < P; ++p) theta[p] = s_re[p] / (double)P;
  free(s_re);
  free(s_im);
}

/* ------------------------------------------------------------------------------------ */
/* Restarted GMRES(m) (Sec. 4.2; Saad's algorithm with MGS Arnoldi and Givens rotations)   */
/* ------------------------------------------------------------------------------------ */

typedef void (*matvec_fn)(void *ctx, const double *x, double *y);

static double dot(const double *a, const double *b, long n) {
  double s = 0.0;
  for (long k = 0; k < n; ++k) s += a[k] * b[k];
  return s;
}

/* Solves A x = b from x = 0.  Stops when the Givens estimate of ||b - A x||_2 falls to
 * eta ||b||_2 or below (or on breakdown), or after max_restarts cycles.  At the end of a
 * cycle that did not converge the residual is recomputed explicitly.
 * out: iters = Arnoldi steps, cycles = restart cycles begun, relres = estimate / ||b||.
 * Returns 0 if converged, 1 otherwise. */
static int gmres(matvec_fn A, void *ctx, const double *b, long n, int m, double eta,
                 int max_restarts, double *x, int *iters, int *cycles, double *relres) {
  double *V = (double *)malloc(sizeof(double) * n * (m + 1));
  double *H = (double *)calloc((size_t)(m + 1) * m, sizeof(double));
  double *cs = (double *)malloc(sizeof(double) * m);
  double *sn = (double *)malloc(sizeof(double) * m);
  double *g = (double *)malloc(sizeof(double) * (m + 1));
  double *y = (double *)malloc(sizeof(double) * m);
  double *w = (double *)malloc(sizeof(double) * n);
  for (long k = 0; k < n; ++k) x[k] = 0.0;
  double bnorm = sqrt(dot(b, b, n));
  *iters = 0;
  *cycles = 0;
  *relres = 0.0;
  int converged = 0;
  if (bnorm == 0.0) {
    converged = 1;
    goto done;
  }
  /* r0 = b */
  for (long k = 0; k < n; ++k) w[k] = b[k];
  double beta = bnorm;
  for (int cyc = 0; cyc < max_restarts; ++cyc) {
    (*cycles)++;
    for (long k = 0; k < n; ++k) V[k] = w[k] / beta;
    for (int k = 0; k <= m; ++k) g[k] = 0.0;
    g[0] = beta;
    int jend = 0;
    for (int j = 0; j < m; ++j) {
      double *vj = V + (long)j * n;
      A(ctx, vj, w);
      for (int i = 0; i <= j; ++i) { /* modified Gram-Schmidt */
        double *vi = V + (long)i * n;
        double h = dot(w, vi, n);
        H[i * m + j] = h;
        for (long k = 0; k < n; ++k) w[k] -= h * vi[k];
      }
      double hn = sqrt(dot(w, w, n));
      H[(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) { /* previous rotations on column j */
        double t0 = H[i * m + j], t1 = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * t0 + sn[i] * t1;
        H[(i + 1) * m + j] = -sn[i] * t0 + cs[i] * t1;
      }
      double a = H[j * m + j], bb = H[(j + 1) * m + j];
      double r = sqrt(a * a + bb * bb);
      cs[j] = (r == 0.0) ? 1.0 : a / r;
      sn[j] = (r == 0.0) ? 0.0 : bb / r;
      H[j * m + j] = r;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      (*iters)++;
      jend = j + 1;
      *relres = fabs(g[j + 1]) / bnorm;
      if (fabs(g[j + 1]) <= eta * bnorm || hn == 0.0) {
        converged = 1;
        break;
      }
      double *vn = V + (long)(j + 1) * n;
      for (long k = 0; k < n; ++k) vn[k] = w[k] / hn;
    }
    /* y = R^{-1} g (back substitution), x += V y */
    for (int i = jend - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < jend; ++k) s -= H[i * m + k] * y[k];
      y[i] = s / H[i * m + i];
    }
    for (int i = 0; i < jend; ++i) {
      double *vi = V + (long)i * n;
      for (long k = 0; k < n; ++k) x[k] += y[i] * vi[k];
    }
    if (converged) break;
    /* explicit residual for the restart */
    A(ctx, x, w);
    for (long k = 0; k < n; ++k) w[k] = b[k] - w[k];
    beta = sqrt(dot(w, w, n));
    *relres = beta / bnorm;
    if (beta <= eta * bnorm) {
      converged = 1;
      break;
    }
  }
done:
  free(V);
  free(H);
  free(cs);
  free(sn);
  free(g);
  free(y);
  free(w);
  return converged ? 0 : 1;
}

typedef struct {
  const double *A;
  long n;
} dense_ctx;

static void dense_mv(void *ctx, const double *x, double *y) {
  dense_ctx *d = (dense_ctx *)ctx;
  for (long r = 0; r < d->n; ++r) y[r] = dot(d->A + r * d->n, x, d->n);
}

/* The same GMRES(m) routine on a dense row-major n x n matrix (used to pin the Krylov
 * loop against a direct solve). */
int orc_gmres_dense(const double *A, const double *b, int n, int m, double eta,
                    int max_restarts, double *x, int *iters, int *cycles, double *relres) {
  dense_ctx d = {A, n};
  return gmres(dense_mv, &d, b, n, m, eta, max_restarts, x, iters, cycles, relres);
}

typedef struct {
  const double *coef;
  const double *abar;
  int N, M;
} op_ctx;

static void op_mv(void *ctx, const double *x, double *y) {
  op_ctx *o = (op_ctx *)ctx;
  orc_apply_op(o->coef, o->abar, x, o->N, o->M, y);
}

/* GMRES(m) on L Lbar^{-1} sigma = h (first line of Eq. fouriersystem). */
int orc_gmres_op(const double *coef, const double abar[5], const double *h, int N, int M, int m,
                 double eta, int max_restarts, double *sigma, int *iters, int *cycles,
                 double *relres) {
  op_ctx o = {coef, abar, N, M};
  return gmres(op_mv, &o, h, (long)N * M, m, eta, max_restarts, sigma, iters, cycles, relres);
}

/* ------------------------------------------------------------------------------------ */
/* Finite-difference implementation (Sec. 4.1): second-order centred differences of theta, */
/* the augmented square system A~ x = b, unpreconditioned BiCG                             */
/* ------------------------------------------------------------------------------------ */

/* The linear operator of Eq. (linearmaeq) in the coefficient form of orc_residual,
 *   L theta = a11 theta_xx + 2 a12 theta_xy + a22 theta_yy + b1 theta_x + b2 theta_y,
 * with second-order centred differences (spacings 1/M along j, 1/N along i):
 *   theta_x  ~ (t[j+1] - t[j-1]) M / 2,          theta_xx ~ (t[j+1] - 2 t + t[j-1]) M^2,
 *   theta_xy ~ (t[+1,+1] - t[+1,-1] - t[-1,+1] + t[-1,-1]) N M / 4   (offsets (di, dj)).
 * Row r of the matrix A holds, at column r + (di, dj), the weight of that neighbour.  The
 * extra equation sum_k x_k = 0 (int theta = 0) added to every row and then dropped gives
 * A~ = A + 1 1^T (every entry of A~ is the entry of A plus one). */
#define FD_TAPS 9
static void fd_row(const double *coef, long P, long r, int N, int M, double w[FD_TAPS]) {
  /* weights of row r at the 3 x 3 offsets, index (di + 1) * 3 + (dj + 1) */
  double a11 = coef[r], a12 = coef[P + r], a22 = coef[2 * P + r];
  double b1 = coef[3 * P + r], b2 = coef[4 * P + r];
  double m2 = (double)M * M, n2 = (double)N * N, xy = 2.0 * a12 * (double)N * M / 4.0;
  for (int t = 0; t < FD_TAPS; ++t) w[t] = 0.0;
  w[4] += -2.0 * a11 * m2 - 2.0 * a22 * n2;
  w[3] += a11 * m2 - b1 * 0.5 * M;  /* (0, -1) */
  w[5] += a11 * m2 + b1 * 0.5 * M;  /* (0, +1) */
  w[1] += a22 * n2 - b2 * 0.5 * N;  /* (-1, 0) */
  w[7] += a22 * n2 + b2 * 0.5 * N;  /* (+1, 0) */
  w[8] += xy;                       /* (+1, +1) */
  w[6] -= xy;                       /* (+1, -1) */
  w[2] -= xy;                       /* (-1, +1) */
  w[0] += xy;                       /* (-1, -1) */
}

/* y = A~ x: each row of A applied to x (gather), plus sum(x). */
void orc_fd_apply(const double *coef, const double *x, int N, int M, double *y) {
  long P = (long)N * M;
  double sx = 0.0;
  for (long k = 0; k < P; ++k) sx += x[k];
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < M; ++j) {
      long r = (long)i * M + j;
      double w[FD_TAPS], acc = 0.0;
      fd_row(coef, P, r, N, M, w);
      for (int di = -1; di <= 1; ++di)
        for (int dj = -1; dj <= 1; ++dj)
          acc += w[(di + 1) * 3 + (dj + 1)] * x[wrap(i + di, N) * M + wrap(j + dj, M)];
      y[r] = acc + sx;
    }
}

/* y = A~^T x: every row r of A scatters its weight times x[r] onto the columns it touches
 * (sum_r A[r][k] x[r]), plus sum(x) (the all-ones part is symmetric). */
void orc_fd_apply_t(const double *coef, const double *x, int N, int M, double *y) {
  long P = (long)N * M;
  double sx = 0.0;
  for (long k = 0; k < P; ++k) {
    sx += x[k];
    y[k] = 0.0;
  }
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < M; ++j) {
      long r = (long)i * M + j;
      double w[FD_TAPS];
      fd_row(coef, P, r, N, M, w);
      for (int di = -1; di <= 1; ++di)
        for (int dj = -1; dj <= 1; ++dj)
          y[wrap(i + di, N) * M + wrap(j + dj, M)] += w[(di + 1) * 3 + (dj + 1)] * x[r];
    }
  for (long k = 0; k < P; ++k) y[k] += sx;
}

/* Biconjugate gradients without preconditioning (Sec. 4.1; Fletcher's form as in Saad,
 * Iterative Methods for Sparse Linear Systems, Alg. 7.3) for A x = b from x = 0 with the
 * shadow residual r*_0 = r_0:
 *   alpha = (r, r*) / (A p, p*);  x += alpha p;  r -= alpha A p;  r* -= alpha A^T p*;
 *   beta = (r_new, r*_new) / (r, r*);  p = r + beta p;  p* = r* + beta p*.
 * Stops when ||r||_2 <= eta ||b||_2, after max_iters iterations, or on breakdown (a zero
 * denominator).  out: iters, relres = ||r|| / ||b||.  Returns 0 if converged, 1 if the
 * iteration cap was reached, 2 on breakdown. */
static int bicg(matvec_fn A, matvec_fn At, void *ctx, const double *b, long n, double eta,
                int max_iters, double *x, int *iters, double *relres) {
  double *r = (double *)malloc(sizeof(double) * n);
  double *rs = (double *)malloc(sizeof(double) * n);
  double *p = (double *)malloc(sizeof(double) * n);
  double *ps = (double *)malloc(sizeof(double) * n);
  double *q = (double *)malloc(sizeof(double) * n);
  double *qs = (double *)malloc(sizeof(double) * n);
  int rc = 1;
  double bnorm = sqrt(dot(b, b, n));
  for (long k = 0; k < n; ++k) {
    x[k] = 0.0;
    r[k] = rs[k] = p[k] = ps[k] = b[k];
  }
  *iters = 0;
  *relres = 0.0;
  if (bnorm == 0.0) {
    rc = 0;
    goto done;
  }
  double rho = dot(r, rs, n);
  *relres = 1.0;
  while (*iters < max_iters) {
    A(ctx, p, q);
    At(ctx, ps, qs);
    double den = dot(q, ps, n);
    if (den == 0.0) {
      rc = 2;
      break;
    }
    double alpha = rho / den;
    for (long k = 0; k < n; ++k) {
      x[k] += alpha * p[k];
      r[k] -= alpha * q[k];
      rs[k] -= alpha * qs[k];
    }
    (*iters)++;
    double rnorm = sqrt(dot(r, r, n));
    *relres = rnorm / bnorm;
    if (rnorm <= eta * bnorm) {
      rc = 0;
      break;
    }
    double rho_new = dot(r, rs, n);
    if (rho_new == 0.0) {
      rc = 2;
      break;
    }
    double beta = rho_new / rho;
    rho = rho_new;
    for (long k = 0; k < n; ++k) {
      p[k] = r[k] + beta * p[k];
      ps[k] = rs[k] + beta * ps[k];
    }
  }
done:
  free(r);
  free(rs);
  free(p);
  free(ps);
  free(q);
  free(qs);
  return rc;
}

static void dense_mv_t(void *ctx, const double *x, double *y) {
  dense_ctx *d = (dense_ctx *)ctx;
  for (long c = 0; c < d->n; ++c) {
    double s = 0.0;
    for (long r = 0; r < d->n; ++r) s += d->A[r * d->n + c] * x[r];
    y[c] = s;
  }
}

/* The BiCG routine on a dense row-major n x n matrix (pinned against a direct solve). */
int orc_bicg_dense(const double *A, const double *b, int n, double eta, int max_iters,
                   double *x, int *iters, double *relres) {
  dense_ctx d = {A, n};
  return bicg(dense_mv, dense_mv_t, &d, b, n, eta, max_iters, x, iters, relres);
}

typedef struct {
  const double *coef;
  int N, M;
} fd_ctx;

static void fd_mv(void *ctx, const double *x, double *y) {
  fd_ctx *o = (fd_ctx *)ctx;
  orc_fd_apply(o->coef, x, o->N, o->M, y);
}
static void fd_mv_t(void *ctx, const double *x, double *y) {
  fd_ctx *o = (fd_ctx *)ctx;
  orc_fd_apply_t(o->coef, x, o->N, o->M, y);
}

/* BiCG on A~ theta = h (Sec. 4.1). */
int orc_bicg_fd(const double *coef, const double *h, int N, int M, double eta, int max_iters,
                double *theta, int *iters, double *relres) {
  fd_ctx o = {coef, N, M};
  return bicg(fd_mv, fd_mv_t, &o, h, (long)N * M, eta, max_iters, theta, iters, relres);
}

/* Linear solver of the Newton steps: 0 (default) the Fourier method of Sec. 4.2, 1 the
 * finite-difference system with BiCG of Sec. 4.1 (at most max_iters iterations per step). */
static int g_linsolver = 0, g_max_bicg = 20000;
void orc_set_linear_solver(int mode, int max_iters) {
  g_linsolver = mode == 1 ? 1 : 0;
  g_max_bicg = max_iters > 0 ? max_iters : 20000;
}

/* ------------------------------------------------------------------------------------ */
/* Damped Newton (Sec. 3.1, Eq. linma) with the Fourier implementation of Sec. 4.2          */
/* ------------------------------------------------------------------------------------ */

/* Eq. (translation) applied to an input density: d <- d - mean(d) + 1.  Fails on a
 * non-finite entry or a non-positive result (the convergence theorem needs positive
 * densities). */
static int translate_density(const double *in, double *out, long P) {
  double s = 0.0;
  for (long p = 0; p < P; ++p) {
    if (!isfinite(in[p])) return -1;
    s += in[p];
  }
  double mean = s / (double)P;
  for (long p = 0; p < P; ++p) {
    out[p] = in[p] - mean + 1.0;
    if (!(out[p] > 0.0)) return -1;
  }
  return 0;
}

void orc_default_opts(orc_opts *o) {
  o->tau = 1.0;
  o->tol = 1e-8;
  o->eta = 1e-4;
  o->restart = 10;
  o->max_restarts = 50;
  o->max_newton = 200;
  o->translate_inputs = 1;
  o->safeguard = 1;
  o->tau_switch = 0.0;
}

/* Convexity of the iterate: the proof of convergence keeps I + D^2 u_n positive definite
 * at every step (Sec. 3.2 remarks), which in 2-D is det > 0 together with 1 + u_xx > 0;
 * since u_n stays a perturbation of the convex start we test det > 0 and finiteness. */
static int iterate_admissible(const double scal[5]) {
  return scal[4] == 0.0 && isfinite(scal[1]) && scal[3] > 0.0;
}

/* u (in/out): initial guess u0 on entry (zero for the constant start of the convergence
 * theorem), mean-zero iterate on exit.  hist_res (optional, max_newton + 1 entries):
 * max|F| before each Newton solve; hist_gmres (optional, max_newton entries): Arnoldi
 * steps of each solve.
 *
 * Step control: the Newton update is theta_n solving D_{u_n}M theta = (f - f~_n)/tau.  With
 * safeguard on, the candidate u_n + s theta_n (s = 1, 1/2, 1/4, ...; i.e. a step-size
 * parameter tau/s, the paper's remedy of a larger tau) is accepted once it is admissible;
 * after an accepted step s doubles again, capped at 1.  theta is linear in 1/tau, so no
 * new linear solve is needed.  With safeguard off the plain iteration of Eq. (linma) runs
 * and an inadmissible iterate ends the solve as diverged. */
int orc_solve(const double *f_in, const double *g_in, int N, int M, const orc_opts *o,
              double *u, orc_stats *st, double *hist_res, int *hist_gmres) {
  memset(st, 0, sizeof(*st));
  if (N < 4 || M < 4 || (N % 2) || (M % 2) || o->tau < 1.0 || !(o->tol > 0.0) ||
      o->restart < 1) {
    st->status = ORC_EINVAL;
    return ORC_EINVAL;
  }
  long P = (long)N * M;
  double *f = (double *)malloc(sizeof(double) * P);
  double *g = (double *)malloc(sizeof(double) * P);
  double *c = (double *)malloc(sizeof(double) * P);
  double *F = (double *)malloc(sizeof(double) * P);
  double *coef = (double *)malloc(sizeof(double) * 5 * P);
  double *h = (double *)malloc(sizeof(double) * P);
  double *sigma = (double *)malloc(sizeof(double) * P);
  double *theta = (double *)malloc(sizeof(double) * P);
  double *cand = (double *)malloc(sizeof(double) * P);
  int status = ORC_OK;
  double s = 1.0;
  if (o->translate_inputs) {
    if (translate_density(f_in, f, P) || translate_density(g_in, g, P)) {
      status = ORC_EINVAL;
      goto out;
    }
  } else {
    memcpy(f, f_in, sizeof(double) * P);
    memcpy(g, g_in, sizeof(double) * P);
  }
  if (g_interp)
    memcpy(c, g, sizeof(double) * P); /* nearest / bilinear: the grid values themselves */
  else
    orc_bspline_coeffs(g, N, M, c);
  double scal[5];
  orc_residual(f, c, u, N, M, F, coef, scal);
  double tau = o->tau;
  for (int n = 0;; ++n) {
    st->mean_fn = scal[0];
    st->res_inf = scal[1];
    st->res_l2 = scal[2];
    st->min_det = scal[3];
    if (hist_res) hist_res[n] = scal[1];
    if (!iterate_admissible(scal)) {
      status = ORC_EDIVERGED;
      break;
    }
    if (scal[1] < o->tol) break;
    if (n >= o->max_newton) {
      status = ORC_ENOCONV;
      break;
    }
    if (o->tau_switch > 0.0 && scal[1] < o->tau_switch) tau = 1.0; /* kept from here on */
    double abar[5];
    for (int q = 0; q < 5; ++q) abar[q] = orc_simpson_mean(coef + q * P, N, M);
    for (long p = 0; p < P; ++p) h[p] = F[p] / tau;
    int it, cy;
    double rr;
    if (g_linsolver == 1) {
      /* Sec. 4.1: the augmented finite-difference system, BiCG from theta = 0 */
      orc_bicg_fd(coef, h, N, M, o->eta, g_max_bicg, theta, &it, &rr);
      cy = 1;
    } else {
      orc_gmres_op(coef, abar, h, N, M, o->restart, o->eta, o->max_restarts, sigma, &it, &cy,
                   &rr);
      orc_apply_lbar_inv(abar, sigma, N, M, theta);
    }
    st->gmres_iters += it;
    st->gmres_cycles += cy;
    if (hist_gmres) hist_gmres[n] = it;
    for (;;) {
      for (long p = 0; p < P; ++p) cand[p] = u[p] + s * theta[p];
      orc_residual(f, c, cand, N, M, F, coef, scal);
      if (!o->safeguard || iterate_admissible(scal) || s < 0x1p-30) break;
      s *= 0.5;
      st->step_halvings++;
    }
    memcpy(u, cand, sizeof(double) * P);
    st->newton_iters = n + 1;
    s = (2.0 * s < 1.0) ? 2.0 * s : 1.0;
  }
  /* mean-zero gauge (Sec. 3.1): theta has zero mean by construction; remove the start's
   * mean and any rounding drift */
  double su = 0.0;
  for (long p = 0; p < P; ++p) su += u[p];
  st->u_mean = su / (double)P;
  for (long p = 0; p < P; ++p) u[p] -= st->u_mean;
out:
  st->status = status;
  free(f);
  free(g);
  free(c);
  free(F);
  free(coef);
  free(h);
  free(sigma);
  free(theta);
  free(cand);
  return status;
}

/* ------------------------------------------------------------------------------------ */
/* Learned warm start: FD Poisson solve and per-point features (not in the paper; the     */
/* network's inputs are built from the paper's quantities: the stencils, the interpolant   */
/* G, T = x + grad h and det(I + D^2 h) of Eq. ma2, at the linearised potential h).        */
/* ------------------------------------------------------------------------------------ */

/* Eigenvalue of the 4th-order second-difference stencil for frequency k on L points. */
static double fd2_eig(long k, int L) {
  double th = TWO_PI * (double)k / (double)L;
  return (-2.0 * cos(2.0 * th) + 32.0 * cos(th) - 30.0) / 12.0 * (double)L * (double)L;
}

/* out = the mean-zero solution of (D_xx + D_yy) out = src - mean(src), by division of the
 * spectrum by the stencil eigenvalues (the zero frequency is set to 0).  lowpass != 0 also
 * multiplies frequency (k1, k2) (signed, |k| <= L/2) by the Gaussian
 * exp(-((k1 / (M/4))^2 + (k2 / (N/4))^2) / 2). */
int orc_fd_poisson(const double *src, int N, int M, int lowpass, double *out) {
  long P = (long)N * M;
  double *re = (double *)malloc(sizeof(double) * P);
  double *im = (double *)calloc(P, sizeof(double));
  for (long p = 0; p < P; ++p) re[p] = src[p];
  int rc = orc_fft2(re, im, N, M, -1);
  for (int i = 0; i < N && rc == 0; ++i)
    for (int j = 0; j < M; ++j) {
      long p = (long)i * M + j;
      double lam = fd2_eig(j, M) + fd2_eig(i, N);
      double w = 1.0;
      if (lowpass) {
        double k1 = (double)(2 * j <= M ? j : j - M) / (0.25 * M);
        double k2 = (double)(2 * i <= N ? i : i - N) / (0.25 * N);
        w = exp(-0.5 * (k1 * k1 + k2 * k2));
      }
      if (i == 0 && j == 0) {
        re[p] = im[p] = 0.0;
      } else {
        re[p] *= w / lam;
        im[p] *= w / lam;
      }
    }
  if (rc == 0) rc = orc_fft2(re, im, N, M, +1);
  for (long p = 0; p < P; ++p) out[p] = re[p] / (double)P;
  free(re);
  free(im);
  return rc;
}

/* Features of the warm-start network at every grid point, ORC_WS_K per point:
 *   h = the linearised potential (orc_fd_poisson of log f - log g), T = x + grad h,
 *   G, grad G = the B-spline interpolant of g at T, det = det(I + D^2 h),
 *   lg = log max(G, floor), ld = log max(det, floor), iG = 1 / max(G, floor):
 *   [log f, log g, lg, log f - lg - ld, hxx + hyy, hxx - hyy, 2 hxy, hxx hyy - hxy^2,
 *    10 hx, 10 hy, 0.1 Gx iG, 0.1 Gy iG, (Gx hx + Gy hy) iG, (hxx - hyy)^2 + 4 hxy^2,
 *    (log f - lg - ld)(hxx + hyy), 0]. */
void orc_ws_features(const double *f, const double *g, const double *c, const double *h,
                     int N, int M, double *X) {
  const double floor_v = 1e-3;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < M; ++j) {
      long p = (long)i * M + j;
      double hx = d1x(h, N, M, i, j), hy = d1y(h, N, M, i, j);
      double hxx = d2x(h, N, M, i, j), hyy = d2y(h, N, M, i, j);
      double hxy = dxy(h, N, M, i, j);
      double G, Gx, Gy;
      orc_bspline_eval_grid(c, N, M, (double)j + (double)M * hx, (double)i + (double)N * hy,
                            &G, &Gx, &Gy);
      double det = (1.0 + hxx) * (1.0 + hyy) - hxy * hxy;
      double Gc = G > floor_v ? G : floor_v;
      double lf = log(f[p]), lg = log(Gc), ld = log(det > floor_v ? det : floor_v);
      double r = lf - lg - ld;
      double *x = X + p * ORC_WS_K;
      x[0] = lf;
      x[1] = log(g[p]);
      x[2] = lg;
      x[3] = r;
      x[4] = hxx + hyy;
      x[5] = hxx - hyy;
      x[6] = 2.0 * hxy;
      x[7] = hxx * hyy - hxy * hxy;
      x[8] = 10.0 * hx;
      x[9] = 10.0 * hy;
      x[10] = 0.1 * Gx / Gc;
      x[11] = 0.1 * Gy / Gc;
      x[12] = (Gx * hx + Gy * hy) / Gc;
      x[13] = (hxx - hyy) * (hxx - hyy) + 4.0 * hxy * hxy;
      x[14] = r * (hxx + hyy);
      x[15] = 0.0;
    }
}
