/*
 * ot_oracle.h -- FP64 CPU oracle of the damped-Newton Monge-Ampere OT solver
 * (arXiv:1009.6039).  TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and
 * the CPU-baseline leg of the benchmark, never by the CUDA product path.
 */
#ifndef OT_ORACLE_H
#define OT_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOCONV = -2, ORC_EDIVERGED = -3 };

typedef struct {
  double tau;          /* damping, tau >= 1 (Eq. linma) */
  double tol;          /* Newton stop: max|f - f~_n| < tol */
  double eta;          /* GMRES relative tolerance */
  int restart;         /* GMRES restart length m */
  int max_restarts;    /* GMRES cycle cap */
  int max_newton;      /* Newton step cap */
  int translate_inputs;/* apply Eq. (translation) to f and g on entry */
  int safeguard;       /* halve a step that loses convexity (larger effective tau) */
  double tau_switch;   /* tau schedule (0 = off): once max|F| < tau_switch the damping is 1
                          for the rest of the solve (a larger tau for the start, tau = 1 near
                          convergence: the remarks of Sec. 3.3 and the tau study of Sec. 5.1) */
} orc_opts;

typedef struct {
  int status;
  int newton_iters;
  int gmres_iters;
  int gmres_cycles;
  int step_halvings;
  double res_inf;
  double res_l2;
  double min_det;
  double mean_fn;
  double u_mean;
} orc_stats;

void orc_default_opts(orc_opts *o);
int orc_fft1(double *re, double *im, int L, int sign);
int orc_fft2(double *re, double *im, int N, int M, int sign);
int orc_dft2(const double *re, const double *im, int N, int M, int sign, double *o_re,
             double *o_im);
void orc_derivatives(const double *u, int N, int M, double *ux, double *uy, double *uxx,
                     double *uyy, double *uxy);
int orc_bspline_coeffs(const double *g, int N, int M, double *c);
void orc_bspline_eval(const double *c, int N, int M, double x, double y, double *val,
                      double *dgdx, double *dgdy);
void orc_bspline_eval_grid(const double *c, int N, int M, double gx_pos, double gy_pos,
                           double *val, double *dgdx, double *dgdy);
int orc_residual(const double *f, const double *c, const double *u, int N, int M, double *F,
                 double *coef, double *scal);
double orc_simpson_mean(const double *a, int N, int M);
void orc_apply_op(const double *coef, const double abar[5], const double *sigma, int N, int M,
                  double *w);
void orc_apply_lbar_inv(const double abar[5], const double *sigma, int N, int M,
                        double *theta);
int orc_gmres_dense(const double *A, const double *b, int n, int m, double eta,
                    int max_restarts, double *x, int *iters, int *cycles, double *relres);
int orc_gmres_op(const double *coef, const double abar[5], const double *h, int N, int M, int m,
                 double eta, int max_restarts, double *sigma, int *iters, int *cycles,
                 double *relres);
/* Sec. 4.1: y = A~ x and y = A~^T x for the second-order finite-difference operator with the
 * augmented row sum; BiCG on dense systems and on A~ theta = h; the Newton steps' solver */
void orc_fd_apply(const double *coef, const double *x, int N, int M, double *y);
void orc_fd_apply_t(const double *coef, const double *x, int N, int M, double *y);
int orc_bicg_dense(const double *A, const double *b, int n, double eta, int max_iters,
                   double *x, int *iters, double *relres);
int orc_bicg_fd(const double *coef, const double *h, int N, int M, double eta, int max_iters,
                double *theta, int *iters, double *relres);
void orc_set_linear_solver(int mode, int max_iters);
int orc_solve(const double *f_in, const double *g_in, int N, int M, const orc_opts *o,
              double *u, orc_stats *st, double *hist_res, int *hist_gmres);

/* symbols of the linear operator: 0 spectral (Sec. 4.2, default), 1 those of the stencils */
void orc_set_fd_symbols(int on);
/* 1: residual coefficients b1 = b2 = 0 (the simplified operator of the Sec. 3.3 remark) */
void orc_set_simplified(int on);
/* interpolation of g: 0 cubic B-spline (default), 1 bilinear, 2 nearest node */
void orc_set_interp(int mode);
int orc_get_interp(void);

/* learned warm start: FD Poisson solve and network features */
#define ORC_WS_K 16
int orc_fd_poisson(const double *src, int N, int M, int lowpass, double *out);
void orc_ws_features(const double *f, const double *g, const double *c, const double *h,
                     int N, int M, double *X);

#ifdef __cplusplus
}
#endif
#endif
