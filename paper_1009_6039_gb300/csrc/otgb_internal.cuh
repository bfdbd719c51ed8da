// Internal declarations shared by the CUDA translation units of libotgb.
// Grid convention: row-major N x M planes; row index i is y = i/N, column index j is
// x = j/M.  Half spectra are N x (M/2) complex in "packed" form: column 0 of every row
// holds the two real row coefficients X(k1 = 0) + i X(k1 = M/2).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dd.cuh"

#define OTGB_MAXM 16  // largest GMRES restart length + 1 held on the device

namespace otgb {

template <typename T> struct c2;
template <> struct c2<float> { using type = float2; };
template <> struct c2<double> { using type = double2; };
template <> struct c2<dd> { using type = ddc; };
template <typename T> using C2 = typename c2<T>::type;

// Scalars of one solve, resident in device memory.  Kernels that end in a grid-wide
// reduction write their block partials to a scratch array; the last block to finish
// (ticket counter) reduces them in a fixed order and updates this struct, so results are
// deterministic and no host round trip is needed.
struct DevScalars {
  // input translation (Eq. translation applied to f and g)
  double in_mean[2], in_min[2];
  int in_nonfinite[2];
  int in_bad;
  // residual / coefficient evaluation
  double mean_fn, shift, res_inf, min_det, abar[5];
  // the averaged coefficients of the current Newton iterate (Sec. 4.2), kept for theta =
  // Lbar^{-1} sigma: the residual at a candidate iterate writes abar, and a rejected
  // candidate must not change the operator of the step being halved
  double abar_n[5];
  double res_l2sum;
  int k1_nonfinite;
  int admissible;
  // GMRES(m) state
  double bnorm, beta;
  double H[(OTGB_MAXM + 1) * OTGB_MAXM];
  double cs[OTGB_MAXM], sn[OTGB_MAXM], gv[OTGB_MAXM + 1], y[OTGB_MAXM];
  double scale[OTGB_MAXM + 1];  // V_i is stored unnormalised; v_i = scale[i] * V_i
  double h2[OTGB_MAXM];         // second Gram-Schmidt pass (reorthogonalisation)
  double hcol[OTGB_MAXM];       // column j of H before the rotations (the update's weights)
  double relres;
  int j, jend, m, cycle_done, converged, iters, cycles;
  int jd;  // FP32 single-reduction step: the step index of the last multi-dot (for the update)
  double eta, tau;
  double tau_switch;  // tau schedule: tau becomes 1 once res_inf < tau_switch (0: off)
  // Newton control, resident on the device for the graph-launched solve
  double tol, step_s;
  // inexact-Newton forcing: forcing = 1 sets eta per step from eta_max and the residual
  // ratio (Eisenstat & Walker's choice 2); res_prev = max|F| at the previous step
  double eta_max, res_prev;
  int forcing;
  int newton_n, halvings, status, upar, safeguard, max_newton, max_restarts;
  int gmres_iters_total, gmres_cycles_total, graph, reorth;
  int steps_uncond;  // graph: Arnoldi steps 0..steps_uncond-1 of a cycle are not IF nodes
  int step_kernels;  // kernels per Arnoldi step: 5, 7 reorthogonalised, 4 fused update
  long long kcount;  // kernels executed by the graph-launched solve
  // conditional-node handles of the captured solve (0 outside a graph)
  unsigned long long h_newton, h_cycle, h_restart, h_halve, h_step[OTGB_MAXM];
  // learned warm start: the scale alpha applied to the network's potential, and an error
  // flag set by the network kernel (a bounded wait that gave up)
  double ws_alpha;
  // transport distance d(f, g) of ot_transport_outputs
  double dist;
  int ws_err;
  // device time per phase of a solve (OT_OPT_PHASE_TIMES): a one-thread stamp kernel at each
  // phase change adds the %globaltimer interval since the previous stamp to the phase that
  // stamp opened (PH_* below); stamp_cls = -1 before the first stamp
  unsigned long long stamp_t;
  unsigned long long phase_ns[5];
  // OT_OPT_PHASE_TIMES = 2: the same per kernel class (stamp codes 100 + class)
  unsigned long long class_ns[16];
  int stamp_cls;
  // 1 while the input statistics run without the translation (OT_OPT_TRANSLATE = 0): the
  // inputs must then be positive as given
  int in_plain;
  // per-pair flags of a batched solve (one DevScalars per pair): the pair's Newton loop
  // runs, it is in the current GMRES cycle loop, it repeats its candidate (step halving)
  int active, in_cycle, halve;
  int excluded;       // the pair sits out this launch of the batched graph (a retry of others)
  double gauge_mean;  // mean removed by the final gauge of a batched solve
  double pw_norm;     // 2-norm of the last vector normalised by launch_normalize
  // BiCG on the finite-difference system (Sec. 4.1): rho = (r, r*), alpha, beta, ||b||^2,
  // ||r||^2, the sums of p and p* (the all-ones part of A~ = A + 1 1^T); status 0 converged,
  // 1 iteration cap, 2 breakdown; done stops the self-skipping iteration kernels
  double bicg_rho, bicg_alpha, bicg_beta, bicg_b2, bicg_r2, bicg_sp, bicg_sps;
  int bicg_done, bicg_iters, bicg_max, bicg_status;
  // ticket counters of the last-block reductions
  unsigned int ticket[12];
};
// phases of OT_OPT_PHASE_TIMES
enum { PH_RESIDUAL = 0, PH_FFT = 1, PH_KRYLOV = 2, PH_UPDATE = 3, PH_OTHER = 4, PH_COUNT = 5 };

// Batched launches (the size classes of a plan set): B pairs of one grid size, each pair's
// buffers in its own slab of `slab` bytes at equal offsets, so that a pointer into pair b's
// memory is the pair-0 pointer plus b * slab.  A batched launch has gridDim.z = B (blockIdx.z
// is the pair); `mask` selects the pairs it serves (the other pairs' blocks return at once).
// The default (on = 0) is a plain single-problem launch.
enum { MASK_ALL = 0, MASK_NEWTON = 1, MASK_CYCLE = 2, MASK_HALVE = 3 };
struct Bat {
  int on = 0;  // a batched launch (of a plan set's size class, even of one pair)
  int n = 1;
  size_t slab = 0;
  int mask = MASK_ALL;
};
template <typename T>
__device__ __forceinline__ T* badv(T* p, const Bat& b) {
  return (p && b.on)
             ? reinterpret_cast<T*>(reinterpret_cast<uintptr_t>(p) + (size_t)blockIdx.z * b.slab)
             : p;
}
// the pair of this block does not take part in the launch (sc: this pair's scalars)
__device__ __forceinline__ bool bskip(const DevScalars* sc, const Bat& b) {
  if (b.on && sc->excluded) return true;
  if (b.mask == MASK_ALL) return false;
  if (!sc->active) return true;
  return (b.mask == MASK_CYCLE && !sc->in_cycle) || (b.mask == MASK_HALVE && !sc->halve);
}
inline dim3 bgrid(dim3 g, const Bat& b) { return dim3(g.x, g.y, b.on ? b.n : 1); }

// Control operations of the device-resident Newton loop (k_ctl)
enum CtlOp {
  CTL_NEWTON = 0,       // set status; continue while admissible, res >= tol, n < max
  CTL_ACCEPT = 1,       // accept the candidate (flip upar, n++, s = min(1, 2s)) or halve s
  CTL_PRE_CYCLE = 2,    // enter the GMRES cycle loop unless already converged
  CTL_CYCLE_BEGIN = 3,  // arm Arnoldi step 0, disarm the others
  CTL_CYCLE_END = 4,    // another cycle (with a restart residual) unless converged / capped
  CTL_GMRES_DONE = 5,   // accumulate the GMRES counters of this Newton step
  CTL_FORCING = 6       // GMRES tolerance of this Newton step (Eisenstat-Walker when set)
};

// The two buffers of the iterate u; `upar` in DevScalars names the current one.
struct UPair {
  double* a;
  double* b;
};

enum {
  TK_INPUT = 0,
  TK_RESID = 1,
  TK_DOTS = 2,
  TK_UPDATE = 3,
  TK_INIT = 4,
  TK_NORM = 5,
  TK_WS = 6,
  TK_TRANSPORT = 7,
  TK_BICG = 8
};

// Spectral kernels (instantiated for float and double) --------------------------------
// COL_POISSON: divide by the eigenvalues of the 4th-order stencil Laplacian (0 at k = 0);
// COL_POISSON_LP: the same times the Gaussian exp(-((k1/(M/4))^2 + (k2/(N/4))^2) / 2)
enum ColMode {
  COL_FWD = 0,
  COL_INV = 1,
  COL_MATVEC = 2,
  COL_LBARINV = 3,
  // 4: unused (the B-spline prefilter runs as recursive filters, launch_prefilter)
  COL_POISSON = 5,
  COL_POISSON_LP = 6
};
enum RowInvMode { ROWINV_PLAIN = 0, ROWINV_COMBINE = 1, ROWINV_UPDATE = 2 };

struct SpecTables {
  // twL and twN are each followed by the stage-ordered tables of widths 4, 8, 12 (one
  // transform length each; see stage_table_slot in spectral.cuh)
  const void* twL;  // exp(-2 pi i t / (M/2)), t < M/2 (row transforms)
  const void* twM;  // exp(-2 pi i k / M), k < M/2 (real-to-complex split)
  const void* twN;  // exp(-2 pi i t / N), t < N (column transforms)
  // derivative symbols of the linear operator, (s1, s2) per frequency index: i s1 the first-
  // derivative symbol (0 at Nyquist), s2 the second-derivative symbol; symx: k1 = 0..M/2,
  // symy: k2 index 0..N-1 (spectral 2 pi k, -(2 pi k)^2, or the 4th-order stencils')
  const void* symx = nullptr;
  const void* symy = nullptr;
  // kernel variants of the FP32 matvec passes (chosen by the plan's autotuner):
  // -1 default, 0 generic (8 or 12 elements per thread, one transform after the other),
  // 1 concurrent transforms in separate thread groups, 2 warp-synchronous radix-32,
  // 3 generic with 4 elements per thread (radix 4, twice the threads; power-of-two lengths),
  // 4 column / row pairs with packed FP32 arithmetic (spectral_pair.cu, row_pair.cu)
  int var_r2c = -1, var_col = -1, var_comb = -1;
  // generic column matvec pass: columns per block (0: the default heuristic)
  int col_q = 0;
  // register-resident matvec passes on the transposed half spectrum (FP32, power-of-two
  // lengths 64..1024; spectral_reg.cu): mv_reg = 1 uses them for all three passes.
  // Exchange twiddles W_L^{t ka} of the two-level transforms, for the row length L = M/2
  // (t2r) and the column length N (t2c): A at [ka * (L/32) + t], B at [t * 32 + ka].
  int mv_reg = 0;
  // theta's double-float column / row passes and the warm start's Poisson solves on column /
  // row pairs with packed arithmetic where the sizes allow (spectral_pair_dd.cu)
  int theta_pair = 0;
  const void* t2rA = nullptr;
  const void* t2rB = nullptr;
  const void* t2cA = nullptr;
  const void* t2cB = nullptr;
};
enum { VAR_DEFAULT = -1, VAR_GENERIC = 0, VAR_PAR = 1, VAR_WARP = 2, VAR_E4 = 3, VAR_PAIR = 4 };

// the FP32 row combine pass on row pairs (M / 2 a power of two in 256..1024, N even)
bool comb_pair_supported(int N, int M);
cudaError_t launch_comb_pair(const float2* q0, const float2* q1, const float2* q2,
                             const float* coef, float* out, int N, int M, const SpecTables& tb,
                             const int* skip, cudaStream_t st);
// the FP32 row real-to-complex pass on row pairs, and the Arnoldi update fused with it
// (the sizes of the combine pair pass)
cudaError_t launch_row_r2c_pair(const float* x, size_t xs, const int* jptr, const double* scale,
                                float2* spec, int N, int M, const SpecTables& tb,
                                const int* skip, cudaStream_t st);
cudaError_t launch_gmres_update_r2c_pair(float* V, const float* w, long P,
                                         const double* partials, int nb, DevScalars* sc,
                                         float2* spec, int N, int M, const SpecTables& tb,
                                         cudaStream_t st);
// theta's double-float column pass (modes COL_LBARINV, COL_POISSON, COL_POISSON_LP) on
// column pairs and its row pass + update on row pairs (the sizes of the FP32 pair passes)
cudaError_t launch_col_lbarinv_pair(const float2* spec, ddc* out, int N, int M,
                                    const SpecTables& tb32, const SpecTables& tbdd,
                                    const DevScalars* sc, cudaStream_t st, int mode);
cudaError_t launch_row_update_pair(const ddc* q, const double* u_in, double* u_out,
                                   double step, int N, int M, const SpecTables& tbdd,
                                   const DevScalars* sc, cudaStream_t st);
// the FP32 column matvec pass on column pairs (power-of-two N in 256..2048, M % 4 == 0)
bool col_pair_supported(int N, int M);
cudaError_t launch_col_pair(const float2* spec, float2* o0, float2* o1, float2* o2, int N,
                            int M, const SpecTables& tb, const DevScalars* sc, const int* skip,
                            cudaStream_t st);

bool fft_length_supported(int L);

// (bat: a batched launch, the generic kernels only; msc: the pair scalars its mask reads)
template <typename T>
cudaError_t launch_row_r2c(const T* x, size_t x_stride, const int* jptr, const double* scale,
                           C2<T>* spec, int N, int M, const SpecTables& tb, const int* skip,
                           cudaStream_t st, Bat bat = Bat(), const DevScalars* msc = nullptr);
template <typename T>
cudaError_t launch_col(int mode, const C2<T>* spec, C2<T>* out0, C2<T>* out1, C2<T>* out2,
                       int N, int M, const SpecTables& tb, const DevScalars* sc,
                       const int* skip, cudaStream_t st, Bat bat = Bat());
template <typename T>
cudaError_t launch_row_c2r(int mode, const C2<T>* q0, const C2<T>* q1, const C2<T>* q2,
                           const T* coef, T* out, const double* u_in, double* u_out,
                           double step, double out_scale, int N, int M, const SpecTables& tb,
                           const int* skip, cudaStream_t st, const DevScalars* sc = nullptr,
                           Bat bat = Bat());

// register-resident FP32 matvec passes on the transposed half spectrum specT (M/2 x N,
// entry (k1, k2) at k1 N + k2): mvT_supported(N, M) when N and M/2 are powers of two in
// 64..1024
bool mvT_supported(int N, int M);
cudaError_t launch_mvT_r2c(const float* x, size_t x_stride, const int* jptr,
                           const double* scale, float2* specT, int N, int M,
                           const SpecTables& tb, const int* skip, cudaStream_t st);
cudaError_t launch_mvT_col(const float2* specT, float2* out0, float2* out1, float2* out2,
                           int N, int M, const SpecTables& tb, const DevScalars* sc,
                           const int* skip, cudaStream_t st);
cudaError_t launch_mvT_combine(const float2* q0T, const float2* q1T, const float2* q2T,
                               const float* coef, float* out, int N, int M,
                               const SpecTables& tb, const int* skip, cudaStream_t st);

// theta = Lbar^{-1} sigma column pass, FP32 forward / FP64 inverse (mixed mode)
cudaError_t launch_col_lbarinv_mixed(const float2* spec, double2* out, int N, int M,
                                     const SpecTables& tb32, const SpecTables& tb64,
                                     const DevScalars* sc, cudaStream_t st);
// the same with the inverse column transform in double-float (tbdd: dd twiddle tables);
// mode COL_POISSON / COL_POISSON_LP: the FD Poisson solve of the warm start instead (sc
// unused)
cudaError_t launch_col_lbarinv_dd(const float2* spec, ddc* out, int N, int M,
                                  const SpecTables& tb32, const SpecTables& tbdd,
                                  const DevScalars* sc, cudaStream_t st,
                                  int mode = COL_LBARINV, Bat bat = Bat());
// theta rows in double-float and the update u_out = u_in + step theta (FP64 u; u_in may be
// null: u_out = step theta); with sc, step and the buffer pair come from the device scalars
// (graph)
cudaError_t launch_row_c2r_update_dd(const ddc* q, const double* u_in, double* u_out,
                                     double step, int N, int M, const SpecTables& tbdd,
                                     const DevScalars* sc, cudaStream_t st, Bat bat = Bat());

// Residual / coefficients, input translation ------------------------------------------
// c = cubic B-spline coefficients of g (periodic), by recursive filters along y then x
// (scratch: N x M FP64); cdd (optional) also receives c as (hi, lo) float pairs
cudaError_t launch_prefilter(const double* g, double* scratch, double* c, float2* cdd, int N,
                             int M, cudaStream_t st, Bat bat = Bat());
cudaError_t launch_translate_inputs(const double* f, const double* g, double* ft, double* gt,
                                    int N, int M, double* partials, DevScalars* sc,
                                    cudaStream_t st, Bat bat = Bat());
// the statistics of f and g alone (means, minima, non-finite counts) for inputs used as given
// (sc->in_plain must be 1: then in_bad flags a non-positive or non-finite value)
cudaError_t launch_input_stats(const double* f, const double* g, int N, int M,
                               double* partials, DevScalars* sc, cudaStream_t st,
                               Bat bat = Bat());
// phase stamp (OT_OPT_PHASE_TIMES): cls opens a phase, -1 closes the last one
cudaError_t launch_stamp(DevScalars* sc, int cls, cudaStream_t st);
// interpolation of g at the displaced points: mode 0 cubic B-spline of the coefficients c;
// 1 bilinear, 2 nearest node of the grid values (c = g) and of the grid gradient (gx, gy in
// FP64 for the FP64 kernel, gx32, gy32 for the double-float one)
struct Interp {
  int mode = 0;
  const double* gx = nullptr;
  const double* gy = nullptr;
  const float* gx32 = nullptr;
  const float* gy32 = nullptr;
};
cudaError_t launch_grad4(const double* g, int N, int M, double* gx, double* gy, float* gx32,
                         float* gy32, cudaStream_t st);
// u = ub ? (upar ^ sel ? ub : ua) : ua   (sel 0: current iterate, 1: candidate);
// simplified: b = 0 in the coefficients (the operator without the grad g term)
// c32 (optional, FP32 copy of c): used for the gradient of the interpolant in FP32 mode
template <typename T>
cudaError_t launch_residual(const double* f, const double* c, const double* ua, int N, int M,
                            double* Fraw, T* coef, double* partials, DevScalars* sc,
                            cudaStream_t st, const double* ub = nullptr, int sel = 0,
                            const float* c32 = nullptr, int simplified = 0,
                            Interp ip = Interp());
// mixed mode: the residual in double-float arithmetic from (hi, lo) float pairs of f and c
cudaError_t launch_residual_dd(const float2* fdd, const float2* cdd, const double* ua, int N,
                               int M, double* Fraw, float* coef, double* partials,
                               DevScalars* sc, cudaStream_t st, const double* ub = nullptr,
                               int sel = 0, int simplified = 0, Bat bat = Bat(),
                               Interp ip = Interp());
// out[k] = (hi, lo) float pair of in[k]
cudaError_t launch_split_dd(const double* in, float2* out, long n, cudaStream_t st,
                            Bat bat = Bat());
cudaError_t launch_residual_l2(const double* Fraw, int N, int M, double* partials,
                               DevScalars* sc, cudaStream_t st, Bat bat = Bat());
cudaError_t launch_shifted_residual(const double* Fraw, double* F, int N, int M,
                                    const DevScalars* sc, cudaStream_t st);
cudaError_t launch_subtract_mean(double* u, int N, int M, double* partials, DevScalars* sc,
                                 double* mean_out, cudaStream_t st);
// out = u[upar] - mean(u[upar])
cudaError_t launch_final_gauge(UPair u, double* out, int N, int M, double* partials,
                               DevScalars* sc, double* mean_out, cudaStream_t st,
                               Bat bat = Bat());
// kernel timing: sc->j = j, cycle open (one thread)
cudaError_t launch_set_step(DevScalars* sc, int j, cudaStream_t st);
// x <- x / ||x||_2 (two launches: the norm into sc->pw_norm, then the scaling; x = 0 stays 0)
cudaError_t launch_normalize(double* x, long P, double* partials, DevScalars* sc,
                             cudaStream_t st);
// Finite-difference comparison path (Sec. 4.1): the BiCG vectors (FP64 planes) ...
struct FdBufs {
  double *x, *r, *rs, *p, *ps, *q, *qs;
};
// ... set up from b = h (when given) or (F_raw + shift) / tau, x = 0 ...
cudaError_t launch_bicg_init(const double* Fraw, const double* h, FdBufs b, long P,
                             double* partials, DevScalars* sc, int max_iters,
                             cudaStream_t st);
// ... and one BiCG iteration on A~ x = b (three launches that skip themselves once
// sc->bicg_done is set); coef: the residual's 5 coefficient planes
cudaError_t launch_bicg_iteration(const double* coef, FdBufs b, int N, int M,
                                  double* partials, DevScalars* sc, cudaStream_t st);
// y = A~ x or A~^T x (tmp: a scratch plane; needs sc->bicg_done = 0)
cudaError_t launch_fd_apply(const double* coef, const double* x, int transpose, double* y,
                            double* tmp, int N, int M, double* partials, DevScalars* sc,
                            cudaStream_t st);
// u_out = u_in + s theta
cudaError_t launch_axpy_to(const double* u_in, const double* th, double s, double* u_out,
                           long P, cudaStream_t st);
// batched solve: dst (pair 0's plane, advanced by the slab per pair) <- tab[pair]; and the
// reverse (tab[pair] <- src of pair), skipping excluded pairs (sc: pair 0's scalars)
cudaError_t launch_gather(const double* const* tab, double* dst, long P, Bat bat,
                          cudaStream_t st);
cudaError_t launch_scatter(const double* src, double* const* tab, long P, const DevScalars* sc,
                           Bat bat, cudaStream_t st);
// `add`: kernels of the graph segment this control op closes (launch accounting); batched:
// one thread per pair, the handle set to "any pair continues" (at most 1024 pairs)
cudaError_t launch_ctl(int op, DevScalars* sc, cudaStream_t st, int add = 0, Bat bat = Bat());
int residual_partial_blocks(int N, int M);

// Krylov kernels -------------------------------------------------------------------------
// restart 0: V0 = h (and sigma = 0 when sigma is given); 1: V0 = h - w
template <typename T>
cudaError_t launch_gmres_init(const double* Fraw, const T* w, T* V0, long P, int restart,
                              double* partials, DevScalars* sc, int nblocks, cudaStream_t st,
                              T* sigma = nullptr, Bat bat = Bat());
// pass 0: H[:, j] = V^T w; pass 1 (reorthogonalisation): h2 = V^T V_{j+1}, H[:, j] += h2
template <typename T>
cudaError_t launch_gmres_dots(const T* V, const T* w, long P, double* partials, DevScalars* sc,
                              int nblocks, cudaStream_t st, int pass = 0, Bat bat = Bat());
// mode 0: V_{j+1} = w - V H[:, j], norm + Givens; mode 1: the same without norm (first of
// two passes); mode 2: V_{j+1} -= V h2 in place, norm + Givens
template <typename T>
cudaError_t launch_gmres_update(T* V, const T* w, long P, double* partials, DevScalars* sc,
                                int nblocks, cudaStream_t st, int mode = 0, Bat bat = Bat());
// FP32, single problem: the split update of step jd (block 0 closes the step) fused with the
// row real-to-complex pass of step jd + 1's product on v_(jd+1) / hn (gmres_fused.cu); nb:
// the multi-dot's block count.  update_r2c_fits: whether the fused form exists for this size
// and row-pass variant.
bool update_r2c_fits(int N, int M, int var_r2c);
cudaError_t launch_gmres_update_r2c(float* V, const float* w, long P, const double* partials,
                                    int nb, DevScalars* sc, float2* spec, int N, int M,
                                    const SpecTables& tb, cudaStream_t st);
cudaError_t launch_gmres_finish(DevScalars* sc, cudaStream_t st, Bat bat = Bat());
template <typename T>
cudaError_t launch_gmres_combine(const T* V, T* sigma, long P, const DevScalars* sc,
                                 int nblocks, cudaStream_t st, Bat bat = Bat());
template <typename T>
cudaError_t launch_convert(const void* in, int in_is_double, void* out, int out_is_double,
                           long n, cudaStream_t st);

// Learned warm start ---------------------------------------------------------------------
#define OTGB_WS_K 16    // features per grid point
#define OTGB_WS_H 128   // hidden units per layer (three hidden layers)
#define WS_ROW_CHUNK 2048  // rows per partial sum of the weight gradients
constexpr long ws_param_count() {
  return (long)OTGB_WS_H * OTGB_WS_K + OTGB_WS_H +
         2 * ((long)OTGB_WS_H * OTGB_WS_H + OTGB_WS_H) + OTGB_WS_H + 1;
}
// buffers of one training step with B rows (FP32 unless noted)
struct WsTrainBuffers {
  float *Xb, *tb;                  // gathered rows (B x 16) and targets (B)
  float *Z0, *A0, *Z1, *A1, *Z2, *A2;  // pre-activations / activations (B x H each)
  float *dy, *dZ1, *dZ2;           // output gradient (B), layer gradients (B x H)
  float *part;                     // partial sums: ceil(B / WS_ROW_CHUNK) x H x H
  float *grad;                     // gradient (ws_param_count())
  double *loss_part, *loss;        // ceil(B / 8) partials, mean squared error
};
cudaError_t launch_ws_source(const double* f, const double* g, double* src, long P,
                             cudaStream_t st);
// transport outputs: *dist (device) = mean |grad u|^2 f, div (optional) = u_xx + u_yy;
// partials: one (hi, lo) pair per 32 x 32 tile
cudaError_t launch_transport(const double* f, const double* u, int N, int M, double* div,
                             double* partials, unsigned int* ticket, double* dist,
                             cudaStream_t st);
// the same source in FP32 (input of the mixed-precision Poisson solve)
cudaError_t launch_ws_source32(const double* f, const double* g, float* src, long P,
                               cudaStream_t st);
// c32: FP32 copy of the B-spline coefficients of g
cudaError_t launch_ws_features(const double* f, const double* g, const float* c32,
                               const double* h, int N, int M, float* X, cudaStream_t st);
// t = (D_xx + D_yy)(phi - h); scratch: N x M FP64
cudaError_t launch_ws_target(const double* phi, const double* h, int N, int M, double* scratch,
                             float* t, cudaStream_t st);
// out = (double)s
cudaError_t launch_ws_widen(const float* s, double* out, long P, cudaStream_t st);
// u = h + t
cudaError_t launch_ws_sum(const double* h, const double* t, double* u, long P, cudaStream_t st);
int ws_admissible_blocks(int N, int M);
// alpha = largest of 1, 1/2, 1/4, 1/8 with det(I + alpha D^2 u) > 0 (0 if none or *err);
// then u *= alpha.  partials: 4 x ws_admissible_blocks(N, M) doubles; *ticket must start
// at 0.
cudaError_t launch_ws_admissible(double* u, int N, int M, double* partials,
                                 unsigned int* ticket, const int* err, double* alpha,
                                 cudaStream_t st);
size_t ws_packed_bytes();
cudaError_t launch_ws_pack(const float* params, unsigned char* wpack, cudaStream_t st);
// BF16 tensor-core forward of the network: out[r] = MLP(X[r, :]); *err set on a timeout
// (stall != 0 makes one wait run out on purpose: a test of that path)
cudaError_t launch_ws_mlp(const unsigned char* wpack, const float* params, const float* X,
                          long rows, float* out, int* err, int sms, cudaStream_t st,
                          int stall = 0);
// gradient of the mean squared error over the rows idx[0..B) of (X, t) into tb.grad
cudaError_t launch_ws_grad(const float* params, const float* X, const float* t,
                           const long long* idx, int B, WsTrainBuffers& tb, cudaStream_t st);
cudaError_t launch_ws_adam(float* p, float* m, float* v, const float* g, long n, float lr,
                           int t, cudaStream_t st);

}  // namespace otgb
