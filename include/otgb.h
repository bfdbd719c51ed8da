/*
 * otgb.h -- C ABI of libotgb, a GB300 (sm_103a) solver for the periodic L2 optimal
 * transport problem by the damped-Newton Monge-Ampere method of Saumier, Agueh & Khouider
 * (arXiv:1009.6039).
 *
 * Problem (Sec. 2, Sec. 3.1 Eq. ma2): given 1-periodic densities f, g > 0 on the unit
 * square, find a 1-periodic potential phi with mean zero such that
 *     g(x + grad phi) det(I + D^2 phi) = f,
 * so that T(x) = x + grad phi(x) is the optimal map pushing f onto g.
 *
 * Conventions for every entry point:
 *   - Planes are row-major N x M arrays of double: element (i, j) at [i * M + j], row index
 *     i is y = i / N, column index j is x = j / M.
 *   - Unless stated otherwise, pointers are DEVICE pointers (cudaMalloc / torch CUDA
 *     tensors) on the current device, owned by the caller, and every call is
 *     stream-ordered on the plan's stream and returns after the results are complete.
 *   - Every call returns OT_OK (0) or a negative status code; ot_strerror() names it.
 *     On an error the output buffers may have been partly written.
 *   - N and M must be even, each of the form 2^a (>= 8) or 3 * 2^a (>= 12), M >= 16, and
 *     at most 2048 (the supported FFT lengths; M/2 must also be supported).
 */
#ifndef OTGB_H
#define OTGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define OT_OK 0
#define OT_EINVAL (-1)       /* bad argument: size, tau < 1, tol <= 0, null pointer, or an
                                input density that is non-finite or not positive after the
                                mean translation of Eq. (translation) */
#define OT_ENOCONV (-2)      /* max Newton steps reached; phi holds the last iterate */
#define OT_EDIVERGED (-3)    /* an iterate lost convexity (det(I + D^2 phi) <= 0) or became
                                non-finite; phi holds that last iterate */
#define OT_ECUDA (-4)        /* a CUDA runtime call failed */
#define OT_ENOMEM (-5)       /* device or pinned-host allocation failed */
#define OT_EUNSUPPORTED (-6) /* grid size outside the supported FFT lengths */
#define OT_ETIMEOUT (-7)     /* a bounded device-side wait gave up (the kernel returned and
                                reported it through its flag; the context stays usable) */

/* Plan options (ot_plan_set_option keys). */
#define OT_OPT_RESTART 1        /* GMRES restart length m, 1..15 (default 10, Sec. 5.1) */
#define OT_OPT_ETA 2            /* GMRES relative tolerance (default 1e-4, Sec. 5.1) */
#define OT_OPT_MAX_NEWTON 3     /* Newton step cap (default 200) */
#define OT_OPT_MAX_RESTARTS 4   /* GMRES cycle cap per Newton step (default 50) */
#define OT_OPT_PRECISION 5      /* 0 = FP64 throughout (default); 1 = mixed: FFTs, the
                                   preconditioner and Krylov vectors in FP32, residual,
                                   det/cof, update and convergence test in FP64 */
#define OT_OPT_SAFEGUARD 6      /* 1 (default): halve a Newton step whose iterate loses
                                   convexity (a larger effective tau, Sec. 3.2 remarks);
                                   0: plain Eq. (linma), such an iterate ends the solve */
#define OT_OPT_TRANSLATE 7      /* 1 (default): apply Eq. (translation) d - mean(d) + 1 to
                                   f and g on entry; 0: use them as given (they must then be
                                   positive and finite as they are, else OT_EINVAL) */
#define OT_OPT_WARM_START 8     /* 1: phi_inout holds the initial iterate u0 on entry;
                                   0 (default): u0 = 0, the constant start of Thm 3.2;
                                   2: u0 = the learned warm start (ot_ws_set_weights or
                                   ot_warmstart_load first, else OT_EINVAL) */
#define OT_OPT_TAU 9            /* step-size parameter tau >= 1 (Eq. linma) */
#define OT_OPT_TOL 10           /* Newton stop: max |f - f~_n| < tol */
#define OT_OPT_PROFILE 11       /* 1: time every kernel launch with CUDA events on the
                                   plan's stream, per class below (default 0); forces the
                                   host-driven solve (OT_OPT_GRAPH is ignored meanwhile) */
#define OT_OPT_GRAPH 12         /* 1 (default): run the whole solve as one CUDA graph whose
                                   Newton, GMRES-cycle, Arnoldi-step and step-halving loops
                                   are conditional nodes driven by device-side tests (no host
                                   round trip until the end); 0: host-driven loop that
                                   synchronises once per GMRES cycle and per Newton step */
#define OT_OPT_REORTH 13        /* 0 (default): one classical Gram-Schmidt pass per Arnoldi
                                   step; 1: two passes (reorthogonalisation) */
#define OT_OPT_THETA_FP64 14    /* mixed mode only: precision of the inverse transforms of
                                   theta = Lbar^{-1} sigma and of the update: 2 (default)
                                   double-float (FP32 pairs, 48-bit significand), 1 FP64,
                                   0 FP32 (FP32 round-off in theta is amplified ~M^2 by the
                                   stencils at the grid scale and slows the Newton tail) */
#define OT_OPT_AUTOTUNE 15      /* mixed mode: 1 (default) times the kernel variants of the
                                   FP32 transform passes at the first solve of each grid size
                                   and keeps the fastest (cached per size in the process) */
#define OT_OPT_SYMBOLS 17       /* derivative symbols of the linear operator L and of Lbar:
                                   0 (default) the spectral symbols 2 pi i k, -(2 pi k)^2 of
                                   Sec. 4.2; 1 the Fourier symbols of the 4th-order stencils
                                   that F itself uses, (8 sin t - sin 2t)/(6h) and
                                   (-2 cos 2t + 32 cos t - 30)/(12 h^2), t = 2 pi k h, which
                                   make L the exact linearisation of F (Newton then converges
                                   quadratically at tau = 1 with accurate inner solves) */
#define OT_OPT_FORCING 18       /* GMRES tolerance per Newton step: 0 (default) the fixed
                                   OT_OPT_ETA; 1 Eisenstat & Walker's choice 2 (eta_k =
                                   0.9 (|F_k| / |F_k-1|)^2, safeguarded, capped by OT_OPT_ETA
                                   and no tighter than 0.5 tol / |F_k|) */
#define OT_OPT_TAU_RETRY 19     /* 0..8 (default 0): when a solve ends with OT_EDIVERGED
                                   (an iterate lost convexity), solve again from the start
                                   with twice tau, up to this many times -- the remedy of
                                   Sec. 3.2 / Sec. 5.3; phi and stats are those of the last
                                   attempt (ot_solve, ot_solve_batched) */
#define OT_OPT_WS_TEST_STALL 20 /* test of the failure path: 1 makes the next
                                   ot_ws_mlp_forward, or the network launch of the next
                                   host-driven solve (OT_OPT_GRAPH = 0) with the learned warm
                                   start, skip one tensor-core MMA group, so its bounded
                                   mbarrier wait runs out (tens of milliseconds); the kernel
                                   sets its error flag, frees its TMEM and returns;
                                   ot_ws_mlp_forward then returns OT_ETIMEOUT, the solve goes on
                                   from the zero start with ws_alpha = -2; resets itself after
                                   one use */
#define OT_OPT_OPERATOR 21      /* linear operator of the Newton step: 0 (default) the full
                                   linearisation of Eq. linearmaeq (a : D^2 theta + b . grad
                                   theta, b = det(I + D^2 u) grad g(x + grad u)); 1 the
                                   simplified g(x + grad u) Tr(Adj(I + D^2 u) D^2 theta) that
                                   Sec. 3.3 reports working in practice (b = 0; the same root,
                                   a different Newton path) */
#define OT_OPT_PHASE_TIMES 22  /* 1: the solve records the device time of each phase
                                   (ms_residual, ms_fft, ms_krylov, ms_update, ms_other of
                                   ot_stats) with a one-thread stamp kernel (%globaltimer) at
                                   every phase change, in the graph and the host-driven solve
                                   alike (a few microseconds per phase change; the stamps are
                                   not in kernel_launches); 2: the same at every change of
                                   kernel class (OT_PROF_*): the phase fields are then the
                                   sums of their classes (theta's row R2C counted with the
                                   transforms) and ot_plan_get_profile returns the device ms
                                   per class of the last solve (launch counts 0); 0
                                   (default): those fields are -1 */
#define OT_OPT_TRANSPORT 23     /* 1: the solve ends with the transport distance d(f, g) of
                                   Sec. 5.2 (as ot_transport_outputs, on the translated f) in
                                   ot_stats.transport_dist; 0 (default): it is -1 */
#define OT_OPT_TAU_SWITCH 24    /* tau schedule: 0 (default) off; s > 0: once max|F| < s the
                                   damping is 1 for the rest of the solve (a larger tau for
                                   the start, tau = 1 near convergence; the remarks of Sec. 3.3
                                   and the tau study of Sec. 5.1) */
#define OT_OPT_INTERP 25        /* g and grad g at the displaced points x + grad phi: 0
                                   (default) the periodic cubic B-spline interpolant of g and
                                   its exact gradient; 1 bilinear, 2 nearest grid node (Sec. 4:
                                   closest-neighbour interpolation for images, Sec. 5.2;
                                   linear, Sec. 5.3) of the grid values of g and, by the same
                                   rule, of its grid gradient by the 4th-order centred
                                   differences (then no prefilter: ot_prefilter copies g and
                                   ot_eval_residual takes g for c); not with the learned warm
                                   start (OT_EINVAL) nor in plan sets */
#define OT_OPT_LINEAR_SOLVER 26 /* linear solver of the Newton steps: 0 (default) the Fourier
                                   method of Sec. 4.2 (Strain's preconditioned GMRES(m)); 1 the
                                   paper's comparison path of Sec. 4.1: second-order centred
                                   differences of theta, the extra equation sum theta = 0
                                   added to every row (A~ = A + 1 1^T), unpreconditioned BiCG
                                   from theta = 0 to ||r|| <= eta ||b||.  FP64 only (OT_EINVAL
                                   in the mixed mode, and OPT_PRECISION = 1 is refused while it
                                   is set); the solve then runs host-driven whatever
                                   OT_OPT_GRAPH says (the state read once per 16 iterations);
                                   gmres_iters / gmres_cycles of ot_stats count BiCG iterations
                                   and BiCG runs, and its launches are profiled as
                                   OT_PROF_GMRES_OTHER.  Setting 1 allocates 7 FP64 planes */
#define OT_OPT_MAX_BICG 27      /* BiCG iterations per Newton step, >= 1 (default 20000) */
#define OT_OPT_UNCOND_STEPS 28  /* graph structure: the first s Arnoldi steps of every GMRES
                                   cycle are captured as plain kernels that skip themselves
                                   once the cycle has ended, the later ones as the body of one
                                   conditional WHILE node, a step per iteration (0 <= s <= 16,
                                   default 7; a plan set captures every step plainly).  Same
                                   arithmetic for every s */
#define OT_OPT_KRYLOV_BLOCKS 29 /* blocks of 256 threads per SM for the GMRES vector kernels
                                   (multi-dot, update, init, combine), 1..8 (default 2); the
                                   block partial sums change with it, so results differ in
                                   the last bits between settings (each is deterministic) */
#define OT_OPT_L2_PERSIST 30    /* 1: the graph-launched solve marks the GMRES basis V_0..V_m
                                   as persisting L2 lines (an access-policy window on its
                                   kernels; the process's persisting-L2 limit is raised to
                                   the window, at most the device maximum), so that the
                                   transform passes between two Arnoldi steps do not evict it;
                                   0 (default): no window.  Same arithmetic either way */
#define OT_OPT_FUSED_UPDATE 31  /* mixed mode, single problem: 1 (default) runs each Arnoldi
                                   step's update fused with the row transform pass of the
                                   next step's product (the update forms v_(j+1) row by row
                                   and transforms it in place of a separate row pass); 0: two
                                   launches.  Same arithmetic either way (bit for bit) */
#define OT_OPT_THETA_PAIRS 32   /* mixed mode, double-float theta (OT_OPT_THETA_FP64 = 2),
                                   single problem: 1 (default) runs theta's column and row
                                   passes and the learned start's Poisson solves on column /
                                   row pairs with packed FP32 arithmetic where the sizes allow
                                   (N a power of two in 256..2048 and M a multiple of 4 for the
                                   column pass, M/2 a power of two in 256..1024 and N even for
                                   the row pass); 0: one column / row per thread group.  The
                                   double-float inverse transforms are the same arithmetic per
                                   column either way; the FP32 forward column transform
                                   rounds differently */
#define OT_OPT_FFT_VARIANT 16   /* mixed mode: fix the FP32 transform kernels instead of
                                   autotuning: value r + 4 c + 16 b with r (row R2C), c
                                   (column matvec) and b (row combine) each 0 = generic,
                                   1 = concurrent transforms (r: same as 0), 2 = warp-
                                   synchronous radix-32, 3 = generic with 4 elements per
                                   thread (where the size allows, else a variant that does);
                                   + 64: the generic column pass with 4 columns per block;
                                   + 256: the column pass on column pairs with packed FP32
                                   arithmetic (N a power of two in 256..2048, M a multiple
                                   of 4; elsewhere c = 3); + 512: the combine pass on row
                                   pairs (M/2 a power of two in 256..1024, N even; elsewhere
                                   b = 3); + 1024: the row R2C pass and the fused Arnoldi
                                   update on row pairs (the same sizes; elsewhere r = 3);
                                   turns OT_OPT_AUTOTUNE off */

/* Kernel classes of the profile (ot_plan_get_profile). */
#define OT_PROF_RESIDUAL 0         /* residual + coefficients (Eq. ma2, linearmaeq) */
#define OT_PROF_ROW_R2C 1          /* row real-to-complex FFT pass (matvec and theta) */
#define OT_PROF_COL_MATVEC 2       /* column FFT pass with the rho-bar and symbol multiplies */
#define OT_PROF_ROW_C2R_COMBINE 3  /* row complex-to-real pass, coefficient apply */
#define OT_PROF_COL_LBARINV 4      /* column pass of theta = Lbar^{-1} sigma */
#define OT_PROF_ROW_C2R_UPDATE 5   /* row complex-to-real pass of theta, u += s theta */
#define OT_PROF_GMRES_DOTS 6       /* Arnoldi multi-dot */
#define OT_PROF_GMRES_UPDATE 7     /* Arnoldi update + norm + Givens */
#define OT_PROF_GMRES_OTHER 8      /* GMRES init / restart residual / finish / combine */
#define OT_PROF_OTHER 9            /* input translation, prefilter, final reductions */
#define OT_PROF_WARMSTART 10       /* learned warm start (features, network, Poisson solves) */
#define OT_PROF_CLASSES 11
/* ot_plan_time_kernel only (not a profile class): the learned warm start's network kernel
 * (BF16 tcgen05) on the plan's feature planes, one row per grid point; needs a plan with
 * weights set that has run a solve with the learned warm start */
#define OT_TIME_WS_NETWORK 32

typedef struct ot_plan ot_plan;

/* Filled by the solve entry points. */
typedef struct {
  int32_t status;          /* same value as returned */
  int32_t newton_iters;    /* accepted Newton updates */
  int32_t gmres_iters;     /* Arnoldi steps, all Newton steps */
  int32_t gmres_cycles;    /* GMRES(m) cycles begun, all Newton steps */
  int32_t step_halvings;   /* safeguard rejections */
  int32_t kernel_launches; /* CUDA kernels launched by the call */
  double res_inf;          /* max |f - f~_n| at the returned phi */
  double res_l2;           /* sqrt(mean (f - f~_n)^2) at the returned phi */
  double min_det;          /* min det(I + D^2 phi) */
  double mean_fn;          /* mean of f_n before translation (mass defect = mean_fn - 1) */
  double phi_mean;         /* mean removed from the final iterate (gauge, Sec. 3.1) */
  double ms_total;         /* wall time of the call on the plan's stream (ms) */
  double ws_alpha;         /* learned warm start: scale applied to the network's potential
                              (1, 1/2, 1/4, 1/8 or 0 = zero start); -1 without it; -2 if
                              the network kernel's bounded wait gave up (the solve went on
                              from the zero start and ot_last_error names it) */
  double mass_defect_f;    /* mean(f) - 1 of the input f, before Eq. (translation) */
  double mass_defect_g;    /* mean(g) - 1 of the input g */
  double transport_dist;   /* d(f, g) = mean |grad phi|^2 f (Sec. 5.2) with OT_OPT_TRANSPORT,
                              else -1 */
  double ms_residual;      /* with OT_OPT_PHASE_TIMES (else -1): device ms in the residual
                              and coefficient evaluations (Eq. ma2, linearmaeq), */
  double ms_fft;           /* the preconditioned matvecs' transform passes (Sec. 4.2), */
  double ms_krylov;        /* the GMRES vector kernels (Arnoldi, Givens, restarts), */
  double ms_update;        /* theta = Lbar^{-1} sigma and the candidate u + s theta, */
  double ms_other;         /* and the rest (inputs, prefilter, warm start, control, gauge) */
} ot_stats;

/* Create a plan for N x M grids (N rows, M columns), damping tau >= 1 (Eq. linma) and
 * Newton tolerance tol > 0.  Allocates all device workspace (no allocation happens in
 * the solve calls).  *out receives the plan, or NULL on error. */
int ot_plan_create(ot_plan** out, int32_t N, int32_t M, double tau, double tol);

/* Set an OT_OPT_* option.  Changing OT_OPT_PRECISION or OT_OPT_RESTART reallocates the
 * workspace.  Returns OT_EINVAL for an unknown key or an out-of-range value. */
int ot_plan_set_option(ot_plan* plan, int32_t key, double value);

/* Read an OT_OPT_* option into *value.  OT_OPT_FFT_VARIANT reads the FP32 transform
 * kernels in use (the autotuner's choice after the first mixed solve) in the encoding that
 * ot_plan_set_option takes, or -1 while none is chosen.  OT_EINVAL for an unknown key. */
int ot_plan_get_option(ot_plan* plan, int32_t key, double* value);

/* Run the plan on a cudaStream_t (NULL = legacy default stream). */
int ot_plan_set_stream(ot_plan* plan, void* cuda_stream);

/* Solve (Sec. 3.1 damped Newton with the Fourier implementation of Sec. 4.2).
 * f, g: device N x M densities (read only).  phi_inout: device N x M, the mean-zero
 * potential on return (and u0 on entry if OT_OPT_WARM_START is set).  stats may be NULL. */
int ot_solve(ot_plan* plan, const double* f, const double* g, double* phi_inout,
             ot_stats* stats);

/* Same as ot_solve with HOST buffers (pageable or pinned): copies f, g (and phi when
 * warm-starting) to the plan's device buffers, solves, and copies phi back. */
int ot_solve_host(ot_plan* plan, const double* f, const double* g, double* phi_inout,
                  ot_stats* stats);

/* Solve `count` independent problems on existing plans, plans[k] sized for problem k (sizes
 * may differ; problems sharing a plan run one after the other on its stream, different plans
 * concurrently); f[k], g[k], phi[k] are device pointers for plans[k]; stats (array of count)
 * may be NULL.  Keeps a process-wide pinned result buffer, grown when a call has more
 * problems than any before.  Returns OT_OK if every problem converged, else the first
 * non-OK status. */
int ot_solve_plans(int32_t count, ot_plan* const* plans, const double* const* f,
                   const double* const* g, double* const* phi, ot_stats* stats);

/* ---- Plan sets: many problems of uneven sizes in one graph launch ------------------------
 * Not in the paper, which solves one image pair at a time: the damped Newton iteration of
 * Sec. 3.1 with the solver of Sec. 4.2 run for many independent pairs at once.  The pairs are
 * grouped by size; each size class runs every kernel of the mixed-precision solve for all its
 * pairs together (one launch serves the class, each pair's buffers in its own slab), with
 * per-pair state on the device: a pair leaves the Newton loop, a GMRES cycle or the step-
 * halving loop on its own test while the others go on, and each loop of the captured graph
 * runs while any pair of the class needs it.  The classes are parallel branches of one CUDA
 * graph, so a call is one graph launch (plus one more per OT_OPT_TAU_RETRY round).
 *
 * ot_plan_set_create: count problems, problem k of N[k] x M[k] (each size as for
 * ot_plan_create; at most 1024 problems of one size, else OT_EUNSUPPORTED), damping tau >= 1,
 * tolerance tol > 0.  Device memory is allocated at the first ot_solve_batched (and after an
 * OT_OPT_RESTART change): about 170 bytes per grid point of every problem plus the shared
 * tables.  The solve is always the mixed-precision one (OT_OPT_PRECISION = 1, THETA_FP64 = 2)
 * from u0 = 0. */
typedef struct ot_plan_set ot_plan_set;
int ot_plan_set_create(ot_plan_set** out, int32_t count, const int32_t* N, const int32_t* M,
                       double tau, double tol);
/* Options for every problem of the set: OT_OPT_TAU, TOL, ETA, RESTART, MAX_NEWTON,
 * MAX_RESTARTS, SAFEGUARD, TRANSLATE, SYMBOLS, FORCING, OPERATOR, REORTH as for a plan;
 * OT_OPT_TAU_RETRY: rounds in which the problems that lost convexity are solved again from
 * u0 = 0 with twice their last tau (the others sit the round out); OT_OPT_PRECISION accepts
 * only 1 and OT_OPT_THETA_FP64 only 2.  Any other key: OT_EINVAL. */
int ot_batch_set_option(ot_plan_set* set, int32_t key, double value);
int ot_batch_set_stream(ot_plan_set* set, void* cuda_stream);
/* Solve the set's problems: count, N, M must repeat the set's sizes (else OT_EINVAL); f[k],
 * g[k] (read) and phi[k] (written, mean zero) are device pointers to N[k] x M[k] planes owned
 * by the caller; stats (HOST array of count, may be NULL) receives each problem's statistics
 * (ms_total: the whole call; kernel_launches: the launches of the problem's size class).
 * Returns after the results are complete: OT_OK if every problem converged, else the first
 * non-OK status (the per-problem statuses are in stats). */
int ot_solve_batched(ot_plan_set* set, int32_t count, const int32_t* N, const int32_t* M,
                     const double* const* f, const double* const* g, double* const* phi,
                     ot_stats* stats);
void ot_plan_set_destroy(ot_plan_set* set);

void ot_plan_destroy(ot_plan* plan);
const char* ot_strerror(int status);

/* Description of the last failed CUDA call made by the library on this thread ("" if none):
 * the call site and the CUDA error name and text. */
const char* ot_last_error(void);

/* Profile accumulated since the last reset: for each of the first n classes (n <=
 * OT_PROF_CLASSES) the summed event time in ms and the number of timed launches (ms,
 * launches may be NULL); *total_launches (may be NULL) counts every kernel launched by the
 * plan, including the no-op launches of Arnoldi steps after GMRES converged (those are not
 * timed).  Times are recorded only while OT_OPT_PROFILE is 1. */
int ot_plan_get_profile(ot_plan* plan, double* ms, int64_t* launches, int32_t n,
                        int64_t* total_launches);
int ot_plan_reset_profile(ot_plan* plan);

/* Steady-state duration of one kernel class (OT_PROF_RESIDUAL .. OT_PROF_GMRES_UPDATE, or
 * OT_TIME_WS_NETWORK; the
 * multi-dot and the Arnoldi update are timed at step j = 4 of an open cycle, reset by a
 * one-thread kernel before each launch whose own time is subtracted): after a solve,
 * captures `reps` back-to-back launches of that kernel on the plan's own buffers
 * (overwriting workspace only: the residual, spectra, w, the basis, the candidate iterate
 * and the device scalars) into a CUDA graph and times one replay between two CUDA events on
 * the plan's stream; *ms receives the mean time per launch. */
int ot_plan_time_kernel(ot_plan* plan, int32_t kernel_class, int32_t reps, double* ms);

/* ---- Step-level entry points: one stage of a Newton step each, on device buffers ---- */

/* Coefficients c of the periodic cubic B-spline interpolant of g (sum over the 4 x 4 taps
 * of c times the B-spline weights reproduces g at the nodes), used to sample g at the
 * displaced points x + grad phi (Sec. 4).  Computed in FP64 as the exact periodic inverse of
 * the stencil (1, 4, 1)/6 along each axis, by first-order recursive filters (pole
 * sqrt(3) - 2); c and g are device N x M row-major; the plan's residual buffer is used as
 * scratch.  Returns OT_EINVAL for null pointers or an unready plan. */
int ot_prefilter(ot_plan* plan, const double* g, double* c);

/* Residual and linearised coefficients at the iterate u (Eq. ma2, linearmaeq,
 * translation), with c from ot_prefilter and f as given (no translation here):
 *   F = f - (f_n - mean f_n + 1),  f_n = G(x + grad u) det(I + D^2 u)
 *   coef (5 planes, N x M each): a11 = G (1+u_yy), a12 = -G u_xy, a22 = G (1+u_xx),
 *                                b1 = det dG/dx, b2 = det dG/dy
 * scal (HOST, 10 doubles): mean f_n, max|F|, sqrt(mean F^2), min det, non-finite count,
 * then the Simpson averages of a11, a12, a22, b1, b2 (Sec. 4.2).  F, coef may be NULL. */
int ot_eval_residual(ot_plan* plan, const double* f, const double* c, const double* u,
                     double* F, double* coef, double* scal);

/* w = L Lbar^{-1} sigma (Sec. 4.2): coef as from ot_eval_residual, abar (HOST, 5 doubles)
 * the averaged coefficients.  Runs in the plan's precision. */
int ot_apply_operator(ot_plan* plan, const double* coef, const double* abar,
                      const double* sigma, double* w);

/* theta = Lbar^{-1} sigma = sum_{k != 0} rho-bar(k) sigma-hat(k) e^{2 pi i k.x} (Sec. 4.2). */
int ot_apply_lbar_inverse(ot_plan* plan, const double* abar, const double* sigma,
                          double* theta);

/* Unnormalised 2-D real FFT of x (N x M) into the packed half spectrum spec: N x (M/2)
 * complex values stored as interleaved (re, im) doubles; entry (k2, k1) for 1 <= k1 < M/2
 * is X(k2, k1) = sum x(i,j) exp(-2 pi i (k1 j / M + k2 i / N)); column k1 = 0 holds
 * A(k2) + i B(k2) where A, B are the transforms of the real k1 = 0 and k1 = M/2 row
 * coefficients.  Runs in the plan's precision. */
int ot_fft_forward(ot_plan* plan, const double* x, double* spec);

/* Inverse of ot_fft_forward without the 1/(N M) factor (spec -> N M x). */
int ot_fft_inverse(ot_plan* plan, const double* spec, double* x);

/* Transport outputs (Sec. 5.2): *dist = d(f, g) = int |x - T(x)|^2 f dx = int |grad phi|^2 f dx
 * with T = x + grad phi, as the grid mean of |grad phi|^2 f (the periodic trapezoid rule) with
 * the 4th-order centred differences of F; and, when div_out is not NULL, div_out = phi_xx +
 * phi_yy, the divergence of the displacement T(x) - x (the map the paper plots).  f, phi,
 * div_out: device N x M row-major (f as given: pass the density the solve used, e.g. its
 * translated form when it was not of mean 1); dist: HOST.  Double-float arithmetic (unit
 * round-off 2^-48).  OT_EINVAL for null f, phi or dist or an unready plan. */
int ot_transport_outputs(ot_plan* plan, const double* f, const double* phi, double* dist,
                         double* div_out);

/* Finite-difference comparison path (Sec. 4.1), step level; both need OT_OPT_LINEAR_SOLVER
 * = 1 on the plan (else OT_EINVAL).  coef: device, the 5 coefficient planes of
 * ot_eval_residual (a11, a12, a22, b1, b2).
 * ot_fd_apply: y = A~ x (transpose = 0) or A~^T x (1), A the second-order centred-difference
 * discretisation of a11 d_xx + 2 a12 d_xy + a22 d_yy + b1 d_x + b2 d_y, A~ = A + 1 1^T; x, y:
 * device N x M.
 * ot_fd_bicg: theta (device, written) from A~ theta = h (device) by BiCG from 0, stopping at
 * ||r||_2 <= eta ||h||_2 or after max_iters iterations; iters, relres (HOST, may be NULL):
 * the iterations run and ||r|| / ||h||.  OT_OK when converged, OT_ENOCONV at the cap,
 * OT_EDIVERGED on a breakdown (a zero BiCG denominator).  Uses the plan's workspace. */
int ot_fd_apply(ot_plan* plan, const double* coef, const double* x, int32_t transpose,
                double* y);
int ot_fd_bicg(ot_plan* plan, const double* coef, const double* h, double eta,
               int32_t max_iters, double* theta, int32_t* iters, double* relres);

/* Spectral radius of the inverse of the discretised linearised operator at the iterate phi
 * (the stability measure of Sec. 5.1, about 0.03 in the paper's experiments), by the power
 * iteration the paper uses: b_(k+1) = A^{-1} b_k / ||A^{-1} b_k||_2 with A^{-1} b = Lbar^{-1}
 * sigma, sigma from GMRES(m) on L Lbar^{-1} sigma = b at the plan's eta, m and symbols (the
 * Fourier method of Sec. 4.2), L = D_phi M of Eq. (linearmaeq) for the densities f, g
 * (translated as by the solve when OT_OPT_TRANSLATE is set).  b0: device N x M start vector
 * (projected to mean zero: the operator acts on mean-zero potentials, Sec. 3.1); rho (HOST,
 * iters doubles) receives ||A^{-1} b_k||_2 for the unit vectors b_k, k = 0..iters-1, whose
 * last entries approximate the spectral radius.  Uses the plan's workspace (the plan's next
 * solve starts afresh).  OT_EINVAL for null pointers, iters < 1 or invalid densities. */
int ot_inverse_spectral_radius(ot_plan* plan, const double* f, const double* g,
                               const double* phi, const double* b0, int32_t iters,
                               double* rho);

/* ---- Learned warm start -----------------------------------------------------------------
 * Not in the paper, which starts Newton from u0 = 0 and needs only an admissible start,
 * det(I + D^2 u0) > 0 (Thm 3.2).  After the input translation (Eq. translation):
 *   h  = P(log f - log g), P the mean-zero inverse of the 4th-order stencil Laplacian
 *        D_xx + D_yy of Sec. 4 (the linearisation of log det(I + D^2 u) + log g(x + grad u)
 *        = log f about u = 0);
 *   X  = 16 features per grid point at h: [log f, log g, lg, r, hxx + hyy, hxx - hyy, 2 hxy,
 *        hxx hyy - hxy^2, 10 hx, 10 hy, 0.1 Gx / Gc, 0.1 Gy / Gc, (Gx hx + Gy hy) / Gc,
 *        (hxx - hyy)^2 + 4 hxy^2, r (hxx + hyy), 0], where G, Gx, Gy are the cubic B-spline
 *        interpolant of g and its gradient at T = x + grad h, Gc = max(G, 1e-3),
 *        lg = log Gc, r = log f - lg - log max(det(I + D^2 h), 1e-3);
 *   s  = MLP(X): 16 -> 128 -> 128 -> 128 -> 1, SiLU, per point, trained to predict
 *        s* = (D_xx + D_yy)(phi* - h) for converged potentials phi*;
 *   u0 = alpha (h + P(G s)), G the Gaussian low-pass exp(-((k1/(M/4))^2 + (k2/(N/4))^2)/2)
 *        on frequency (k1, k2), alpha the largest of 1, 1/2, 1/4, 1/8 with
 *        det(I + alpha D^2 u0) > 0 at every point, else 0.
 * Inference runs the three matrix products on the tensor cores (tcgen05, BF16 operands, FP32
 * accumulation); training runs in FP32.  Parameters are one FP32 vector of
 * ot_ws_param_count() values: W0[128,16], b0[128], W1[128,128], b1[128], W2[128,128],
 * b2[128], w3[128], b3 (weights row-major [out][in]). */
int64_t ot_ws_param_count(void);

/* Upload the network parameters (HOST array of `count` floats) to the plan and allow
 * OT_OPT_WARM_START = 2.  Allocates the warm-start workspace on first use (about 100 bytes
 * per grid point).  OT_EINVAL if count != ot_ws_param_count(). */
int ot_ws_set_weights(ot_plan* plan, const float* params_host, int64_t count);

/* Parameter file: 8 bytes "OTWS0001", an int64 count, then count little-endian floats.
 * ot_warmstart_load reads one into the plan (as ot_ws_set_weights); ot_ws_save_weights
 * writes one from a HOST array.  OT_EINVAL on a missing, short or mismatched file. */
int ot_warmstart_load(ot_plan* plan, const char* weights_path);
int ot_ws_save_weights(const char* weights_path, const float* params_host, int64_t count);

/* The warm start alone for densities f, g (translated as by the solve when
 * OT_OPT_TRANSLATE is set): phi0 receives u0; *alpha_out (HOST, may be NULL) the scale. */
int ot_ws_predict(ot_plan* plan, const double* f, const double* g, double* phi0,
                  double* alpha_out);

/* Training data of one pair: X (N*M x 16 floats) receives the features at h and, when
 * phi_star is not NULL, target (N*M floats) receives s* = (D_xx + D_yy)(phi_star - h).
 * f, g are translated as by the solve.  Needs no weights. */
int ot_ws_features(ot_plan* plan, const double* f, const double* g, const double* phi_star,
                   float* X, float* target);

/* out[r] = MLP(X[r, 0..15]) for r < rows with the plan's weights (the BF16 tensor-core
 * kernel of the solve).  OT_ETIMEOUT if the kernel reported a timeout. */
int ot_ws_mlp_forward(ot_plan* plan, const float* X, int64_t rows, float* out);

/* u = P(src) (the FD Poisson solve of h; src, u: N x M); lowpass != 0: u = P(G src). */
int ot_ws_poisson(ot_plan* plan, const double* src, int32_t lowpass, double* u);

/* Trainer: Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the mean squared error of the network
 * over minibatches of `batch` rows (a multiple of 64, 64..1048576), FP32 master parameters,
 * on its own stream (ot_ws_trainer_set_stream; default the legacy stream). */
typedef struct ot_ws_trainer ot_ws_trainer;
int ot_ws_trainer_create(ot_ws_trainer** out, int32_t batch, const float* params_host,
                         int64_t count);
int ot_ws_trainer_set_stream(ot_ws_trainer* tr, void* cuda_stream);
/* Gradient of the loss over the rows idx[0..batch) (device int64, each < the row count of
 * X and t) of X (rows x 16) and t (rows): grad_host (HOST, count floats, may be NULL) and
 * loss_host (HOST, may be NULL) receive it; the parameters do not change. */
int ot_ws_trainer_grad(ot_ws_trainer* tr, const float* X, const float* t, const int64_t* idx,
                       float* grad_host, double* loss_host);
/* One Adam step with learning rate lr on the rows idx[0..batch).  With loss_host NULL the
 * call only enqueues work and does not synchronise; otherwise it returns the step's loss
 * (before the update). */
int ot_ws_trainer_step(ot_ws_trainer* tr, const float* X, const float* t, const int64_t* idx,
                       float lr, double* loss_host);
int ot_ws_trainer_get_params(ot_ws_trainer* tr, float* params_host, int64_t count);
void ot_ws_trainer_destroy(ot_ws_trainer* tr);

/* ---- Allocation-free variant ------------------------------------------------------------
 * No counterpart in the paper: a library-level addition for callers that cannot allocate
 * device memory -- code whose device memory is all owned by its own pool (a framework's
 * caching allocator, a fixed-budget service) and latency-critical loops that cannot afford
 * cudaMalloc's implicit device-wide synchronisation.
 *
 * Same result as ot_eval_residual on an FP64 plan (F, the five coefficient planes as
 * doubles, scal as there), but needs no plan and calls no cudaMalloc, cudaFree or other
 * allocating routine: its scratch (reduction partials and a block of device scalars,
 * about 330 KB) is a fixed file-scope device array that every GPU loading the library holds
 * until the process exits.  f, c, u, F, coef: device pointers (coef: 5 planes of N x M);
 * scal: HOST, 10 doubles, may be NULL; cuda_stream: a cudaStream_t of the current device
 * (NULL = its legacy default stream); a stream of another device returns OT_EINVAL.
 * The call synchronises cuda_stream and returns after the results are complete, so it
 * cannot be called while that stream is being captured into a CUDA graph.
 *   - Sizes: 8 <= N, M <= 2048; larger grids return OT_EUNSUPPORTED before touching
 *     memory, smaller ones or a NULL pointer OT_EINVAL.
 *   - The first call on a device looks up the array's device address (set-up, once per
 *     device, with that device current).
 *   - All calls share the one array and clear what must start at zero themselves; calls
 *     that overlap on the GPU (other streams or host threads) race on it and must be
 *     serialised by the caller. */
int ot_eval_residual_noalloc(int32_t N, int32_t M, const double* f, const double* c,
                             const double* u, double* F, double* coef, double* scal,
                             void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
