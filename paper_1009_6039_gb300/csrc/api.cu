// C ABI of libotgb: plans, the damped-Newton driver (Sec. 3.1, Eq. linma) with Strain's
// FFT-preconditioned GMRES(m) (Sec. 4.2), and the step-level entry points.
#include <math.h>
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/otgb.h"
#include "otgb_internal.cuh"

using namespace otgb;

struct ot_plan {
  int N = 0, M = 0;
  double tau = 1.0, tol = 1e-8;
  int m = 10;
  double eta = 1e-4;
  int max_newton = 200, max_restarts = 50;
  int precision = 0, safeguard = 1, translate = 1, warm_start = 0;
  int reorth = 0;  // Gram-Schmidt passes - 1 (OT_OPT_REORTH)
  // mixed mode: precision of theta's inverse transforms and the update (OT_OPT_THETA_FP64):
  // 0 FP32, 1 FP64, 2 double-float (default)
  int theta64 = 2;
  int autotune = 1, tuned = 0;  // FP32 matvec kernel variants timed at the first solve
  cudaStream_t stream = 0;
  int device = 0;
  // FP64 planes
  double *f = nullptr, *g = nullptr, *c = nullptr, *u = nullptr, *ucand = nullptr,
         *Fraw = nullptr;
  // planes in the inner precision (FP64 or FP32)
  void *coef = nullptr, *V = nullptr, *w = nullptr, *sigma = nullptr;
  void *spec = nullptr, *q0 = nullptr, *q1 = nullptr, *q2 = nullptr;
  // FP64 spectrum used by the prefilter when the inner precision is FP32
  void *spec64 = nullptr, *q64 = nullptr;
  void *tw64 = nullptr, *tw32 = nullptr;  // twiddles: M/2 row (base + 3 stage tables), W_M, N column (base + 3)
  void* twdd = nullptr;                    // the same as (hi, lo) float pairs
  void* tw2 = nullptr;  // FP32 exchange twiddles of the register-resident matvec passes
  void *sym64 = nullptr, *sym32 = nullptr;  // derivative symbol tables (M/2 + 1 + N pairs)
  int symbols = 0;  // OT_OPT_SYMBOLS: 0 spectral (Sec. 4.2), 1 the stencils' symbols
  int forcing = 0;  // OT_OPT_FORCING: 0 fixed eta, 1 Eisenstat-Walker with eta as the cap
  int tau_retry = 0;  // OT_OPT_TAU_RETRY: re-solves with doubled tau after a divergence
  double tau_switch = 0.0;  // OT_OPT_TAU_SWITCH: tau schedule (tau -> 1 below this max|F|)
  // OT_OPT_INTERP: interpolation of g (0 cubic B-spline, 1 bilinear, 2 nearest node); the
  // latter two use the grid gradient of g (2 planes, FP64 and FP32)
  int interp = 0;
  double* gxy = nullptr;
  float* gxy32 = nullptr;
  // OT_OPT_LINEAR_SOLVER = 1: the finite-difference system of Sec. 4.1 with BiCG (FP64,
  // host-driven); its 7 vector planes and the iteration cap OT_OPT_MAX_BICG
  // OT_OPT_UNCOND_STEPS: Arnoldi steps per GMRES cycle captured as plain self-skipping
  // kernels rather than IF nodes (graph)
  int uncond = 7;
  int kbps = 2;  // OT_OPT_KRYLOV_BLOCKS: blocks per SM of the GMRES vector kernels
  int l2persist = 0;  // OT_OPT_L2_PERSIST: the Krylov basis as persisting L2 lines (graph)
  int fused_update = 1;  // OT_OPT_FUSED_UPDATE: Arnoldi update fused with the next row pass
  int theta_pairs = 1;   // OT_OPT_THETA_PAIRS: theta's double-float passes on pairs
  int linsolver = 0;
  int max_bicg = 20000;
  double* fdv = nullptr;
  int op_simple = 0;  // OT_OPT_OPERATOR: 1 drops the grad g term of the linearisation
  int ws_stall = 0;   // OT_OPT_WS_TEST_STALL: the next ot_ws_mlp_forward stalls (test hook)
  // mixed mode: f and the B-spline coefficients as (hi, lo) float pairs (double-float
  // residual; hi is also the FP32 copy used for the interpolant's gradient)
  float2 *fdd = nullptr, *cdd = nullptr;
  SpecTables tb64{}, tb32{}, tbdd{};
  double* partials = nullptr;
  double* dmean = nullptr;
  DevScalars* sc = nullptr;
  DevScalars* hsc = nullptr;    // pinned host mirror
  DevScalars* hinit = nullptr;  // pinned initial scalars of a batched solve (upload source)
  int kblocks = 0;
  bool ready = false;
  // kernel launch count and per-class event timing (OT_OPT_PROFILE)
  long long launches = 0;
  int profile = 0;
  struct Mark {
    int cls, tag;
    cudaEvent_t a, b;
  };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> pool;
  double prof_ms[OT_PROF_CLASSES] = {0};
  long long prof_n[OT_PROF_CLASSES] = {0};
  long long prof_skipped = 0;
  // graph-launched solve (OT_OPT_GRAPH): captured once per (precision, m, translate)
  int use_graph = 1;
  double* uout = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t cs[4] = {nullptr, nullptr, nullptr, nullptr};
  int gkey_prec = -1, gkey_m = -1, gkey_translate = -1;
  unsigned long long h_newton = 0, h_cycle = 0, h_restart = 0, h_halve = 0;
  unsigned long long h_step[OTGB_MAXM] = {0};
  int top_kernels = 0;
  double* gu_a = nullptr;  // iterate buffers as captured (upar = 0 names gu_a)
  double* gu_b = nullptr;
  // learned warm start (OT_OPT_WARM_START = 2)
  float* ws_params = nullptr;         // FP32 parameters
  unsigned char* ws_wpack = nullptr;  // BF16 weights in the tensor-core operand layout
  double *ws_src = nullptr, *ws_h = nullptr, *ws_tmp = nullptr;  // FP64 planes
  float *ws_X = nullptr, *ws_s = nullptr;  // features (P x 16), network output (P)
  float* ws_c32 = nullptr;                 // FP32 B-spline coefficients for the features
  int ws_have = 0, gkey_ws = -1, sms = 0;
  // OT_OPT_PHASE_TIMES: stamp kernels at phase changes while a solve is issued or captured
  int phase_times = 0, stamping = 0, last_phase = -1, phase_force = -1;
  int transport = 0;  // OT_OPT_TRANSPORT: d(f, g) of Sec. 5.2 at the end of each solve
  // batched plan (one size class of a plan set): `batch` pairs, each with all its per-pair
  // buffers in its own slab of `slab` bytes (the pointers above are pair 0's); cur_mask: the
  // pairs the launches being captured serve
  int batch = 1;
  size_t slab = 0;
  int cur_mask = MASK_ALL;
  void* slab_base = nullptr;
};

// batch descriptor of a plan's launches (a single problem: the plain launch)
static Bat btc(const ot_plan* p) {
  Bat b;
  b.on = p->slab_base ? 1 : 0;
  b.n = p->batch;
  b.slab = p->slab;
  b.mask = b.on ? p->cur_mask : MASK_ALL;
  return b;
}

template <typename T> static const SpecTables& tables(ot_plan* p);
template <> const SpecTables& tables<double>(ot_plan* p) { return p->tb64; }
template <> const SpecTables& tables<float>(ot_plan* p) { return p->tb32; }

// residual + coefficients of the iterate: FP64 kernel, or the double-float kernel in mixed
// mode (which reads the split copies of the plan's f and c)
template <typename T>
static cudaError_t residual_launch(ot_plan* p, const double* f, const double* c,
                                   const double* ua, double* Fraw, const double* ub = nullptr,
                                   int sel = 0) {
  const size_t P = (size_t)p->N * p->M;
  Interp ip;
  if (p->interp) {
    ip.mode = p->interp;
    ip.gx = p->gxy;
    ip.gy = p->gxy + P;
    ip.gx32 = p->gxy32;
    ip.gy32 = p->gxy32 + P;
  }
  if (sizeof(T) == 4)
    return launch_residual_dd(p->fdd, p->cdd, ua, p->N, p->M, Fraw, (float*)p->coef,
                              p->partials, p->sc, p->stream, ub, sel, p->op_simple, btc(p),
                              ip);
  return launch_residual<double>(f, c, ua, p->N, p->M, Fraw, (double*)p->coef, p->partials,
                                 p->sc, p->stream, ub, sel, nullptr, p->op_simple, ip);
}

static bool reorth_on(const ot_plan* p) { return p->reorth == 1; }

// whether this plan's Arnoldi steps run the update fused with the next product's row pass
// (FP32 single problem, the row pass in a form the fused kernel has, no reorthogonalisation,
// not the register-resident passes); the steps then leave out their own row pass, and each
// cycle starts with the row pass of v_0
template <typename T>
static bool fused_update_on(ot_plan* p) {
  if (sizeof(T) != 4 || !p->fused_update || p->slab_base || reorth_on(p)) return false;
  const SpecTables& tb = tables<T>(p);
  if (tb.mv_reg && tb.t2rA) return false;
  return update_r2c_fits(p->N, p->M, tb.var_r2c);
}


static cudaEvent_t ev_get(ot_plan* p) {
  if (!p->pool.empty()) {
    cudaEvent_t e = p->pool.back();
    p->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Accumulate the recorded marks (the stream has been synchronised).  Arnoldi-step marks
// carry their step index j; those with j >= jend ran as no-op launches of a finished cycle
// and are counted as skipped, not timed.
static void prof_harvest(ot_plan* p, int jend) {
  for (auto& mk : p->marks) {
    if (mk.tag >= 0 && mk.tag >= jend) {
      p->prof_skipped++;
    } else {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, mk.a, mk.b);
      p->prof_ms[mk.cls] += ms;
      p->prof_n[mk.cls] += 1;
    }
    p->pool.push_back(mk.a);
    p->pool.push_back(mk.b);
  }
  p->marks.clear();
}

// Launch wrapper: counts `nk` kernel launches; with profiling on, brackets them with events
// on the plan's stream.
#define RET(x)                  \
  do {                          \
    int r_ = (x);               \
    if (r_ != OT_OK) return r_; \
  } while (0)

#define LAUNCH(p, cls, tag, nk, expr)                                  \
  do {                                                                 \
    if ((p)->stamping) RET(stamp_phase(p, cls));                       \
    cudaEvent_t a_ = nullptr;                                          \
    if ((p)->profile) {                                                \
      a_ = ev_get(p);                                                  \
      cudaEventRecord(a_, (p)->stream);                                \
    }                                                                  \
    CK(expr);                                                          \
    (p)->launches += (nk);                                             \
    if ((p)->profile) {                                                \
      cudaEvent_t b_ = ev_get(p);                                      \
      cudaEventRecord(b_, (p)->stream);                                \
      (p)->marks.push_back({(cls), (tag), a_, b_});                     \
    }                                                                  \
  } while (0)

// Phase of a kernel class for OT_OPT_PHASE_TIMES (a forced phase overrides it: the theta
// passes are tagged with the transform classes but belong to the update)
static int phase_of(int cls) {
  switch (cls) {
    case OT_PROF_RESIDUAL: return PH_RESIDUAL;
    case OT_PROF_ROW_R2C:
    case OT_PROF_COL_MATVEC:
    case OT_PROF_ROW_C2R_COMBINE: return PH_FFT;
    case OT_PROF_COL_LBARINV:
    case OT_PROF_ROW_C2R_UPDATE: return PH_UPDATE;
    case OT_PROF_GMRES_DOTS:
    case OT_PROF_GMRES_UPDATE:
    case OT_PROF_GMRES_OTHER: return PH_KRYLOV;
  }
  return PH_OTHER;
}
static int stamp_phase(ot_plan* p, int cls);

static const char* kErr[] = {"ok", "invalid argument", "Newton did not converge",
                             "iterate lost convexity or became non-finite", "CUDA error",
                             "out of memory", "unsupported grid size",
                             "a bounded device-side wait gave up"};

extern "C" const char* ot_strerror(int s) {
  if (s <= 0 && s >= -7) return kErr[-s];
  return "unknown status";
}

// last CUDA failure seen by this thread (ot_last_error)
static thread_local char g_last_error[160] = "";
static void record_error(cudaError_t e, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "api.cu:%d: %s (%s)", line,
           cudaGetErrorName(e), cudaGetErrorString(e));
}
// a failure a kernel reported through its error flag (the CUDA context stays usable)
static void record_kernel_error(const char* what, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "api.cu:%d: %s", line, what);
}

extern "C" const char* ot_last_error(void) { return g_last_error; }

// The learned warm start's network kernel gave up a bounded wait during a solve: the
// admissibility step then chose the zero start and the solve went on from it.  The stats
// say so (ws_alpha = -2) and ot_last_error names it.
static void note_ws_timeout(ot_stats* st, int line) {
  st->ws_alpha = -2.0;
  record_kernel_error("learned warm start: the network kernel's bounded wait gave up; "
                      "solved from the zero start", line);
}

#define CK(x)                                 \
  do {                                        \
    cudaError_t e_ = (x);                     \
    if (e_ != cudaSuccess) {                  \
      record_error(e_, __LINE__);             \
      if (e_ == cudaErrorMemoryAllocation)    \
        return OT_ENOMEM;                     \
      return OT_ECUDA;                        \
    }                                         \
  } while (0)

// a stamp kernel before the first launch of a new phase (the host tracks the phase of the
// launch sequence it issues or captures; -1 = unknown, e.g. at a conditional body's start)
static int stamp_phase(ot_plan* p, int cls) {
  // OT_OPT_PHASE_TIMES = 2: a stamp at every change of kernel class (code 100 + class)
  const int ph = p->phase_times == 2 ? 100 + (cls < 0 ? OT_PROF_OTHER : cls)
                                     : (p->phase_force >= 0 ? p->phase_force : phase_of(cls));
  if (ph == p->last_phase) return OT_OK;
  CK(launch_stamp(p->sc, ph, p->stream));
  p->last_phase = ph;
  return OT_OK;
}


namespace otgb {
bool fft_length_supported(int L) {
  if (L < 8 || L > 2048) return false;
  int r = L;
  if (r % 3 == 0) {
    r /= 3;
    if (L < 12) return false;
  }
  return (r & (r - 1)) == 0;
}
}  // namespace otgb

static bool size_supported(int N, int M) {
  return N % 2 == 0 && M % 2 == 0 && M >= 16 && fft_length_supported(N) &&
         fft_length_supported(M / 2) && (M <= 2048);
}

static void free_events(ot_plan* p) {
  for (auto& mk : p->marks) {
    cudaEventDestroy(mk.a);
    cudaEventDestroy(mk.b);
  }
  p->marks.clear();
  for (auto e : p->pool) cudaEventDestroy(e);
  p->pool.clear();
}

static void free_graph(ot_plan* p) {
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->gexec = nullptr;
  p->graph = nullptr;
  p->gkey_prec = p->gkey_m = p->gkey_translate = -1;
}

static void free_buffers(ot_plan* p) {
  free_graph(p);
  if (p->slab_base) {
    // a batched plan's per-pair buffers live in its slabs: one allocation
    p->f = p->g = p->c = p->u = p->ucand = p->Fraw = p->uout = nullptr;
    p->coef = p->V = p->w = p->sigma = p->spec = p->q0 = p->q1 = p->q2 = p->q64 = nullptr;
    p->fdd = p->cdd = nullptr;
    p->partials = nullptr;
    p->sc = nullptr;
    cudaFree(p->slab_base);
    p->slab_base = nullptr;
    p->batch = 1;
    p->slab = 0;
  }
  if (p->uout) cudaFree(p->uout);
  p->uout = nullptr;
  void* ptrs[] = {p->fdd, p->cdd, p->f, p->g, p->c, p->u, p->ucand, p->Fraw, p->coef, p->V, p->w,
                  p->sigma, p->spec, p->q0, p->q1, p->q2, p->spec64, p->q64, p->tw64,
                  p->tw32, p->twdd, p->tw2, p->sym64, p->sym32, p->partials, p->dmean, p->sc, p->ws_src, p->ws_h, p->ws_tmp,
                  p->ws_X, p->ws_s, p->ws_c32};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  p->ws_src = p->ws_h = p->ws_tmp = nullptr;
  p->ws_X = p->ws_s = p->ws_c32 = nullptr;
  if (p->hsc) cudaFreeHost(p->hsc);
  if (p->hinit) cudaFreeHost(p->hinit);
  if (p->gxy) cudaFree(p->gxy);
  if (p->gxy32) cudaFree(p->gxy32);
  if (p->fdv) cudaFree(p->fdv);
  p->gxy = nullptr;
  p->gxy32 = nullptr;
  p->fdv = nullptr;
  p->hinit = nullptr;
  p->f = p->g = p->c = p->u = p->ucand = p->Fraw = nullptr;
  p->coef = p->V = p->w = p->sigma = p->spec = p->q0 = p->q1 = p->q2 = nullptr;
  p->spec64 = p->q64 = p->tw64 = p->tw32 = p->twdd = p->tw2 = nullptr;
  p->tb32.t2rA = p->tb32.t2rB = p->tb32.t2cA = p->tb32.t2cB = nullptr;
  p->sym64 = p->sym32 = nullptr;
  p->fdd = p->cdd = nullptr;
  p->partials = p->dmean = nullptr;
  p->sc = nullptr;
  p->hsc = nullptr;
  p->ready = false;
}

// exp(-2 pi i t / L) with exact reduction of the angle's numerator
static void roots(int L, int count, std::vector<double>& out) {
  for (int t = 0; t < count; ++t) {
    const double a = 2.0 * M_PI * (double)(t % L) / (double)L;
    out.push_back(std::cos(a));
    out.push_back(-std::sin(a));
  }
}

// Stage-ordered twiddles of the Stockham transform of length L with E elements per thread
// (the kernels' radix sequence: a radix-3 stage first for E = 12, then radix 8 while it
// divides for E = 8, else 4, else 2): stage (Ns, R) holds exp(-2 pi i k r / (Ns R)),
// r = 1..R-1, k = 0..Ns-1, at (Ns - 1) + (r - 1) Ns + k.  L entries; zero where the width
// does not apply to L (E = 12 needs the factor 3, E = 4 and 8 exclude it).
static void stage_roots(int L, int E, std::vector<double>& out) {
  std::vector<double> t(2 * (size_t)L, 0.0);
  if ((E == 12) == (L % 3 == 0)) {
    int Ns = 1, rem = L;
    auto stage = [&](int R) {
      for (int r = 1; r < R; ++r)
        for (int k = 0; k < Ns; ++k) {
          const double a = 2.0 * M_PI * (double)k * (double)r / ((double)Ns * (double)R);
          const size_t i = (size_t)(Ns - 1) + (size_t)(r - 1) * Ns + k;
          t[2 * i] = std::cos(a);
          t[2 * i + 1] = -std::sin(a);
        }
      Ns *= R;
      rem /= R;
    };
    if (E % 3 == 0) stage(3);
    while (rem > 1) {
      if (E % 8 == 0 && rem % 8 == 0)
        stage(8);
      else if (rem % 4 == 0)
        stage(4);
      else
        stage(2);
    }
  }
  out.insert(out.end(), t.begin(), t.end());
}

// a transform length's base table followed by its stage tables for E = 4, 8, 12 (the
// layout fft_smem expects)
static void transform_roots(int L, std::vector<double>& out) {
  roots(L, L, out);
  for (int E : {4, 8, 12}) stage_roots(L, E, out);
}

// (s1, s2) of frequency index k of length L (k <= L/2 for the half axis): spectral
// 2 pi k (0 at Nyquist) and -(2 pi k)^2 (Sec. 4.2, reading R4), or the Fourier symbols of the
// 4th-order stencils (8 sin t - sin 2t) L / 6 and (-2 cos 2t + 32 cos t - 30) L^2 / 12,
// t = 2 pi k / L (reading R1), which make L the exact linearisation of the discrete F.
static void deriv_symbols(int k, int L, int stencil, double* s1, double* s2) {
  const long ks = (2 * k <= L) ? k : (long)k - L;
  const bool nyq = 2 * k == L;
  if (stencil) {
    const double t = 2.0 * M_PI * (double)k / (double)L;
    *s1 = nyq ? 0.0 : (8.0 * std::sin(t) - std::sin(2.0 * t)) / 6.0 * (double)L;
    *s2 = (-2.0 * std::cos(2.0 * t) + 32.0 * std::cos(t) - 30.0) / 12.0 * (double)L * (double)L;
  } else {
    const double q = 2.0 * M_PI * (double)ks;
    *s1 = nyq ? 0.0 : q;
    *s2 = -q * q;
  }
}

static int fill_symbols(ot_plan* p) {
  const int nx = p->M / 2 + 1, n = nx + p->N;
  std::vector<double> d(2 * (size_t)n);
  for (int k = 0; k < nx; ++k) deriv_symbols(k, p->M, p->symbols, &d[2 * k], &d[2 * k + 1]);
  for (int k = 0; k < p->N; ++k)
    deriv_symbols(k, p->N, p->symbols, &d[2 * (nx + k)], &d[2 * (nx + k) + 1]);
  std::vector<float> f(d.begin(), d.end());
  if (!p->sym64) CK(cudaMalloc(&p->sym64, (size_t)n * 16));
  if (!p->sym32) CK(cudaMalloc(&p->sym32, (size_t)n * 8));
  CK(cudaMemcpy(p->sym64, d.data(), (size_t)n * 16, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p->sym32, f.data(), (size_t)n * 8, cudaMemcpyHostToDevice));
  p->tb64.symx = p->sym64;
  p->tb64.symy = (const double2*)p->sym64 + nx;
  p->tb32.symx = p->sym32;
  p->tb32.symy = (const float2*)p->sym32 + nx;
  return OT_OK;
}

// Exchange twiddles W_L^{t ka} = exp(-2 pi i t ka / L) (t < L/32, ka < 32) of the two-level
// register transforms, for the row length L = M/2 and the column length N, in the two layouts
// the kernels read contiguously: A at [ka * (L/32) + t], B at [t * 32 + ka].
static int fill_reg_twiddles(ot_plan* p) {
  const int Ls[2] = {p->M / 2, p->N};
  std::vector<float> h;
  for (int L : Ls) {
    const int T = L / 32;
    std::vector<float> A(2 * (size_t)L), B(2 * (size_t)L);
    for (int ka = 0; ka < 32; ++ka)
      for (int t = 0; t < T; ++t) {
        const long e = ((long)t * ka) % L;
        const double a = 2.0 * M_PI * (double)e / (double)L;
        const float c = (float)std::cos(a), sn = (float)-std::sin(a);
        A[2 * ((size_t)ka * T + t)] = c;
        A[2 * ((size_t)ka * T + t) + 1] = sn;
        B[2 * ((size_t)t * 32 + ka)] = c;
        B[2 * ((size_t)t * 32 + ka) + 1] = sn;
      }
    h.insert(h.end(), A.begin(), A.end());
    h.insert(h.end(), B.begin(), B.end());
  }
  CK(cudaMalloc(&p->tw2, h.size() * sizeof(float)));
  CK(cudaMemcpy(p->tw2, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
  const float2* b = (const float2*)p->tw2;
  const size_t Lr = p->M / 2;
  p->tb32.t2rA = b;
  p->tb32.t2rB = b + Lr;
  p->tb32.t2cA = b + 2 * Lr;
  p->tb32.t2cB = b + 2 * Lr + p->N;
  return OT_OK;
}

// Transform and symbol tables (shared by all problems of a plan), the device and its SM count.
static int alloc_tables(ot_plan* p) {
  const size_t L = p->M / 2;
  // twiddle tables
  // [row FFT length M/2 (4 L) | split W_M^k, k < M/2 (L) | column FFT length N (4 N)]
  std::vector<double> tw;
  transform_roots((int)L, tw);
  roots(p->M, (int)L, tw);
  transform_roots(p->N, tw);
  const size_t ntw = tw.size() / 2;
  CK(cudaMalloc(&p->tw64, ntw * 16));
  CK(cudaMemcpy(p->tw64, tw.data(), ntw * 16, cudaMemcpyHostToDevice));
  std::vector<float> twf(tw.begin(), tw.end());
  CK(cudaMalloc(&p->tw32, ntw * 8));
  CK(cudaMemcpy(p->tw32, twf.data(), ntw * 8, cudaMemcpyHostToDevice));
  std::vector<float> twd(tw.size() * 2);
  for (size_t k = 0; k < tw.size(); ++k) {
    const float h = (float)tw[k];
    twd[2 * k] = h;
    twd[2 * k + 1] = (float)(tw[k] - (double)h);
  }
  CK(cudaMalloc(&p->twdd, ntw * 16));
  CK(cudaMemcpy(p->twdd, twd.data(), ntw * 16, cudaMemcpyHostToDevice));
  p->tb32.theta_pair = p->tbdd.theta_pair = p->theta_pairs;
  p->tbdd.twL = p->twdd;
  p->tbdd.twM = (const ddc*)p->twdd + 4 * L;
  p->tbdd.twN = (const ddc*)p->twdd + 5 * L;
  RET(fill_symbols(p));
  if (p->precision && mvT_supported(p->N, p->M)) RET(fill_reg_twiddles(p));
  p->tb64.twL = p->tw64;
  p->tb64.twM = (const double2*)p->tw64 + 4 * L;
  p->tb64.twN = (const double2*)p->tw64 + 5 * L;
  p->tb32.twL = p->tw32;
  p->tb32.twM = (const float2*)p->tw32 + 4 * L;
  p->tb32.twN = (const float2*)p->tw32 + 5 * L;
  int sms = 0;
  CK(cudaGetDevice(&p->device));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
  // GMRES vector kernels: OT_OPT_KRYLOV_BLOCKS blocks of 256 threads per SM
  p->kblocks = (sms > 0 ? sms : 148) * p->kbps;
  p->sms = sms > 0 ? sms : 148;
  return OT_OK;
}

static int alloc_grad_planes(ot_plan* p);
static int alloc_fd_planes(ot_plan* p);
constexpr int kMaxKrylovBlocksPerSm = 8;

static int alloc_buffers(ot_plan* p) {
  free_buffers(p);
  const size_t P = (size_t)p->N * p->M;
  const size_t ts = p->precision ? sizeof(float) : sizeof(double);
  const size_t L = p->M / 2;
  CK(cudaMalloc(&p->f, P * 8));
  CK(cudaMalloc(&p->g, P * 8));
  CK(cudaMalloc(&p->c, P * 8));
  CK(cudaMalloc(&p->u, P * 8));
  CK(cudaMalloc(&p->ucand, P * 8));
  CK(cudaMalloc(&p->Fraw, P * 8));
  CK(cudaMalloc(&p->uout, P * 8));
  CK(cudaMalloc(&p->coef, 5 * P * ts));
  CK(cudaMalloc(&p->V, (size_t)(p->m + 1) * P * ts));
  CK(cudaMalloc(&p->w, P * ts));
  CK(cudaMalloc(&p->sigma, P * ts));
  // half spectra: N x M/2 complex = P elements of the inner type
  CK(cudaMalloc(&p->spec, P * ts));
  CK(cudaMalloc(&p->q0, P * ts));
  CK(cudaMalloc(&p->q1, P * ts));
  CK(cudaMalloc(&p->q2, P * ts));
  if (p->precision) {
    CK(cudaMalloc(&p->spec64, P * 8));
    CK(cudaMalloc(&p->q64, P * 8));
    CK(cudaMalloc(&p->fdd, P * 8));
    CK(cudaMalloc(&p->cdd, P * 8));
  } else {
    p->spec64 = nullptr;
    p->q64 = nullptr;
  }
  RET(alloc_tables(p));
  if (p->interp) RET(alloc_grad_planes(p));
  if (p->linsolver) RET(alloc_fd_planes(p));
  size_t np = (size_t)residual_partial_blocks(p->N, p->M) * 10;
  size_t nk = (size_t)p->sms * kMaxKrylovBlocksPerSm * OTGB_MAXM;  // any OT_OPT_KRYLOV_BLOCKS
  if (nk > np) np = nk;
  CK(cudaMalloc(&p->partials, np * 8));
  CK(cudaMalloc(&p->dmean, 8));
  CK(cudaMalloc(&p->sc, sizeof(DevScalars)));
  CK(cudaMemset(p->sc, 0, sizeof(DevScalars)));
  CK(cudaMallocHost(&p->hsc, sizeof(DevScalars)));
  memset(p->hsc, 0, sizeof(DevScalars));
  CK(cudaMallocHost(&p->hinit, sizeof(DevScalars)));
  memset(p->hinit, 0, sizeof(DevScalars));
  p->ready = true;
  return OT_OK;
}

// the BiCG vectors of the finite-difference path: x, r, r*, p, p*, q, q* (FP64 planes)
static int alloc_fd_planes(ot_plan* p) {
  const size_t P = (size_t)p->N * p->M;
  CK(cudaMalloc(&p->fdv, 7 * P * sizeof(double)));
  return OT_OK;
}
static FdBufs fdbufs(const ot_plan* p) {
  const size_t P = (size_t)p->N * p->M;
  double* b = p->fdv;
  return FdBufs{b, b + P, b + 2 * P, b + 3 * P, b + 4 * P, b + 5 * P, b + 6 * P};
}

// grid-gradient planes of g for the nearest / bilinear interpolation modes
static int alloc_grad_planes(ot_plan* p) {
  const size_t P = (size_t)p->N * p->M;
  CK(cudaMalloc(&p->gxy, 2 * P * sizeof(double)));
  CK(cudaMalloc(&p->gxy32, 2 * P * sizeof(float)));
  return OT_OK;
}

// A batched plan: B problems of this plan's size, mixed precision, every per-pair buffer in
// the pair's slab (equal layout, 256-byte aligned offsets), tables shared.
static int alloc_batch(ot_plan* p, int B) {
  free_buffers(p);
  if (!p->precision || B < 1 || B > 1024) return OT_EINVAL;
  const size_t P = (size_t)p->N * p->M;
  RET(alloc_tables(p));
  // GMRES vector kernels: blocks per pair by its size (the pairs fill the GPU together)
  long kb = (long)(P / 2048);
  p->kblocks = (int)std::min<long>(std::max<long>(kb, 8), p->sms);
  size_t np = (size_t)residual_partial_blocks(p->N, p->M) * 10;
  np = std::max(np, (size_t)p->kblocks * OTGB_MAXM);
  np = std::max(np, (size_t)2 * p->sms * 8);  // the 2-blocks-per-SM grid reductions
  struct Item {
    void** ptr;
    size_t bytes;
  };
  const Item items[] = {
      {(void**)&p->f, P * 8}, {(void**)&p->g, P * 8}, {(void**)&p->c, P * 8},
      {(void**)&p->u, P * 8}, {(void**)&p->ucand, P * 8}, {(void**)&p->Fraw, P * 8},
      {(void**)&p->uout, P * 8}, {&p->coef, 5 * P * 4}, {&p->V, (size_t)(p->m + 1) * P * 4},
      {&p->w, P * 4}, {&p->sigma, P * 4}, {&p->spec, P * 4}, {&p->q0, P * 4},
      {&p->q1, P * 4}, {&p->q2, P * 4}, {&p->q64, P * 8}, {(void**)&p->fdd, P * 8},
      {(void**)&p->cdd, P * 8}, {(void**)&p->partials, np * 8},
      {(void**)&p->sc, sizeof(DevScalars)}};
  size_t off[sizeof(items) / sizeof(items[0])];
  size_t slab = 0;
  for (size_t k = 0; k < sizeof(items) / sizeof(items[0]); ++k) {
    off[k] = slab;
    slab += (items[k].bytes + 255) / 256 * 256;
  }
  CK(cudaMalloc(&p->slab_base, slab * (size_t)B));
  for (size_t k = 0; k < sizeof(items) / sizeof(items[0]); ++k)
    *items[k].ptr = (char*)p->slab_base + off[k];
  p->batch = B;
  p->slab = slab;
  CK(cudaMemset2D(p->sc, slab, 0, sizeof(DevScalars), B));
  CK(cudaMalloc(&p->dmean, 8));
  CK(cudaMallocHost(&p->hsc, sizeof(DevScalars)));
  memset(p->hsc, 0, sizeof(DevScalars));
  CK(cudaMallocHost(&p->hinit, sizeof(DevScalars)));
  memset(p->hinit, 0, sizeof(DevScalars));
  p->ready = true;
  return OT_OK;
}

extern "C" int ot_plan_create(ot_plan** out, int32_t N, int32_t M, double tau, double tol) {
  if (!out) return OT_EINVAL;
  *out = nullptr;
  if (!(tau >= 1.0) || !(tol > 0.0)) return OT_EINVAL;
  if (!size_supported(N, M)) return OT_EUNSUPPORTED;
  ot_plan* p = new (std::nothrow) ot_plan();
  if (!p) return OT_ENOMEM;
  p->N = N;
  p->M = M;
  p->tau = tau;
  p->tol = tol;
  int rc = alloc_buffers(p);
  if (rc != OT_OK) {
    free_buffers(p);
    delete p;
    return rc;
  }
  *out = p;
  return OT_OK;
}

extern "C" void ot_plan_destroy(ot_plan* p) {
  if (!p) return;
  free_events(p);
  free_buffers(p);
  if (p->ws_params) cudaFree(p->ws_params);
  if (p->ws_wpack) cudaFree(p->ws_wpack);
  for (int k = 0; k < 4; ++k)
    if (p->cs[k]) cudaStreamDestroy(p->cs[k]);
  delete p;
}

extern "C" int ot_plan_set_stream(ot_plan* p, void* s) {
  if (!p) return OT_EINVAL;
  p->stream = (cudaStream_t)s;
  return OT_OK;
}

extern "C" int ot_plan_set_option(ot_plan* p, int32_t key, double v) {
  if (!p) return OT_EINVAL;
  switch (key) {
    case OT_OPT_RESTART: {
      int m = (int)v;
      if (m < 1 || m > OTGB_MAXM - 1 || m != v) return OT_EINVAL;
      if (m != p->m) {
        p->m = m;
        return alloc_buffers(p);
      }
      return OT_OK;
    }
    case OT_OPT_ETA:
      if (!(v > 0.0 && v < 1.0)) return OT_EINVAL;
      p->eta = v;
      return OT_OK;
    case OT_OPT_MAX_NEWTON:
      if (v < 0 || v != (int)v) return OT_EINVAL;
      p->max_newton = (int)v;
      return OT_OK;
    case OT_OPT_MAX_RESTARTS:
      if (v < 1 || v != (int)v) return OT_EINVAL;
      p->max_restarts = (int)v;
      return OT_OK;
    case OT_OPT_PRECISION: {
      if (v != 0 && v != 1) return OT_EINVAL;
      if (v != 0 && p->linsolver) return OT_EINVAL;  // the FD path is FP64
      if ((int)v != p->precision) {
        p->precision = (int)v;
        return alloc_buffers(p);
      }
      return OT_OK;
    }
    case OT_OPT_SAFEGUARD:
      if (v != 0 && v != 1) return OT_EINVAL;
      p->safeguard = (int)v;
      return OT_OK;
    case OT_OPT_TRANSLATE:
      if (v != 0 && v != 1) return OT_EINVAL;
      p->translate = (int)v;
      free_graph(p);
      return OT_OK;
    case OT_OPT_WARM_START:
      if (v != 0 && v != 1 && v != 2) return OT_EINVAL;
      if (v == 2 && (!p->ws_have || p->interp)) return OT_EINVAL;
      p->warm_start = (int)v;
      free_graph(p);
      return OT_OK;
    case OT_OPT_TAU:
      if (!(v >= 1.0)) return OT_EINVAL;
      p->tau = v;
      return OT_OK;
    case OT_OPT_TOL:
      if (!(v > 0.0)) return OT_EINVAL;
      p->tol = v;
      return OT_OK;
    case OT_OPT_PROFILE:
      if (v != 0 && v != 1) return OT_EINVAL;
      p->profile = (int)v;
      return OT_OK;
    case OT_OPT_GRAPH:
      if (v != 0 && v != 1) return OT_EINVAL;
      p->use_graph = (int)v;
      return OT_OK;
    case OT_OPT_REORTH:
      if (v != 0 && v != 1) return OT_EINVAL;
      p->reorth = (int)v;
      free_graph(p);
      return OT_OK;
    case OT_OPT_THETA_FP64:
      if (v != 0 && v != 1 && v != 2) return OT_EINVAL;
      p->theta64 = (int)v;
      free_graph(p);
      return OT_OK;
    case OT_OPT_FFT_VARIANT: {
      // r2c + 4 col + 16 combine, each 0 generic, 1 concurrent (r2c: same as 0), 2 warp,
      // 3 generic with 4 elements per thread
      // + 64: the generic column pass with 4 columns per block
      // + 128: the register-resident passes on the transposed spectrum for all three (where
      // the lengths allow them; the other bits then apply elsewhere)
      // + 256: the column pass on column pairs with packed FP32 arithmetic (where the sizes
      // allow it, else as col 3); + 512: the combine pass on row pairs (else as comb 3);
      // + 1024: the row R2C pass (and the fused update) on row pairs (else as r2c 3)
      if (v < 0 || v > 2047 || v != (double)(int)v) return OT_EINVAL;
      const int k = (int)v & 63;
      p->tb32.mv_reg = ((int)v & 128) ? 1 : 0;
      p->tb32.var_r2c = ((int)v & 1024) ? VAR_PAIR : (k % 4 == 1 ? VAR_GENERIC : k % 4);
      p->tb32.var_col = ((int)v & 256) ? VAR_PAIR : (k / 4) % 4;
      p->tb32.var_comb = ((int)v & 512) ? VAR_PAIR : k / 16;
      p->tb32.col_q = ((int)v & 64) ? 4 : 0;
      p->autotune = 0;
      p->tuned = 1;
      free_graph(p);
      return OT_OK;
    }
    case OT_OPT_WS_TEST_STALL:
      if (v != 0 && v != 1) return OT_EINVAL;
      p->ws_stall = (int)v;
      return OT_OK;
    case OT_OPT_OPERATOR:
      if (v != 0 && v != 1) return OT_EINVAL;
      if (p->op_simple != (int)v) {
        p->op_simple = (int)v;
        free_graph(p);
      }
      return OT_OK;
    case OT_OPT_TAU_RETRY:
      if (!(v >= 0 && v <= 8) || v != (double)(int)v) return OT_EINVAL;
      p->tau_retry = (int)v;
      return OT_OK;
    case OT_OPT_FORCING:
      if (v != 0 && v != 1) return OT_EINVAL;
      p->forcing = (int)v;
      free_graph(p);
      return OT_OK;
    case OT_OPT_SYMBOLS:
      if (v != 0 && v != 1) return OT_EINVAL;
      if (p->symbols != (int)v) {
        p->symbols = (int)v;
        if (p->ready) RET(fill_symbols(p));
      }
      return OT_OK;
    case OT_OPT_TAU_SWITCH:
      if (!(v >= 0.0)) return OT_EINVAL;
      p->tau_switch = v;
      return OT_OK;
    case OT_OPT_INTERP:
      if (v != 0 && v != 1 && v != 2) return OT_EINVAL;
      if (v != 0 && p->warm_start == 2) return OT_EINVAL;  // the features sample the B-spline
      if ((int)v != p->interp) {
        p->interp = (int)v;
        free_graph(p);
      }
      if (p->interp && p->ready && !p->gxy) RET(alloc_grad_planes(p));
      return OT_OK;
    case OT_OPT_LINEAR_SOLVER:
      if (v != 0 && v != 1) return OT_EINVAL;
      if (v != 0 && p->precision) return OT_EINVAL;
      p->linsolver = (int)v;
      if (p->linsolver && p->ready && !p->fdv) RET(alloc_fd_planes(p));
      return OT_OK;
    case OT_OPT_MAX_BICG:
      if (v < 1 || v > 1e9 || v != (double)(int)v) return OT_EINVAL;
      p->max_bicg = (int)v;
      return OT_OK;
    case OT_OPT_KRYLOV_BLOCKS:
      if (v < 1 || v > kMaxKrylovBlocksPerSm || v != (double)(int)v) return OT_EINVAL;
      if (p->kbps != (int)v) {
        p->kbps = (int)v;
        p->kblocks = p->sms * p->kbps;
        free_graph(p);
      }
      return OT_OK;
    case OT_OPT_L2_PERSIST:
      if (v != 0 && v != 1) return OT_EINVAL;
      if (p->l2persist != (int)v) {
        p->l2persist = (int)v;
        free_graph(p);
      }
      return OT_OK;
    case OT_OPT_FUSED_UPDATE:
      if (v != 0 && v != 1) return OT_EINVAL;
      if (p->fused_update != (int)v) {
        p->fused_update = (int)v;
        free_graph(p);
      }
      return OT_OK;
    case OT_OPT_THETA_PAIRS:
      if (v != 0 && v != 1) return OT_EINVAL;
      if (p->theta_pairs != (int)v) {
        p->theta_pairs = (int)v;
        p->tb32.theta_pair = p->tbdd.theta_pair = p->theta_pairs;
        free_graph(p);
      }
      return OT_OK;
    case OT_OPT_UNCOND_STEPS:
      if (v < 0 || v > OTGB_MAXM || v != (double)(int)v) return OT_EINVAL;
      if (p->uncond != (int)v) {
        p->uncond = (int)v;
        free_graph(p);
      }
      return OT_OK;
    case OT_OPT_PHASE_TIMES:
      if (v != 0 && v != 1 && v != 2) return OT_EINVAL;
      if (p->phase_times != (int)v) {
        p->phase_times = (int)v;
        free_graph(p);
      }
      return OT_OK;
    case OT_OPT_TRANSPORT:
      if (v != 0 && v != 1) return OT_EINVAL;
      if (p->transport != (int)v) {
        p->transport = (int)v;
        free_graph(p);
      }
      return OT_OK;
    case OT_OPT_AUTOTUNE:
      if (v != 0 && v != 1) return OT_EINVAL;
      p->autotune = (int)v;
      if (!p->autotune) {
        p->tb32.var_r2c = p->tb32.var_col = p->tb32.var_comb = VAR_DEFAULT;
        p->tb32.mv_reg = 0;
        p->tuned = 0;
      }
      free_graph(p);
      return OT_OK;
  }
  return OT_EINVAL;
}

extern "C" int ot_plan_get_option(ot_plan* p, int32_t key, double* v) {
  if (!p || !v) return OT_EINVAL;
  switch (key) {
    case OT_OPT_RESTART: *v = p->m; return OT_OK;
    case OT_OPT_ETA: *v = p->eta; return OT_OK;
    case OT_OPT_MAX_NEWTON: *v = p->max_newton; return OT_OK;
    case OT_OPT_MAX_RESTARTS: *v = p->max_restarts; return OT_OK;
    case OT_OPT_PRECISION: *v = p->precision; return OT_OK;
    case OT_OPT_SAFEGUARD: *v = p->safeguard; return OT_OK;
    case OT_OPT_TRANSLATE: *v = p->translate; return OT_OK;
    case OT_OPT_WARM_START: *v = p->warm_start; return OT_OK;
    case OT_OPT_TAU: *v = p->tau; return OT_OK;
    case OT_OPT_TOL: *v = p->tol; return OT_OK;
    case OT_OPT_PROFILE: *v = p->profile; return OT_OK;
    case OT_OPT_GRAPH: *v = p->use_graph; return OT_OK;
    case OT_OPT_REORTH: *v = p->reorth; return OT_OK;
    case OT_OPT_THETA_FP64: *v = p->theta64; return OT_OK;
    case OT_OPT_AUTOTUNE: *v = p->autotune; return OT_OK;
    case OT_OPT_SYMBOLS: *v = p->symbols; return OT_OK;
    case OT_OPT_FORCING: *v = p->forcing; return OT_OK;
    case OT_OPT_TAU_RETRY: *v = p->tau_retry; return OT_OK;
    case OT_OPT_WS_TEST_STALL: *v = p->ws_stall; return OT_OK;
    case OT_OPT_OPERATOR: *v = p->op_simple; return OT_OK;
    case OT_OPT_PHASE_TIMES: *v = p->phase_times; return OT_OK;
    case OT_OPT_TAU_SWITCH: *v = p->tau_switch; return OT_OK;
    case OT_OPT_INTERP: *v = p->interp; return OT_OK;
    case OT_OPT_LINEAR_SOLVER: *v = p->linsolver; return OT_OK;
    case OT_OPT_MAX_BICG: *v = p->max_bicg; return OT_OK;
    case OT_OPT_UNCOND_STEPS: *v = p->uncond; return OT_OK;
    case OT_OPT_KRYLOV_BLOCKS: *v = p->kbps; return OT_OK;
    case OT_OPT_L2_PERSIST: *v = p->l2persist; return OT_OK;
    case OT_OPT_FUSED_UPDATE: *v = p->fused_update; return OT_OK;
    case OT_OPT_THETA_PAIRS: *v = p->theta_pairs; return OT_OK;
    case OT_OPT_TRANSPORT: *v = p->transport; return OT_OK;
    case OT_OPT_FFT_VARIANT: {
      // the variants in use, in the encoding ot_plan_set_option takes; -1 before the
      // autotuner has run (or in FP64 mode, which has one variant)
      const SpecTables& tb = p->tb32;
      if (!p->precision || !p->tuned || tb.var_r2c < 0 || tb.var_col < 0 || tb.var_comb < 0) {
        *v = -1;
        return OT_OK;
      }
      *v = (tb.var_r2c == VAR_PAIR ? 1024 : tb.var_r2c) +
           4 * (tb.var_col == VAR_PAIR ? 0 : tb.var_col) +
           16 * (tb.var_comb == VAR_PAIR ? 0 : tb.var_comb) + (tb.col_q == 4 ? 64 : 0) +
           (tb.mv_reg && tb.t2rA ? 128 : 0) + (tb.var_col == VAR_PAIR ? 256 : 0) +
           (tb.var_comb == VAR_PAIR ? 512 : 0);
      return OT_OK;
    }
  }
  return OT_EINVAL;
}

extern "C" int ot_plan_get_profile(ot_plan* p, double* ms, int64_t* launches, int32_t n,
                                   int64_t* total_launches) {
  if (!p || n < 0) return OT_EINVAL;
  for (int k = 0; k < n && k < OT_PROF_CLASSES; ++k) {
    if (ms) ms[k] = p->prof_ms[k];
    if (launches) launches[k] = p->prof_n[k];
  }
  if (total_launches) *total_launches = p->launches;
  return OT_OK;
}

// Device time of `reps` back-to-back launches issued by one() on p->stream, captured and
// replayed as one CUDA graph (total in *ms).  Kernels launched one by one into a stream are
// paced on this system at multiples of about 2 us each, which rounds every short kernel up
// to that grid; inside a graph they follow each other a fraction of a microsecond apart, as
// in the captured solve.  p->stream is switched to the plan's capture stream while one()
// is recorded.
template <typename F>
static int graph_time(ot_plan* p, F&& one, int reps, float* ms) {
  if (!p->cs[0]) CK(cudaStreamCreateWithFlags(&p->cs[0], cudaStreamNonBlocking));
  cudaStream_t run = p->stream;
  cudaEvent_t a = nullptr, b = nullptr;
  CK(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
  CK(cudaEventRecord(a, run));
  CK(cudaStreamWaitEvent(p->cs[0], a, 0));
  cudaEventDestroy(a);
  a = nullptr;
  p->stream = p->cs[0];
  cudaError_t e = cudaStreamBeginCapture(p->cs[0], cudaStreamCaptureModeRelaxed);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = one();
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(p->cs[0], &g);
  p->stream = run;
  if (e == cudaSuccess) e = e2;
  cudaGraphExec_t ge = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e == cudaSuccess) e = cudaGraphLaunch(ge, run);  // upload and warm
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaEventRecord(a, run);
  if (e == cudaSuccess) e = cudaGraphLaunch(ge, run);
  if (e == cudaSuccess) e = cudaEventRecord(b, run);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  if (ge) cudaGraphExecDestroy(ge);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  CK(e);
  return OT_OK;
}

template <typename T>
static int time_kernel_impl(ot_plan* p, int cls, int reps, double* ms_per_launch) {
  const SpecTables& tb = tables<T>(p);
  const int N = p->N, M = p->M;
  const size_t P = (size_t)N * M;
  const bool reg = sizeof(T) == 4 && tb.mv_reg && tb.t2rA;
  const int jstep = p->m > 4 ? 4 : p->m - 1;
  // the relaunched kernels run outside the solve graph: no kernel may set its conditional
  // handles (the graph may have been destroyed since the solve that left them)
  CK(cudaMemsetAsync((char*)p->sc + offsetof(DevScalars, graph), 0, sizeof(int), p->stream));
  auto one = [&]() -> cudaError_t {
    if (cls == -1) return launch_set_step(p->sc, jstep, p->stream);
    if (reg && cls == OT_PROF_ROW_R2C)
      return launch_mvT_r2c((const float*)p->V, P, nullptr, nullptr, (float2*)p->spec, N, M, tb,
                            nullptr, p->stream);
    if (reg && cls == OT_PROF_COL_MATVEC)
      return launch_mvT_col((const float2*)p->spec, (float2*)p->q0, (float2*)p->q1,
                            (float2*)p->q2, N, M, tb, p->sc, nullptr, p->stream);
    if (reg && cls == OT_PROF_ROW_C2R_COMBINE)
      return launch_mvT_combine((const float2*)p->q0, (const float2*)p->q1,
                                (const float2*)p->q2, (const float*)p->coef, (float*)p->w, N, M,
                                tb, nullptr, p->stream);
    switch (cls) {
      case OT_PROF_RESIDUAL:
        return residual_launch<T>(p, p->f, p->c, p->u, p->Fraw, nullptr, 0);
      case OT_PROF_ROW_R2C:
        return launch_row_r2c<T>((const T*)p->V, P, nullptr, nullptr, (C2<T>*)p->spec, N, M,
                                 tb, nullptr, p->stream);
      case OT_PROF_COL_MATVEC:
        return launch_col<T>(COL_MATVEC, (C2<T>*)p->spec, (C2<T>*)p->q0, (C2<T>*)p->q1,
                             (C2<T>*)p->q2, N, M, tb, p->sc, nullptr, p->stream);
      case OT_PROF_ROW_C2R_COMBINE:
        return launch_row_c2r<T>(ROWINV_COMBINE, (C2<T>*)p->q0, (C2<T>*)p->q1, (C2<T>*)p->q2,
                                 (const T*)p->coef, (T*)p->w, nullptr, nullptr, 0.0, 1.0, N, M,
                                 tb, nullptr, p->stream);
      case OT_PROF_COL_LBARINV:
        if (sizeof(T) == 4 && p->theta64 == 2)
          return launch_col_lbarinv_dd((const float2*)p->spec, (ddc*)p->q64, N, M, p->tb32,
                                       p->tbdd, p->sc, p->stream);
        if (sizeof(T) == 4 && p->theta64)  // FP32 forward / FP64 inverse in this mode
          return launch_col_lbarinv_mixed((const float2*)p->spec, (double2*)p->q64, N, M,
                                          p->tb32, p->tb64, p->sc, p->stream);
        return launch_col<T>(COL_LBARINV, (C2<T>*)p->spec, (C2<T>*)p->q0, nullptr, nullptr, N,
                             M, tb, p->sc, nullptr, p->stream);
      case OT_PROF_ROW_C2R_UPDATE:
        if (sizeof(T) == 4 && p->theta64 == 2)
          return launch_row_c2r_update_dd((const ddc*)p->q64, p->u, p->ucand, 0.5, N, M,
                                          p->tbdd, nullptr, p->stream);
        if (sizeof(T) == 4 && p->theta64)
          return launch_row_c2r<double>(ROWINV_UPDATE, (C2<double>*)p->q64, nullptr, nullptr,
                                        nullptr, nullptr, p->u, p->ucand, 0.5, 1.0, N, M,
                                        p->tb64, nullptr, p->stream);
        return launch_row_c2r<T>(ROWINV_UPDATE, (C2<T>*)p->q0, nullptr, nullptr, nullptr,
                                 nullptr, p->u, p->ucand, 0.5, 1.0, N, M, tb, nullptr,
                                 p->stream);
      case OT_TIME_WS_NETWORK:
        return launch_ws_mlp(p->ws_wpack, p->ws_params, p->ws_X, (long)P, p->ws_s,
                             &p->sc->ws_err, p->sms, p->stream, 0);
      case OT_PROF_GMRES_DOTS:
      case OT_PROF_GMRES_UPDATE: {
        // a representative Arnoldi step: j = 4 (five basis vectors), the cycle put back open
        // before every launch (the step's close moves j on and may end the cycle); the
        // one-thread reset is timed alone and subtracted below
        cudaError_t e = launch_set_step(p->sc, jstep, p->stream);
        if (e != cudaSuccess) return e;
        if (cls == OT_PROF_GMRES_DOTS)
          return launch_gmres_dots<T>((const T*)p->V, (const T*)p->w, (long)P, p->partials,
                                      p->sc, p->kblocks, p->stream);
        if (fused_update_on<T>(p))  // the update as the solve runs it: with the row pass
          return launch_gmres_update_r2c((float*)p->V, (const float*)p->w, (long)P,
                                         p->partials, p->kblocks, p->sc, (float2*)p->spec, N,
                                         M, p->tb32, p->stream);
        return launch_gmres_update<T>((T*)p->V, (const T*)p->w, (long)P, p->partials, p->sc,
                                      p->kblocks, p->stream, 3);
      }
    }
    return cudaErrorInvalidValue;
  };
  CK(one());  // warm
  float ms = 0.f;
  RET(graph_time(p, one, reps, &ms));
  if (cls == OT_PROF_GMRES_DOTS || cls == OT_PROF_GMRES_UPDATE) {
    float ms0 = 0.f;
    const int keep = cls;
    cls = -1;  // the reset alone
    RET(graph_time(p, one, reps, &ms0));
    cls = keep;
    ms -= ms0;
  }
  *ms_per_launch = ms / reps;
  return OT_OK;
}

extern "C" int ot_plan_time_kernel(ot_plan* p, int32_t cls, int32_t reps, double* ms) {
  if (!p || !ms || reps < 1) return OT_EINVAL;
  if (cls == OT_TIME_WS_NETWORK) {
    if (!p->ws_have || !p->ws_X || !p->ws_s) return OT_EINVAL;
  } else if (cls < 0 || cls > OT_PROF_GMRES_UPDATE) {
    return OT_EINVAL;
  }
  CK(cudaSetDevice(p->device));
  return p->precision ? time_kernel_impl<float>(p, cls, reps, ms)
                      : time_kernel_impl<double>(p, cls, reps, ms);
}

extern "C" int ot_plan_reset_profile(ot_plan* p) {
  if (!p) return OT_EINVAL;
  for (int k = 0; k < OT_PROF_CLASSES; ++k) {
    p->prof_ms[k] = 0.0;
    p->prof_n[k] = 0;
  }
  p->prof_skipped = 0;
  p->launches = 0;
  return OT_OK;
}

// ------------------------------------------------------------------------------------------
// pipelines
// ------------------------------------------------------------------------------------------

static int read_scalars(ot_plan* p) {
  CK(cudaMemcpyAsync(p->hsc, p->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  if (p->profile) prof_harvest(p, p->hsc->jend);
  return OT_OK;
}


// c = B-spline coefficients of g in FP64 (recursive filters along y and x; p->Fraw is free
// scratch before the first residual); the mixed mode also keeps c and f as (hi, lo) floats
static int run_prefilter(ot_plan* p, const double* g, double* c) {
  if (p->interp) {
    // nearest / bilinear: the grid values themselves and their gradient
    const long P = (long)p->N * p->M;
    if (c != g) CK(cudaMemcpyAsync(c, g, P * 8, cudaMemcpyDeviceToDevice, p->stream));
    LAUNCH(p, OT_PROF_OTHER, -1, 1,
           launch_grad4(g, p->N, p->M, p->gxy, p->gxy + P, p->gxy32, p->gxy32 + P, p->stream));
    if (p->precision) {
      LAUNCH(p, OT_PROF_OTHER, -1, 1, launch_split_dd(c, p->cdd, P, p->stream));
      LAUNCH(p, OT_PROF_OTHER, -1, 1, launch_split_dd(p->f, p->fdd, P, p->stream));
    }
    return OT_OK;
  }
  LAUNCH(p, OT_PROF_OTHER, -1, 2,
         launch_prefilter(g, p->Fraw, c, p->precision ? p->cdd : nullptr, p->N, p->M,
                          p->stream, btc(p)));
  if (p->precision)
    LAUNCH(p, OT_PROF_OTHER, -1, 1,
           launch_split_dd(p->f, p->fdd, (long)p->N * p->M, p->stream, btc(p)));
  return OT_OK;
}

// w = L Lbar^{-1} x, x = V + (*jptr) P scaled by scale[*jptr] when jptr is given
template <typename T>
static int run_matvec(ot_plan* p, const T* x, const int* jptr, const double* scale, T* w,
                      const int* skip, int tag, bool rows_done = false) {
  const size_t P = (size_t)p->N * p->M;
  const SpecTables& tb = tables<T>(p);
  const DevScalars* msc = p->slab_base ? p->sc : nullptr;
  if (sizeof(T) == 4 && tb.mv_reg && tb.t2rA && !p->slab_base) {
    // register-resident passes on the transposed half spectrum
    LAUNCH(p, OT_PROF_ROW_R2C, tag, 1,
           launch_mvT_r2c((const float*)x, P, jptr, scale, (float2*)p->spec, p->N, p->M, tb,
                          skip, p->stream));
    LAUNCH(p, OT_PROF_COL_MATVEC, tag, 1,
           launch_mvT_col((const float2*)p->spec, (float2*)p->q0, (float2*)p->q1,
                          (float2*)p->q2, p->N, p->M, tb, p->sc, skip, p->stream));
    LAUNCH(p, OT_PROF_ROW_C2R_COMBINE, tag, 1,
           launch_mvT_combine((const float2*)p->q0, (const float2*)p->q1,
                              (const float2*)p->q2, (const float*)p->coef, (float*)w, p->N,
                              p->M, tb, skip, p->stream));
    return OT_OK;
  }
  if (!rows_done)  // else the fused update of the previous step left the row pass's spectrum
    LAUNCH(p, OT_PROF_ROW_R2C, tag, 1,
           launch_row_r2c<T>(x, P, jptr, scale, (C2<T>*)p->spec, p->N, p->M, tb, skip,
                             p->stream, btc(p), msc));
  LAUNCH(p, OT_PROF_COL_MATVEC, tag, 1,
         launch_col<T>(COL_MATVEC, (C2<T>*)p->spec, (C2<T>*)p->q0, (C2<T>*)p->q1,
                       (C2<T>*)p->q2, p->N, p->M, tb, p->sc, skip, p->stream, btc(p)));
  LAUNCH(p, OT_PROF_ROW_C2R_COMBINE, tag, 1,
         launch_row_c2r<T>(ROWINV_COMBINE, (C2<T>*)p->q0, (C2<T>*)p->q1, (C2<T>*)p->q2,
                           (const T*)p->coef, w, nullptr, nullptr, 0.0, 1.0, p->N, p->M, tb,
                           skip, p->stream, msc, btc(p)));
  return OT_OK;
}

// u_out = u_in + step * Lbar^{-1} sigma  (UPDATE) or out = Lbar^{-1} sigma (PLAIN)
template <typename T>
static int run_lbar_inv(ot_plan* p, const T* sigma, const double* u_in, double* u_out,
                        double step, T* out) {
  const SpecTables& tb = tables<T>(p);
  LAUNCH(p, OT_PROF_ROW_R2C, -1, 1,
         launch_row_r2c<T>(sigma, 0, nullptr, nullptr, (C2<T>*)p->spec, p->N, p->M, tb,
                           nullptr, p->stream));
  LAUNCH(p, OT_PROF_COL_LBARINV, -1, 1,
         launch_col<T>(COL_LBARINV, (C2<T>*)p->spec, (C2<T>*)p->q0, nullptr, nullptr, p->N,
                       p->M, tb, p->sc, nullptr, p->stream));
  if (out) {
    LAUNCH(p, OT_PROF_ROW_C2R_UPDATE, -1, 1,
           launch_row_c2r<T>(ROWINV_PLAIN, (C2<T>*)p->q0, nullptr, nullptr, nullptr, out,
                             nullptr, nullptr, 0.0, 1.0, p->N, p->M, tb, nullptr, p->stream));
  } else {
    LAUNCH(p, OT_PROF_ROW_C2R_UPDATE, -1, 1,
           launch_row_c2r<T>(ROWINV_UPDATE, (C2<T>*)p->q0, nullptr, nullptr, nullptr, nullptr,
                             u_in, u_out, step, 1.0, p->N, p->M, tb, nullptr, p->stream));
  }
  return OT_OK;
}

// Newton update candidate u_out = u_in + s Lbar^{-1} sigma.  sc_driven: s and the buffer
// pair come from the device scalars (graph); otherwise the host passes them.  In the mixed
// mode the inverse transforms of theta run in double-float (theta64 = 2) or FP64 (1): theta
// is added to the FP64 iterate, and FP32 round-off in theta is white noise that the
// fourth-order stencils amplify by ~M^2 at the grid scale, where the Newton iteration damps
// it only slowly.  The forward transform of sigma and rho-bar stay FP32 (their round-off is
// damped by rho-bar ~ 1/k^2).
template <typename T>
static int run_theta_impl(ot_plan* p, const double* u_in, double* u_out, double step,
                          bool sc_driven);
template <typename T>
static int run_theta(ot_plan* p, const double* u_in, double* u_out, double step,
                     bool sc_driven) {
  p->phase_force = PH_UPDATE;
  const int rc = run_theta_impl<T>(p, u_in, u_out, step, sc_driven);
  p->phase_force = -1;
  return rc;
}
template <typename T>
static int run_theta_impl(ot_plan* p, const double* u_in, double* u_out, double step,
                          bool sc_driven) {
  const DevScalars* scp = sc_driven ? p->sc : nullptr;
  if (sizeof(T) == 4 && p->theta64 == 2) {
    LAUNCH(p, OT_PROF_ROW_R2C, -1, 1,
           launch_row_r2c<float>((const float*)p->sigma, 0, nullptr, nullptr,
                                 (C2<float>*)p->spec, p->N, p->M, p->tb32, nullptr,
                                 p->stream, btc(p), p->slab_base ? p->sc : nullptr));
    LAUNCH(p, OT_PROF_COL_LBARINV, -1, 1,
           launch_col_lbarinv_dd((const float2*)p->spec, (ddc*)p->q64, p->N, p->M, p->tb32,
                                 p->tbdd, p->sc, p->stream, COL_LBARINV, btc(p)));
    LAUNCH(p, OT_PROF_ROW_C2R_UPDATE, -1, 1,
           launch_row_c2r_update_dd((const ddc*)p->q64, u_in, u_out, step, p->N, p->M,
                                    p->tbdd, scp, p->stream, btc(p)));
    return OT_OK;
  }
  if (sizeof(T) == 4 && p->theta64) {
    C2<double>* qq = (C2<double>*)p->q64;
    LAUNCH(p, OT_PROF_ROW_R2C, -1, 1,
           launch_row_r2c<float>((const float*)p->sigma, 0, nullptr, nullptr,
                                 (C2<float>*)p->spec, p->N, p->M, p->tb32, nullptr,
                                 p->stream));
    LAUNCH(p, OT_PROF_COL_LBARINV, -1, 1,
           launch_col_lbarinv_mixed((const float2*)p->spec, (double2*)qq, p->N, p->M,
                                    p->tb32, p->tb64, p->sc, p->stream));
    LAUNCH(p, OT_PROF_ROW_C2R_UPDATE, -1, 1,
           launch_row_c2r<double>(ROWINV_UPDATE, qq, nullptr, nullptr, nullptr, nullptr, u_in,
                                  u_out, step, 1.0, p->N, p->M, p->tb64, nullptr, p->stream,
                                  scp));
    return OT_OK;
  }
  const SpecTables& tb = tables<T>(p);
  LAUNCH(p, OT_PROF_ROW_R2C, -1, 1,
         launch_row_r2c<T>((const T*)p->sigma, 0, nullptr, nullptr, (C2<T>*)p->spec, p->N,
                           p->M, tb, nullptr, p->stream));
  LAUNCH(p, OT_PROF_COL_LBARINV, -1, 1,
         launch_col<T>(COL_LBARINV, (C2<T>*)p->spec, (C2<T>*)p->q0, nullptr, nullptr, p->N,
                       p->M, tb, p->sc, nullptr, p->stream));
  LAUNCH(p, OT_PROF_ROW_C2R_UPDATE, -1, 1,
         launch_row_c2r<T>(ROWINV_UPDATE, (C2<T>*)p->q0, nullptr, nullptr, nullptr, nullptr,
                           u_in, u_out, step, 1.0, p->N, p->M, tb, nullptr, p->stream, scp));
  return OT_OK;
}

// One Arnoldi step j on the device: w = A v_j, Gram-Schmidt against V_0..V_j (classical,
// once or twice), norm, Givens rotation (in the last block of the final update).
template <typename T>
static int run_arnoldi_step(ot_plan* p, int j, const int* skip) {
  const long P = (long)p->N * p->M;
  T* V = (T*)p->V;
  T* w = (T*)p->w;
  const bool fused = fused_update_on<T>(p);
  RET(run_matvec<T>(p, V, &p->sc->j, p->sc->scale, w, skip, j, fused));
  LAUNCH(p, OT_PROF_GMRES_DOTS, j, 1,
         launch_gmres_dots<T>(V, w, P, p->partials, p->sc, p->kblocks, p->stream, 0, btc(p)));
  if (reorth_on(p)) {
    LAUNCH(p, OT_PROF_GMRES_UPDATE, j, 1,
           launch_gmres_update<T>(V, w, P, p->partials, p->sc, p->kblocks, p->stream, 1,
                                  btc(p)));
    LAUNCH(p, OT_PROF_GMRES_DOTS, j, 1,
           launch_gmres_dots<T>(V, w, P, p->partials, p->sc, p->kblocks, p->stream, 1,
                                btc(p)));
    LAUNCH(p, OT_PROF_GMRES_UPDATE, j, 1,
           launch_gmres_update<T>(V, w, P, p->partials, p->sc, p->kblocks, p->stream, 2,
                                  btc(p)));
  } else if (fused) {
    // the update's block 0 closes the step; its other blocks form v_(j+1) row by row and
    // run the next product's row pass on it
    LAUNCH(p, OT_PROF_GMRES_UPDATE, j, 1,
           launch_gmres_update_r2c((float*)V, (const float*)w, P, p->partials, p->kblocks,
                                   p->sc, (float2*)p->spec, p->N, p->M, p->tb32, p->stream));
  } else {
    // the multi-dot closes the step (norm by Pythagoras, Givens); the update only forms
    // v_(j+1) and is skipped when the cycle ends
    LAUNCH(p, OT_PROF_GMRES_UPDATE, j, 1,
           launch_gmres_update<T>(V, w, P, p->partials, p->sc, p->kblocks, p->stream, 3,
                                  btc(p)));
  }
  return OT_OK;
}

// the row pass of a cycle's v_0 where the steps run the fused update (which leaves the row
// pass of every later basis vector)
template <typename T>
static int run_cycle_rows(ot_plan* p, const int* skip) {
  if (!fused_update_on<T>(p)) return OT_OK;
  LAUNCH(p, OT_PROF_ROW_R2C, 0, 1,
         launch_row_r2c<T>((const T*)p->V, (size_t)p->N * p->M, &p->sc->j, p->sc->scale,
                           (C2<T>*)p->spec, p->N, p->M, tables<T>(p), skip, p->stream, btc(p),
                           nullptr));
  return OT_OK;
}

// GMRES(m) on L Lbar^{-1} sigma = (f - f~_n)/tau, sigma from 0.  Host syncs once per cycle.
template <typename T>
static int run_gmres(ot_plan* p) {
  const long P = (long)p->N * p->M;
  T* V = (T*)p->V;
  T* w = (T*)p->w;
  T* sigma = (T*)p->sigma;
  const int* skip = &p->sc->cycle_done;
  CK(cudaMemsetAsync(sigma, 0, P * sizeof(T), p->stream));
  if (p->forcing) LAUNCH(p, OT_PROF_OTHER, -1, 1, launch_ctl(CTL_FORCING, p->sc, p->stream, 1));
  LAUNCH(p, OT_PROF_GMRES_OTHER, -1, 1,
         launch_gmres_init<T>(p->Fraw, w, V, P, 0, p->partials, p->sc, p->kblocks, p->stream));
  for (int cyc = 0; cyc < p->max_restarts; ++cyc) {
    RET(run_cycle_rows<T>(p, skip));
    for (int j = 0; j < p->m; ++j) RET(run_arnoldi_step<T>(p, j, skip));
    LAUNCH(p, OT_PROF_GMRES_OTHER, -1, 1, launch_gmres_finish(p->sc, p->stream));
    LAUNCH(p, OT_PROF_GMRES_OTHER, -1, 1,
           launch_gmres_combine<T>(V, sigma, P, p->sc, p->kblocks, p->stream));
    RET(read_scalars(p));
    if (p->hsc->converged || cyc + 1 == p->max_restarts) break;
    // explicit residual for the restart: V0 = h - A sigma
    RET(run_matvec<T>(p, sigma, nullptr, nullptr, w, nullptr, -1));
    LAUNCH(p, OT_PROF_GMRES_OTHER, -1, 1,
           launch_gmres_init<T>(p->Fraw, w, V, P, 1, p->partials, p->sc, p->kblocks,
                                p->stream));
  }
  return OT_OK;
}

static void set_solver_scalars(ot_plan* p) {
  memset(p->hsc, 0, sizeof(DevScalars));
  p->hsc->m = p->m;
  p->hsc->eta = p->eta;
  p->hsc->tau = p->tau;
  p->hsc->tol = p->tol;
  p->hsc->step_s = 1.0;
  p->hsc->safeguard = p->safeguard;
  p->hsc->reorth = reorth_on(p) ? 1 : 0;
  p->hsc->step_kernels =
      reorth_on(p) ? 7 : ((p->precision && fused_update_on<float>(p)) ? 4 : 5);
  p->hsc->max_newton = p->max_newton;
  p->hsc->max_restarts = p->max_restarts;
  p->hsc->ws_alpha = -1.0;
  p->hsc->eta_max = p->eta;
  p->hsc->res_prev = 0.0;
  p->hsc->forcing = p->forcing;
  p->hsc->stamp_cls = -1;
  p->hsc->tau_switch = p->tau_switch;
  p->hsc->in_plain = p->translate ? 0 : 1;
}

// the stats fields every solve path fills from the final device scalars
static void fill_common_stats(ot_plan* p, const DevScalars* h, ot_stats* st) {
  st->mass_defect_f = h->in_mean[0] - 1.0;
  st->mass_defect_g = h->in_mean[1] - 1.0;
  st->transport_dist = p->transport ? h->dist : -1.0;
  double* ms[PH_COUNT] = {&st->ms_residual, &st->ms_fft, &st->ms_krylov, &st->ms_update,
                          &st->ms_other};
  for (int k = 0; k < PH_COUNT; ++k) *ms[k] = p->phase_times ? 1e-6 * (double)h->phase_ns[k] : -1.0;
  if (p->phase_times == 2) {
    // per kernel class: the phases are the sums of their classes (the row R2C of theta
    // counts with the transforms here), and the profile getters return the classes
    for (int k = 0; k < PH_COUNT; ++k) *ms[k] = 0.0;
    for (int c = 0; c < OT_PROF_CLASSES; ++c) {
      const double v = 1e-6 * (double)h->class_ns[c];
      *ms[phase_of(c)] += v;
      p->prof_ms[c] = v;
      p->prof_n[c] = 0;
    }
  }
}

static int run_autotune(ot_plan* p);

// ------------------------------------------------------------------------------------------
// Learned warm start
// ------------------------------------------------------------------------------------------
static int alloc_ws(ot_plan* p) {
  if (p->ws_src) return OT_OK;
  const size_t P = (size_t)p->N * p->M;
  CK(cudaMalloc(&p->ws_src, P * 8));
  CK(cudaMalloc(&p->ws_h, P * 8));
  CK(cudaMalloc(&p->ws_tmp, P * 8));
  CK(cudaMalloc(&p->ws_X, P * OTGB_WS_K * 4));
  CK(cudaMalloc(&p->ws_s, P * 4));
  CK(cudaMalloc(&p->ws_c32, P * 4));
  return OT_OK;
}

// u = u_add + P(src32) in the mixed mode: FP32 forward transforms (an error relative to the
// source in every coefficient, which P turns into a smooth error), the division and the
// inverse transforms in double-float (FP32 round-off there would be grid-scale noise in u,
// which the second differences of the features and of the residual amplify by ~M^2).
// u_add may be null.
static int run_ws_poisson32(ot_plan* p, const float* src32, double* u, const double* u_add,
                            bool lp) {
  LAUNCH(p, OT_PROF_WARMSTART, -1, 1,
         launch_row_r2c<float>(src32, 0, nullptr, nullptr, (C2<float>*)p->spec, p->N, p->M,
                               p->tb32, nullptr, p->stream));
  LAUNCH(p, OT_PROF_WARMSTART, -1, 1,
         launch_col_lbarinv_dd((const float2*)p->spec, (ddc*)p->q64, p->N, p->M, p->tb32,
                               p->tbdd, nullptr, p->stream, lp ? COL_POISSON_LP : COL_POISSON));
  LAUNCH(p, OT_PROF_WARMSTART, -1, 1,
         launch_row_c2r_update_dd((const ddc*)p->q64, u_add, u, 1.0, p->N, p->M, p->tbdd,
                                  nullptr, p->stream));
  return OT_OK;
}

// u = P(src), the FD Poisson solve (row R2C, column pass dividing by the stencil
// Laplacian's eigenvalues, row C2R): FP64 transforms in the FP64 mode; the mixed mode rounds
// src to FP32 (the learned start's sources are FP32 quantities) and takes run_ws_poisson32
static int run_ws_poisson(ot_plan* p, const double* src, double* u, bool lp = false) {
  if (p->precision) {
    LAUNCH(p, OT_PROF_WARMSTART, -1, 1,
           launch_convert<float>(src, 1, p->ws_s, 0, (long)p->N * p->M, p->stream));
    return run_ws_poisson32(p, p->ws_s, u, nullptr, lp);
  }
  C2<double>* sp = (C2<double>*)(p->precision ? p->spec64 : p->spec);
  C2<double>* qq = (C2<double>*)(p->precision ? p->q64 : p->q0);
  LAUNCH(p, OT_PROF_WARMSTART, -1, 1,
         launch_row_r2c<double>(src, 0, nullptr, nullptr, sp, p->N, p->M, p->tb64, nullptr,
                                p->stream));
  LAUNCH(p, OT_PROF_WARMSTART, -1, 1,
         launch_col<double>(lp ? COL_POISSON_LP : COL_POISSON, sp, qq, nullptr, nullptr, p->N,
                            p->M, p->tb64, nullptr, nullptr, p->stream));
  LAUNCH(p, OT_PROF_WARMSTART, -1, 1,
         launch_row_c2r<double>(ROWINV_PLAIN, qq, nullptr, nullptr, nullptr, u, nullptr,
                                nullptr, 0.0, 1.0, p->N, p->M, p->tb64, nullptr, p->stream));
  return OT_OK;
}

// ws_src = log f - log g, ws_h = P(ws_src), ws_X = features at ws_h (f, g, c: the plan's
// translated densities and B-spline coefficients)
static int run_ws_features(ot_plan* p) {
  RET(alloc_ws(p));
  const long P = (long)p->N * p->M;
  if (p->precision) {
    // mixed: the source in FP32 (in ws_s, which the network overwrites later)
    LAUNCH(p, OT_PROF_WARMSTART, -1, 1,
           launch_ws_source32(p->f, p->g, p->ws_s, P, p->stream));
    RET(run_ws_poisson32(p, p->ws_s, p->ws_h, nullptr, false));
  } else {
    LAUNCH(p, OT_PROF_WARMSTART, -1, 1,
           launch_ws_source(p->f, p->g, p->ws_src, P, p->stream));
    RET(run_ws_poisson(p, p->ws_src, p->ws_h));
  }
  LAUNCH(p, OT_PROF_WARMSTART, -1, 1,
         launch_convert<float>(p->c, 1, p->ws_c32, 0, P, p->stream));
  LAUNCH(p, OT_PROF_WARMSTART, -1, 1,
         launch_ws_features(p->f, p->g, p->ws_c32, p->ws_h, p->N, p->M, p->ws_X, p->stream));
  return OT_OK;
}

// u = alpha (h + P(G MLP(X))), G the Gaussian low-pass; alpha and the network's error flag
// in sc (stall: the failure-path test hook of the network kernel)
static int run_warmstart(ot_plan* p, double* u, int stall = 0) {
  const long P = (long)p->N * p->M;
  RET(run_ws_features(p));
  LAUNCH(p, OT_PROF_WARMSTART, -1, 1,
         launch_ws_mlp(p->ws_wpack, p->ws_params, p->ws_X, P, p->ws_s, &p->sc->ws_err, p->sms,
                       p->stream, stall));
  if (p->precision) {
    // u = h + P(G s) straight from the network's FP32 output
    RET(run_ws_poisson32(p, p->ws_s, u, p->ws_h, true));
  } else {
    LAUNCH(p, OT_PROF_WARMSTART, -1, 1, launch_ws_widen(p->ws_s, p->ws_src, P, p->stream));
    RET(run_ws_poisson(p, p->ws_src, p->ws_tmp, true));
    LAUNCH(p, OT_PROF_WARMSTART, -1, 1, launch_ws_sum(p->ws_h, p->ws_tmp, u, P, p->stream));
  }
  LAUNCH(p, OT_PROF_WARMSTART, -1, 2,
         launch_ws_admissible(u, p->N, p->M, p->partials, &p->sc->ticket[TK_WS],
                              &p->sc->ws_err, &p->sc->ws_alpha, p->stream));
  return OT_OK;
}

// theta of a Newton step from the finite-difference system of Sec. 4.1 (A~ theta = h, h =
// (f - f~_n) / tau unless given) by BiCG from theta = 0, into fdbufs(p).x: the iterations run
// in chunks of self-skipping launches, with the state read once per chunk
static constexpr int kBicgChunk = 16;
static int run_bicg(ot_plan* p, const double* h) {
  const long P = (long)p->N * p->M;
  const FdBufs b = fdbufs(p);
  LAUNCH(p, OT_PROF_GMRES_OTHER, -1, 1,
         launch_bicg_init(p->Fraw, h, b, P, p->partials, p->sc, p->max_bicg, p->stream));
  for (;;) {
    for (int k = 0; k < kBicgChunk; ++k)
      LAUNCH(p, OT_PROF_GMRES_OTHER, -1, 3,
             launch_bicg_iteration((const double*)p->coef, b, p->N, p->M, p->partials, p->sc,
                                   p->stream));
    RET(read_scalars(p));
    if (p->hsc->bicg_done) break;
  }
  return OT_OK;
}

template <typename T>
static int solve_impl(ot_plan* p, const double* f_in, const double* g_in, double* phi,
                      ot_stats* st) {
  ot_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof(*st));
  RET(run_autotune(p));
  const long long launches0 = p->launches;
  const int N = p->N, M = p->M;
  const long P = (long)N * M;
  cudaEvent_t ev0, ev1;
  CK(cudaEventCreate(&ev0));
  CK(cudaEventCreate(&ev1));
  CK(cudaEventRecord(ev0, p->stream));
  set_solver_scalars(p);
  CK(cudaMemcpyAsync(p->sc, p->hsc, sizeof(DevScalars), cudaMemcpyHostToDevice, p->stream));
  if (p->translate) {
    LAUNCH(p, OT_PROF_OTHER, -1, 2,
           launch_translate_inputs(f_in, g_in, p->f, p->g, N, M, p->partials, p->sc,
                                   p->stream));
    RET(read_scalars(p));
    if (p->hsc->in_bad) {
      st->status = OT_EINVAL;
      cudaEventDestroy(ev0);
      cudaEventDestroy(ev1);
      return OT_EINVAL;
    }
  } else {
    if (f_in != p->f) CK(cudaMemcpyAsync(p->f, f_in, P * 8, cudaMemcpyDeviceToDevice, p->stream));
    if (g_in != p->g) CK(cudaMemcpyAsync(p->g, g_in, P * 8, cudaMemcpyDeviceToDevice, p->stream));
    // inputs used as given: their statistics and the positivity check only
    LAUNCH(p, OT_PROF_OTHER, -1, 1,
           launch_input_stats(p->f, p->g, N, M, p->partials, p->sc, p->stream));
    RET(read_scalars(p));
    if (p->hsc->in_bad) {
      st->status = OT_EINVAL;
      cudaEventDestroy(ev0);
      cudaEventDestroy(ev1);
      return OT_EINVAL;
    }
  }
  RET(run_prefilter(p, p->g, p->c));
  if (p->warm_start == 1) {
    if (phi != p->u) CK(cudaMemcpyAsync(p->u, phi, P * 8, cudaMemcpyDeviceToDevice, p->stream));
  } else if (p->warm_start == 2) {
    const int stall = p->ws_stall;
    p->ws_stall = 0;
    RET(run_warmstart(p, p->u, stall));
  } else {
    CK(cudaMemsetAsync(p->u, 0, P * 8, p->stream));
  }
  LAUNCH(p, OT_PROF_RESIDUAL, -1, 1,
         residual_launch<T>(p, p->f, p->c, p->u, p->Fraw, nullptr, 0));
  RET(read_scalars(p));
  int status = OT_OK;
  double s = 1.0;
  bool tau_one = false;
  for (int n = 0;; ++n) {
    const DevScalars* h = p->hsc;
    st->res_inf = h->res_inf;
    st->min_det = h->min_det;
    st->mean_fn = h->mean_fn;
    if (!h->admissible) {
      status = OT_EDIVERGED;
      break;
    }
    if (h->res_inf < p->tol) break;
    if (n >= p->max_newton) {
      status = OT_ENOCONV;
      break;
    }
    if (p->tau_switch > 0.0 && h->res_inf < p->tau_switch && !tau_one) {
      // tau schedule: the damping of the remaining steps is 1
      static const double one = 1.0;
      CK(cudaMemcpyAsync(&p->sc->tau, &one, sizeof(double), cudaMemcpyHostToDevice,
                         p->stream));
      tau_one = true;
    }
    if (p->linsolver) {
      RET(run_bicg(p, nullptr));
      st->gmres_iters += p->hsc->bicg_iters;
      st->gmres_cycles += 1;
    } else {
      int rc = run_gmres<T>(p);
      if (rc != OT_OK) return rc;
      st->gmres_iters += p->hsc->iters;
      st->gmres_cycles += p->hsc->cycles;
    }
    bool accepted = false;
    for (;;) {
      if (p->linsolver)
        LAUNCH(p, OT_PROF_ROW_C2R_UPDATE, -1, 1,
               launch_axpy_to(p->u, fdbufs(p).x, s, p->ucand, P, p->stream));
      else
        RET(run_theta<T>(p, p->u, p->ucand, s, false));
      LAUNCH(p, OT_PROF_RESIDUAL, -1, 1,
             residual_launch<T>(p, p->f, p->c, p->ucand, p->Fraw, nullptr, 0));
      RET(read_scalars(p));
      if (!p->safeguard || p->hsc->admissible || s < 0x1p-30) {
        accepted = true;
        break;
      }
      s *= 0.5;
      st->step_halvings++;
    }
    (void)accepted;
    double* t = p->u;
    p->u = p->ucand;
    p->ucand = t;
    st->newton_iters = n + 1;
    s = (2.0 * s < 1.0) ? 2.0 * s : 1.0;
  }
  // final l2 residual, mean-zero gauge (Sec. 3.1), result
  if (status != OT_EDIVERGED || p->hsc->k1_nonfinite == 0) {
    LAUNCH(p, OT_PROF_OTHER, -1, 1,
           launch_residual_l2(p->Fraw, N, M, p->partials, p->sc, p->stream));
  }
  LAUNCH(p, OT_PROF_OTHER, -1, 2,
         launch_subtract_mean(p->u, N, M, p->partials, p->sc, p->dmean, p->stream));
  if (p->transport)
    LAUNCH(p, OT_PROF_OTHER, -1, 1,
           launch_transport(p->f, p->u, N, M, nullptr, p->partials,
                            &p->sc->ticket[TK_TRANSPORT], &p->sc->dist, p->stream));
  if (p->stamping) CK(launch_stamp(p->sc, -1, p->stream));
  if (phi != p->u) CK(cudaMemcpyAsync(phi, p->u, P * 8, cudaMemcpyDeviceToDevice, p->stream));
  CK(cudaMemcpyAsync(&st->phi_mean, p->dmean, 8, cudaMemcpyDeviceToHost, p->stream));
  CK(cudaEventRecord(ev1, p->stream));
  RET(read_scalars(p));
  st->res_l2 = sqrt(p->hsc->res_l2sum / (double)P);
  st->ws_alpha = p->hsc->ws_alpha;
  if (p->hsc->ws_err) note_ws_timeout(st, __LINE__);
  fill_common_stats(p, p->hsc, st);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev0, ev1);
  st->ms_total = ms;
  st->kernel_launches = (int32_t)(p->launches - launches0);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  st->status = status;
  return status;
}

// ------------------------------------------------------------------------------------------
// Graph-launched solve: the same sequence as solve_impl, captured once.  The Newton loop,
// the GMRES cycle loop, each Arnoldi step and the step-halving loop are conditional nodes
// whose handles are set by the device-side control kernel (k_ctl) and by the Arnoldi update.
// ------------------------------------------------------------------------------------------

// Add a conditional node after the current capture frontier of stream s; *body receives its
// body graph and *h its handle (created in the graph being captured on s).
static int add_conditional(cudaStream_t s, cudaGraphConditionalNodeType type,
                           unsigned long long* h, cudaGraph_t* body) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, &ed, &nd));
  if (cst != cudaStreamCaptureStatusActive) return OT_ECUDA;
  cudaGraphConditionalHandle hc;
  CK(cudaGraphConditionalHandleCreate(&hc, g, 0, 0));
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = hc;
  cp.conditional.type = type;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, deps, ed, nd, &cp));
  CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                         cudaStreamSetCaptureDependencies));
  *h = (unsigned long long)hc;
  *body = cp.conditional.phGraph_out[0];
  return OT_OK;
}

static int begin_body(ot_plan* p, int level, cudaGraph_t body) {
  CK(cudaStreamBeginCaptureToGraph(p->cs[level], body, nullptr, nullptr, 0,
                                   cudaStreamCaptureModeRelaxed));
  p->stream = p->cs[level];
  p->last_phase = -1;
  return OT_OK;
}

static int end_body(ot_plan* p, int level) {
  cudaGraph_t out = nullptr;
  CK(cudaStreamEndCapture(p->cs[level], &out));
  p->stream = p->cs[level - 1];
  p->last_phase = -1;
  return OT_OK;
}

// theta = Lbar^{-1} sigma, candidate u_(1-upar) = u_upar + s theta (s, upar from the device),
// residual at the candidate, accept/halve (batched: for the pairs of the current mask)
template <typename T>
static int capture_candidate(ot_plan* p) {
  RET(run_theta<T>(p, p->u, p->ucand, 1.0, true));
  LAUNCH(p, OT_PROF_RESIDUAL, -1, 1,
         residual_launch<T>(p, p->f, p->c, p->u, p->Fraw, p->ucand, 1));
  LAUNCH(p, OT_PROF_OTHER, -1, 1, launch_ctl(CTL_ACCEPT, p->sc, p->stream, 5, btc(p)));
  return OT_OK;
}

// The solve as one captured sequence.  A batched plan (a size class of a plan set) captures
// the same sequence over all its pairs: every launch serves the pairs its mask selects (the
// current Newton loop, GMRES cycle loop or step-halving loop of each pair), the control
// kernel keeps each loop running while any pair needs it, and all Arnoldi steps are plain
// self-skipping launches (a pair whose cycle ended skips them).
template <typename T>
static int capture_solve(ot_plan* p) {
  const int N = p->N, M = p->M;
  const long P = (long)N * M;
  const bool batched = p->slab_base != nullptr;
  T* V = (T*)p->V;
  T* w = (T*)p->w;
  T* sigma = (T*)p->sigma;
  long long k0 = p->launches;
  p->cur_mask = MASK_ALL;
  if (p->translate)
    LAUNCH(p, OT_PROF_OTHER, -1, 2,
           launch_translate_inputs(p->f, p->g, p->f, p->g, N, M, p->partials, p->sc,
                                   p->stream, btc(p)));
  else
    LAUNCH(p, OT_PROF_OTHER, -1, 1,
           launch_input_stats(p->f, p->g, N, M, p->partials, p->sc, p->stream, btc(p)));
  RET(run_prefilter(p, p->g, p->c));
  if (p->warm_start == 2) RET(run_warmstart(p, p->u));
  LAUNCH(p, OT_PROF_RESIDUAL, -1, 1,
         residual_launch<T>(p, p->f, p->c, p->u, p->Fraw, p->ucand, 0));
  const int top = (int)(p->launches - k0) + 1;
  LAUNCH(p, OT_PROF_OTHER, -1, 1, launch_ctl(CTL_NEWTON, p->sc, p->stream, top, btc(p)));
  cudaGraph_t b1, b2, b3, b4, b5;
  // ---- Newton loop
  RET(add_conditional(p->cs[0], cudaGraphCondTypeWhile, &p->h_newton, &b1));
  RET(begin_body(p, 1, b1));
  p->cur_mask = MASK_NEWTON;
  if (p->forcing)
    LAUNCH(p, OT_PROF_OTHER, -1, 1, launch_ctl(CTL_FORCING, p->sc, p->stream, 1, btc(p)));
  LAUNCH(p, OT_PROF_GMRES_OTHER, -1, 1,
         launch_gmres_init<T>(p->Fraw, w, V, P, 0, p->partials, p->sc, p->kblocks, p->stream,
                              sigma, btc(p)));
  LAUNCH(p, OT_PROF_OTHER, -1, 1, launch_ctl(CTL_PRE_CYCLE, p->sc, p->stream, 2, btc(p)));
  // ---- GMRES cycles
  RET(add_conditional(p->cs[1], cudaGraphCondTypeWhile, &p->h_cycle, &b2));
  RET(begin_body(p, 2, b2));
  p->cur_mask = MASK_CYCLE;
  // (the count: this kernel, and the row pass of v_0 that a fused-update cycle starts with)
  LAUNCH(p, OT_PROF_OTHER, -1, 1,
         launch_ctl(CTL_CYCLE_BEGIN, p->sc, p->stream,
                    batched ? 1 + 5 * p->m : (fused_update_on<T>(p) ? 2 : 1), btc(p)));
  // The first K steps of a cycle are plain kernels that skip themselves once the cycle is
  // done; the rest run as the body of one WHILE node, one step (its index read on the
  // device) per iteration, the node's handle set by each step's Givens close.  Measured on
  // this GB300: a WHILE iteration costs ~4 us over its kernels, an IF node ~6 us when skipped
  // and ~12 us when taken, and a skipped launch of a full-grid step kernel ~2-3 us.  A batched
  // plan runs every step as a plain launch (the cycles of its pairs end at different steps).
  const int K = batched ? p->m : (p->m < p->uncond ? p->m : p->uncond);
  for (int k = 0; k < OTGB_MAXM; ++k) p->h_step[k] = 0;
  RET(run_cycle_rows<T>(p, &p->sc->cycle_done));
  for (int j = 0; j < K; ++j) RET(run_arnoldi_step<T>(p, j, &p->sc->cycle_done));
  if (K < p->m) {
    unsigned long long h_tail = 0;
    RET(add_conditional(p->cs[2], cudaGraphCondTypeWhile, &h_tail, &b3));
    RET(begin_body(p, 3, b3));
    RET(run_arnoldi_step<T>(p, K, nullptr));
    RET(end_body(p, 3));
    // step j's close sets the handle of step j + 1: the tail's for j + 1 = K .. m (at m it
    // ends the loop)
    for (int k = K; k <= p->m && k < OTGB_MAXM; ++k) p->h_step[k] = h_tail;
  }
  LAUNCH(p, OT_PROF_GMRES_OTHER, -1, 1, launch_gmres_finish(p->sc, p->stream, btc(p)));
  LAUNCH(p, OT_PROF_GMRES_OTHER, -1, 1,
         launch_gmres_combine<T>(V, sigma, P, p->sc, p->kblocks, p->stream, btc(p)));
  LAUNCH(p, OT_PROF_OTHER, -1, 1, launch_ctl(CTL_CYCLE_END, p->sc, p->stream, 3, btc(p)));
  RET(add_conditional(p->cs[2], cudaGraphCondTypeIf, &p->h_restart, &b4));
  RET(begin_body(p, 3, b4));
  RET(run_matvec<T>(p, sigma, nullptr, nullptr, w, nullptr, -1));
  LAUNCH(p, OT_PROF_GMRES_OTHER, -1, 1,
         launch_gmres_init<T>(p->Fraw, w, V, P, 1, p->partials, p->sc, p->kblocks, p->stream,
                              nullptr, btc(p)));
  RET(end_body(p, 3));
  RET(end_body(p, 2));
  p->cur_mask = MASK_NEWTON;
  LAUNCH(p, OT_PROF_OTHER, -1, 1, launch_ctl(CTL_GMRES_DONE, p->sc, p->stream, 1, btc(p)));
  // ---- candidate, then halve while inadmissible
  RET(capture_candidate<T>(p));
  RET(add_conditional(p->cs[1], cudaGraphCondTypeWhile, &p->h_halve, &b5));
  RET(begin_body(p, 2, b5));
  p->cur_mask = MASK_HALVE;
  RET(capture_candidate<T>(p));
  RET(end_body(p, 2));
  p->cur_mask = MASK_NEWTON;
  LAUNCH(p, OT_PROF_OTHER, -1, 1, launch_ctl(CTL_NEWTON, p->sc, p->stream, 1, btc(p)));
  RET(end_body(p, 1));
  p->cur_mask = MASK_ALL;
  // ---- final residual norm and mean-zero gauge
  LAUNCH(p, OT_PROF_OTHER, -1, 1,
         launch_residual_l2(p->Fraw, N, M, p->partials, p->sc, p->stream, btc(p)));
  UPair up{p->u, p->ucand};
  LAUNCH(p, OT_PROF_OTHER, -1, 2,
         launch_final_gauge(up, p->uout, N, M, p->partials, p->sc,
                            batched ? &p->sc->gauge_mean : p->dmean, p->stream, btc(p)));
  p->top_kernels = 3;  // residual_l2 + gauge (2), counted on the host
  if (p->transport && !batched) {
    LAUNCH(p, OT_PROF_OTHER, -1, 1,
           launch_transport(p->f, p->uout, N, M, nullptr, p->partials,
                            &p->sc->ticket[TK_TRANSPORT], &p->sc->dist, p->stream));
    p->top_kernels += 1;
  }
  if (p->stamping) CK(launch_stamp(p->sc, -1, p->stream));
  return OT_OK;
}

// ------------------------------------------------------------------------------------------
// Autotuner of the FP32 matvec passes: each variant (generic / concurrent transforms /
// warp-synchronous radix-32 / 4 elements per thread) of the row R2C, column and row combine
// passes is launched back to back on the plan's own buffers inside a captured graph and timed
// with CUDA events; the fastest is kept, and the choice is cached per (N, M) for the process.
// ------------------------------------------------------------------------------------------
static std::mutex g_tune_mutex;
static std::vector<std::vector<int>> g_tune_cache;  // {N, M, r2c, col, comb, col_q, mv_reg}

static int run_autotune(ot_plan* p) {
  if (!p->precision || !p->autotune || p->tuned) return OT_OK;
  const int N = p->N, M = p->M;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    for (auto& e : g_tune_cache)
      if (e[0] == N && e[1] == M) {
        p->tb32.var_r2c = e[2];
        p->tb32.var_col = e[3];
        p->tb32.var_comb = e[4];
        p->tb32.col_q = e[5];
        p->tb32.mv_reg = e[6];
        p->tuned = 1;
        return OT_OK;
      }
  }
  const long P = (long)N * M;
  cudaStream_t st = p->stream;
  CK(cudaMemsetAsync(p->V, 0, P * 4, st));
  CK(cudaMemsetAsync(p->spec, 0, P * 4, st));
  CK(cudaMemsetAsync(p->q0, 0, P * 4, st));
  CK(cudaMemsetAsync(p->q1, 0, P * 4, st));
  CK(cudaMemsetAsync(p->q2, 0, P * 4, st));
  CK(cudaMemsetAsync(p->coef, 0, 5 * P * 4, st));
  CK(cudaMemsetAsync(p->sc, 0, sizeof(DevScalars), st));
  SpecTables& tb = p->tb32;
  auto timed = [&](int cls) -> float {
    auto one = [&]() -> cudaError_t {
      if (tb.mv_reg) {
        if (cls == 0)
          return launch_mvT_r2c((const float*)p->V, P, nullptr, nullptr, (float2*)p->spec, N,
                                M, tb, nullptr, p->stream);
        if (cls == 1)
          return launch_mvT_col((const float2*)p->spec, (float2*)p->q0, (float2*)p->q1,
                                (float2*)p->q2, N, M, tb, p->sc, nullptr, p->stream);
        return launch_mvT_combine((const float2*)p->q0, (const float2*)p->q1,
                                  (const float2*)p->q2, (const float*)p->coef, (float*)p->w, N,
                                  M, tb, nullptr, p->stream);
      }
      if (cls == 0)
        return launch_row_r2c<float>((const float*)p->V, P, nullptr, nullptr,
                                     (C2<float>*)p->spec, N, M, tb, nullptr, p->stream);
      if (cls == 1)
        return launch_col<float>(COL_MATVEC, (C2<float>*)p->spec, (C2<float>*)p->q0,
                                 (C2<float>*)p->q1, (C2<float>*)p->q2, N, M, tb, p->sc,
                                 nullptr, p->stream);
      return launch_row_c2r<float>(ROWINV_COMBINE, (C2<float>*)p->q0, (C2<float>*)p->q1,
                                   (C2<float>*)p->q2, (const float*)p->coef, (float*)p->w,
                                   nullptr, nullptr, 0.0, 1.0, N, M, tb, nullptr, p->stream);
    };
    // 3 warm-up launches, then 30 timed launches replayed as one graph: the candidates are
    // within a few percent of each other at the sizes of interest, and stream launches are
    // paced on a ~2 us grid that would hide their differences
    for (int r = 0; r < 3; ++r)
      if (one() != cudaSuccess) return 1e30f;
    float ms = 0.f;
    if (graph_time(p, one, 30, &ms) != OT_OK) {
      cudaGetLastError();
      return 1e30f;
    }
    return ms;
  };
  tb.col_q = 0;
  tb.mv_reg = 0;
  int* vars[3] = {&tb.var_r2c, &tb.var_col, &tb.var_comb};
  // (the row pass on row pairs is not a candidate: the choice also selects the fused Arnoldi
  // update, which runs once per Krylov step, and its row-pair form measured slower at
  // 512^2 and 1024^2 -- 7.5 / 9.1 us against 6.5 / 8.8 us -- although the pair row pass
  // alone is faster; it stays selectable through OT_OPT_FFT_VARIANT)
  const int ncand[3] = {3, col_pair_supported(N, M) ? 5 : 4, comb_pair_supported(N, M) ? 5 : 4};
  const int cand[3][5] = {{VAR_GENERIC, VAR_WARP, VAR_E4, VAR_E4, VAR_E4},
                          {VAR_GENERIC, VAR_PAR, VAR_WARP, VAR_E4, VAR_PAIR},
                          {VAR_GENERIC, VAR_PAR, VAR_WARP, VAR_E4, VAR_PAIR}};
  // every candidate is timed in two rounds and keeps its faster time: the first launches
  // of a process run while the clocks and caches settle, which would otherwise penalise
  // whichever candidate is timed first
  float tsum = 0.f;  // the chosen per-pass variants' times, summed
  for (int cls = 0; cls < 3; ++cls) {
    int best = VAR_GENERIC, bestq = 0;
    float tbest = 1e30f;
    float tms[2][5][3];
    for (int round = 0; round < 2; ++round)
      for (int k = 0; k < ncand[cls]; ++k) {
        *vars[cls] = cand[cls][k];
        // the column variants with per-block column counts (0 = heuristic)
        const bool qv = cls == 1 && (cand[cls][k] == VAR_GENERIC || cand[cls][k] == VAR_E4);
        int qi = 0;
        for (int qc : {0, 1, 4}) {
          if (qc && !qv) break;
          tb.col_q = qc;
          tms[round][k][qi] = timed(cls);
          if (round == 1) {
            const float t = std::min(tms[0][k][qi], tms[1][k][qi]);
            if (t < tbest) {
              tbest = t;
              best = cand[cls][k];
              bestq = qc;
            }
          }
          ++qi;
        }
      }
    *vars[cls] = best;
    if (cls == 1) tb.col_q = bestq;
    tsum += tbest;
  }
  // the register-resident passes on the transposed spectrum replace all three at once:
  // kept when their summed time is below the per-pass choice's (two rounds, faster kept)
  if (tb.t2rA) {
    tb.mv_reg = 1;
    float treg[2] = {0.f, 0.f};
    for (int round = 0; round < 2; ++round)
      for (int cls = 0; cls < 3; ++cls) treg[round] += timed(cls);
    tb.mv_reg = std::min(treg[0], treg[1]) < tsum ? 1 : 0;
  }

  cudaGetLastError();
  p->tuned = 1;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache.push_back({N, M, tb.var_r2c, tb.var_col, tb.var_comb, tb.col_q, tb.mv_reg});
  return OT_OK;
}

// End every capture still open on the plan's capture streams (after a failed capture).
static void abandon_captures(ot_plan* p) {
  for (int k = 3; k >= 0; --k) {
    if (!p->cs[k]) continue;
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(p->cs[k], &cst) == cudaSuccess &&
        cst != cudaStreamCaptureStatusNone) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(p->cs[k], &g);
      if (g && k == 0) cudaGraphDestroy(g);
    }
  }
  cudaGetLastError();
}

// OT_OPT_L2_PERSIST: the GMRES basis V_0..V_m (read again by every Arnoldi step's multi-dot
// and update) as persisting L2 lines for the kernels of the captured graph, so that the
// transform passes' traffic between two steps does not evict it: an access-policy window on
// the capture streams (captured into every kernel node), with the process's persisting-L2
// limit raised to the window's size (at most the device's maximum).  Off: no window.
static int apply_l2_window(ot_plan* p, size_t elem) {
  cudaStreamAttrValue a;
  memset(&a, 0, sizeof(a));
  if (p->l2persist && !p->slab_base) {
    const size_t vbytes = (size_t)(p->m + 1) * p->N * p->M * elem;
    int maxp = 0, maxw = 0;
    CK(cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, p->device));
    CK(cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, p->device));
    const size_t win = std::min(vbytes, (size_t)maxw);
    const size_t want = std::min(win, (size_t)maxp);
    size_t cur = 0;
    CK(cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize));
    if (cur < want) CK(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want));
    if (win > 0 && want > 0) {
      a.accessPolicyWindow.base_ptr = p->V;
      a.accessPolicyWindow.num_bytes = win;
      a.accessPolicyWindow.hitRatio = (float)std::min(1.0, (double)want / (double)win);
      a.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
      a.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    }
  }
  for (int k = 0; k < 4; ++k)
    CK(cudaStreamSetAttribute(p->cs[k], cudaStreamAttributeAccessPolicyWindow, &a));
  return OT_OK;
}

template <typename T>
static int build_graph(ot_plan* p) {
  RET(run_autotune(p));
  free_graph(p);
  for (int k = 0; k < 4; ++k)
    if (!p->cs[k]) CK(cudaStreamCreateWithFlags(&p->cs[k], cudaStreamNonBlocking));
  RET(apply_l2_window(p, sizeof(T)));
  cudaStream_t saved = p->stream;
  const int saved_prof = p->profile;
  const long long saved_launches = p->launches;
  p->profile = 0;
  p->stream = p->cs[0];
  CK(cudaStreamBeginCapture(p->cs[0], cudaStreamCaptureModeRelaxed));
  p->stamping = p->phase_times;
  p->last_phase = -1;
  int rc = capture_solve<T>(p);
  p->stamping = 0;
  if (rc != OT_OK) {
    p->stream = saved;
    p->profile = saved_prof;
    p->launches = saved_launches;
    abandon_captures(p);
    return rc;
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(p->cs[0], &g);
  p->stream = saved;
  p->profile = saved_prof;
  p->launches = saved_launches;
  if (rc != OT_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc != OT_OK ? rc : OT_ECUDA;
  }
  p->graph = g;
  e = cudaGraphInstantiate(&p->gexec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    p->graph = nullptr;
    p->gexec = nullptr;
    return OT_ECUDA;
  }
  p->gkey_prec = p->precision;
  p->gkey_m = p->m;
  p->gkey_translate = p->translate;
  p->gkey_ws = p->warm_start;
  p->gu_a = p->u;
  p->gu_b = p->ucand;
  return OT_OK;
}

// Fill the initial device scalars of a graph-launched solve into *h (host).
static void graph_scalars(ot_plan* p, DevScalars* h) {
  set_solver_scalars(p);
  *h = *p->hsc;
  h->graph = 1;
  h->h_newton = p->h_newton;
  h->h_cycle = p->h_cycle;
  h->h_restart = p->h_restart;
  h->h_halve = p->h_halve;
  for (int k = 0; k < OTGB_MAXM; ++k) h->h_step[k] = p->h_step[k];
  h->steps_uncond = p->m < p->uncond ? p->m : p->uncond;
}

// Enqueue one graph-launched solve on stream xs: inputs into the plan's buffers, the initial
// scalars from `init` (pinned host), the graph, phi out, and the final scalars / mean into
// the pinned host slots.  Nothing waits here.
template <typename T>
static int graph_enqueue(ot_plan* p, cudaStream_t xs, const double* f_in, const double* g_in,
                         double* phi, const DevScalars* init, DevScalars* slot,
                         double* mean_slot) {
  const long P = (long)p->N * p->M;
  double* ua = p->gu_a;
  if (f_in != p->f) CK(cudaMemcpyAsync(p->f, f_in, P * 8, cudaMemcpyDeviceToDevice, xs));
  if (g_in != p->g) CK(cudaMemcpyAsync(p->g, g_in, P * 8, cudaMemcpyDeviceToDevice, xs));
  if (p->warm_start == 1) {
    if (phi != ua) CK(cudaMemcpyAsync(ua, phi, P * 8, cudaMemcpyDeviceToDevice, xs));
  } else if (p->warm_start == 0) {
    CK(cudaMemsetAsync(ua, 0, P * 8, xs));
  }  // 2: the captured warm start writes ua
  CK(cudaMemcpyAsync(p->sc, init, sizeof(DevScalars), cudaMemcpyHostToDevice, xs));
  CK(cudaGraphLaunch(p->gexec, xs));
  if (phi != p->uout) CK(cudaMemcpyAsync(phi, p->uout, P * 8, cudaMemcpyDeviceToDevice, xs));
  CK(cudaMemcpyAsync(mean_slot, p->dmean, 8, cudaMemcpyDeviceToHost, xs));
  CK(cudaMemcpyAsync(slot, p->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, xs));
  return OT_OK;
}

static void graph_collect(ot_plan* p, const DevScalars* h, double mean, ot_stats* st) {
  const long P = (long)p->N * p->M;
  st->status = h->status;
  st->newton_iters = h->newton_n;
  st->gmres_iters = h->gmres_iters_total;
  st->gmres_cycles = h->gmres_cycles_total;
  st->step_halvings = h->halvings;
  st->res_inf = h->res_inf;
  st->min_det = h->min_det;
  st->mean_fn = h->mean_fn;
  st->res_l2 = sqrt(h->res_l2sum / (double)P);
  st->phi_mean = mean;
  st->kernel_launches = (int32_t)(h->kcount + p->top_kernels);
  st->ws_alpha = h->ws_alpha;
  if (h->ws_err) note_ws_timeout(st, __LINE__);
  fill_common_stats(p, h, st);
  p->launches += h->kcount + p->top_kernels;
}

template <typename T>
static int ensure_graph(ot_plan* p) {
  if (!p->gexec || p->gkey_prec != p->precision || p->gkey_m != p->m ||
      p->gkey_translate != p->translate || p->gkey_ws != p->warm_start)
    return build_graph<T>(p);
  return OT_OK;
}

template <typename T>
static int solve_graph_impl(ot_plan* p, const double* f_in, const double* g_in, double* phi,
                            ot_stats* st) {
  ot_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof(*st));
  RET(ensure_graph<T>(p));
  cudaEvent_t ev0, ev1;
  CK(cudaEventCreate(&ev0));
  CK(cudaEventCreate(&ev1));
  CK(cudaEventRecord(ev0, p->stream));
  graph_scalars(p, p->hsc);
  double mean = 0.0;
  RET(graph_enqueue<T>(p, p->stream, f_in, g_in, phi, p->hsc, p->hsc, &st->phi_mean));
  CK(cudaEventRecord(ev1, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  mean = st->phi_mean;
  graph_collect(p, p->hsc, mean, st);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev0, ev1);
  st->ms_total = ms;
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  return st->status;
}

// host-driven solve, with phase stamps while OT_OPT_PHASE_TIMES is set
static int host_solve(ot_plan* p, const double* f, const double* g, double* phi,
                      ot_stats* st) {
  p->stamping = p->phase_times;
  p->last_phase = -1;
  const int rc =
      p->precision ? solve_impl<float>(p, f, g, phi, st) : solve_impl<double>(p, f, g, phi, st);
  p->stamping = 0;
  return rc;
}

// A solve through the captured graph (else host-driven): the graph option on, no profile,
// and not the finite-difference comparison path, which runs host-driven (one read per BiCG
// chunk)
static bool graph_path(const ot_plan* p) {
  return p->use_graph && !p->profile && !p->linsolver;
}

static int solve_once(ot_plan* p, const double* f, const double* g, double* phi,
                      ot_stats* st) {
  if (graph_path(p))
    return p->precision ? solve_graph_impl<float>(p, f, g, phi, st)
                        : solve_graph_impl<double>(p, f, g, phi, st);
  return host_solve(p, f, g, phi, st);
}

// The remedy of Sec. 3.2 / Sec. 5.3 for an iterate that loses convexity: solve again with
// twice the step parameter tau (up to tau_retry times); phi and stats are those of the last
// attempt.  The plan's tau is restored.
static int solve_with_retry(ot_plan* p, const double* f, const double* g, double* phi,
                            ot_stats* st, int rc) {
  const double tau0 = p->tau;
  for (int r = 0; r < p->tau_retry && rc == OT_EDIVERGED; ++r) {
    p->tau *= 2.0;
    rc = solve_once(p, f, g, phi, st);
  }
  p->tau = tau0;
  return rc;
}

extern "C" int ot_solve(ot_plan* p, const double* f, const double* g, double* phi,
                        ot_stats* st) {
  if (!p || !f || !g || !phi || !p->ready) return OT_EINVAL;
  CK(cudaSetDevice(p->device));
  ot_stats local;
  if (!st) st = &local;
  return solve_with_retry(p, f, g, phi, st, solve_once(p, f, g, phi, st));
}

extern "C" int ot_solve_host(ot_plan* p, const double* f, const double* g, double* phi,
                             ot_stats* st) {
  if (!p || !f || !g || !phi || !p->ready) return OT_EINVAL;
  CK(cudaSetDevice(p->device));
  const size_t bytes = (size_t)p->N * p->M * 8;
  // stage f, g in the plan's translated-density buffers (translated in place)
  CK(cudaMemcpyAsync(p->f, f, bytes, cudaMemcpyHostToDevice, p->stream));
  CK(cudaMemcpyAsync(p->g, g, bytes, cudaMemcpyHostToDevice, p->stream));
  const bool graph = graph_path(p);
  if (p->warm_start == 1)
    CK(cudaMemcpyAsync(graph ? p->uout : p->u, phi, bytes, cudaMemcpyHostToDevice, p->stream));
  int rc;
  if (graph) {
    rc = p->precision ? solve_graph_impl<float>(p, p->f, p->g, p->uout, st)
                      : solve_graph_impl<double>(p, p->f, p->g, p->uout, st);
    if (rc == OT_ECUDA || rc == OT_ENOMEM || rc == OT_EINVAL) return rc;
    CK(cudaMemcpyAsync(phi, p->uout, bytes, cudaMemcpyDeviceToHost, p->stream));
  } else {
    rc = host_solve(p, p->f, p->g, p->u, st);
    if (rc == OT_ECUDA || rc == OT_ENOMEM || rc == OT_EINVAL) return rc;
    CK(cudaMemcpyAsync(phi, p->u, bytes, cudaMemcpyDeviceToHost, p->stream));
  }
  CK(cudaStreamSynchronize(p->stream));
  return rc;
}

// Independent solves on several plans: every problem's graph is enqueued on the execution
// stream of its plan (problems sharing a plan run back to back there; different plans run
// concurrently), and the host synchronises once at the end.  Result slots are pinned host
// memory kept across calls (grown when a call has more problems than any before).
static std::mutex g_batch_mutex;
static DevScalars* g_batch_slots = nullptr;
static double* g_batch_means = nullptr;
static size_t g_batch_cap = 0;

extern "C" int ot_solve_plans(int32_t count, ot_plan* const* plans, const double* const* f,
                                const double* const* g, double* const* phi, ot_stats* stats) {
  if (count < 0 || (count > 0 && (!plans || !f || !g || !phi))) return OT_EINVAL;
  for (int k = 0; k < count; ++k)
    if (!plans[k] || !plans[k]->ready || !f[k] || !g[k] || !phi[k]) return OT_EINVAL;
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  if ((size_t)count > g_batch_cap) {
    if (g_batch_slots) cudaFreeHost(g_batch_slots);
    if (g_batch_means) cudaFreeHost(g_batch_means);
    g_batch_slots = nullptr;
    g_batch_means = nullptr;
    g_batch_cap = 0;
    CK(cudaMallocHost(&g_batch_slots, sizeof(DevScalars) * count));
    CK(cudaMallocHost(&g_batch_means, sizeof(double) * count));
    g_batch_cap = count;
  }
  std::vector<ot_plan*> uniq;
  for (int k = 0; k < count; ++k) {
    ot_plan* p = plans[k];
    bool seen = false;
    for (auto q : uniq) seen |= (q == p);
    if (!seen) uniq.push_back(p);
  }
  // graphs, initial scalars and ordering after each plan's own stream
  for (auto p : uniq) {
    CK(cudaSetDevice(p->device));
    if (!graph_path(p)) continue;
    RET(p->precision ? ensure_graph<float>(p) : ensure_graph<double>(p));
    graph_scalars(p, p->hinit);
    cudaEvent_t e;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CK(cudaEventRecord(e, p->stream));
    CK(cudaStreamWaitEvent(p->cs[0], e, 0));
    cudaEventDestroy(e);
  }
  int first = OT_OK;
  for (int k = 0; k < count; ++k) {
    ot_plan* p = plans[k];
    CK(cudaSetDevice(p->device));
    if (!graph_path(p)) {  // host-driven plans: one after another
      ot_stats tmp;
      int rc = ot_solve(p, f[k], g[k], phi[k], &tmp);
      g_batch_slots[k].status = rc;
      if (stats) stats[k] = tmp;
      continue;
    }
    int rc = p->precision
                 ? graph_enqueue<float>(p, p->cs[0], f[k], g[k], phi[k], p->hinit,
                                        &g_batch_slots[k], &g_batch_means[k])
                 : graph_enqueue<double>(p, p->cs[0], f[k], g[k], phi[k], p->hinit,
                                         &g_batch_slots[k], &g_batch_means[k]);
    if (rc != OT_OK) return rc;
  }
  for (auto p : uniq) {
    CK(cudaSetDevice(p->device));
    if (graph_path(p)) CK(cudaStreamSynchronize(p->cs[0]));
  }
  for (int k = 0; k < count; ++k) {
    ot_plan* p = plans[k];
    if (graph_path(p)) {
      ot_stats tmp;
      memset(&tmp, 0, sizeof(tmp));
      graph_collect(p, &g_batch_slots[k], g_batch_means[k], &tmp);
      if (tmp.status == OT_EDIVERGED && p->tau_retry > 0) {
        const int rc = solve_with_retry(p, f[k], g[k], phi[k], &tmp, OT_EDIVERGED);
        if (rc == OT_ECUDA || rc == OT_ENOMEM || rc == OT_EINVAL) return rc;
      }
      if (stats) stats[k] = tmp;
      if (tmp.status != OT_OK && first == OT_OK) first = tmp.status;
    } else if (g_batch_slots[k].status != OT_OK && first == OT_OK) {
      first = g_batch_slots[k].status;
    }
  }
  return first;
}

// ------------------------------------------------------------------------------------------
// step-level entry points
// ------------------------------------------------------------------------------------------
extern "C" int ot_prefilter(ot_plan* p, const double* g, double* c) {
  if (!p || !p->ready || !g || !c) return OT_EINVAL;
  CK(cudaSetDevice(p->device));
  RET(run_prefilter(p, g, c));
  CK(cudaStreamSynchronize(p->stream));
  return OT_OK;
}

template <typename T>
static int eval_residual_impl(ot_plan* p, const double* f, const double* c, const double* u,
                              double* F, double* coef, double* scal) {
  const int N = p->N, M = p->M;
  const long P = (long)N * M;
  set_solver_scalars(p);
  CK(cudaMemcpyAsync(p->sc, p->hsc, sizeof(DevScalars), cudaMemcpyHostToDevice, p->stream));
  if (sizeof(T) == 4) {
    LAUNCH(p, OT_PROF_OTHER, -1, 1, launch_split_dd(c, p->cdd, P, p->stream));
    LAUNCH(p, OT_PROF_OTHER, -1, 1, launch_split_dd(f, p->fdd, P, p->stream));
  }
  if (p->interp)  // c holds g: its grid gradient for the interpolated grad g
    LAUNCH(p, OT_PROF_OTHER, -1, 1,
           launch_grad4(c, N, M, p->gxy, p->gxy + P, p->gxy32, p->gxy32 + P, p->stream));
  LAUNCH(p, OT_PROF_RESIDUAL, -1, 1,
         residual_launch<T>(p, f, c, u, p->Fraw, nullptr, 0));
  LAUNCH(p, OT_PROF_OTHER, -1, 1,
         launch_residual_l2(p->Fraw, N, M, p->partials, p->sc, p->stream));
  if (F) LAUNCH(p, OT_PROF_OTHER, -1, 1, launch_shifted_residual(p->Fraw, F, N, M, p->sc, p->stream));
  if (coef)
    LAUNCH(p, OT_PROF_OTHER, -1, 1,
           launch_convert<T>(p->coef, sizeof(T) == 8, coef, 1, 5 * P, p->stream));
  RET(read_scalars(p));
  if (scal) {
    const DevScalars* h = p->hsc;
    scal[0] = h->mean_fn;
    scal[1] = h->res_inf;
    scal[2] = sqrt(h->res_l2sum / (double)P);
    scal[3] = h->min_det;
    scal[4] = h->k1_nonfinite;
    for (int a = 0; a < 5; ++a) scal[5 + a] = h->abar[a];
  }
  return OT_OK;
}

extern "C" int ot_eval_residual(ot_plan* p, const double* f, const double* c, const double* u,
                                double* F, double* coef, double* scal) {
  if (!p || !f || !c || !u) return OT_EINVAL;
  CK(cudaSetDevice(p->device));
  return p->precision ? eval_residual_impl<float>(p, f, c, u, F, coef, scal)
                      : eval_residual_impl<double>(p, f, c, u, F, coef, scal);
}

static int upload_abar(ot_plan* p, const double* abar) {
  set_solver_scalars(p);
  for (int a = 0; a < 5; ++a) p->hsc->abar[a] = p->hsc->abar_n[a] = abar[a];
  CK(cudaMemcpyAsync(p->sc, p->hsc, sizeof(DevScalars), cudaMemcpyHostToDevice, p->stream));
  return OT_OK;
}

template <typename T>
static int apply_op_impl(ot_plan* p, const double* coef, const double* abar,
                         const double* sigma, double* w) {
  const long P = (long)p->N * p->M;
  int rc = upload_abar(p, abar);
  if (rc) return rc;
  CK(launch_convert<T>(coef, 1, p->coef, sizeof(T) == 8, 5 * P, p->stream));
  CK(launch_convert<T>(sigma, 1, p->sigma, sizeof(T) == 8, P, p->stream));
  RET(run_matvec<T>(p, (const T*)p->sigma, nullptr, nullptr, (T*)p->w, nullptr, -1));
  CK(launch_convert<T>(p->w, sizeof(T) == 8, w, 1, P, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return OT_OK;
}

extern "C" int ot_apply_operator(ot_plan* p, const double* coef, const double* abar,
                                 const double* sigma, double* w) {
  if (!p || !coef || !abar || !sigma || !w) return OT_EINVAL;
  CK(cudaSetDevice(p->device));
  return p->precision ? apply_op_impl<float>(p, coef, abar, sigma, w)
                      : apply_op_impl<double>(p, coef, abar, sigma, w);
}

template <typename T>
static int lbar_impl(ot_plan* p, const double* abar, const double* sigma, double* theta) {
  const long P = (long)p->N * p->M;
  int rc = upload_abar(p, abar);
  if (rc) return rc;
  CK(launch_convert<T>(sigma, 1, p->sigma, sizeof(T) == 8, P, p->stream));
  RET(run_lbar_inv<T>(p, (const T*)p->sigma, nullptr, nullptr, 0.0, (T*)p->w));
  CK(launch_convert<T>(p->w, sizeof(T) == 8, theta, 1, P, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return OT_OK;
}

extern "C" int ot_apply_lbar_inverse(ot_plan* p, const double* abar, const double* sigma,
                                     double* theta) {
  if (!p || !abar || !sigma || !theta) return OT_EINVAL;
  CK(cudaSetDevice(p->device));
  return p->precision ? lbar_impl<float>(p, abar, sigma, theta)
                      : lbar_impl<double>(p, abar, sigma, theta);
}

template <typename T>
static int fft_fwd_impl(ot_plan* p, const double* x, double* spec) {
  const long P = (long)p->N * p->M;
  const SpecTables& tb = tables<T>(p);
  CK(launch_convert<T>(x, 1, p->sigma, sizeof(T) == 8, P, p->stream));
  CK(launch_row_r2c<T>((const T*)p->sigma, 0, nullptr, nullptr, (C2<T>*)p->spec, p->N, p->M,
                       tb, nullptr, p->stream));
  CK(launch_col<T>(COL_FWD, (C2<T>*)p->spec, (C2<T>*)p->q0, nullptr, nullptr, p->N, p->M, tb,
                   nullptr, nullptr, p->stream));
  CK(launch_convert<T>(p->q0, sizeof(T) == 8, spec, 1, P, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return OT_OK;
}

template <typename T>
static int fft_inv_impl(ot_plan* p, const double* spec, double* x) {
  const long P = (long)p->N * p->M;
  const SpecTables& tb = tables<T>(p);
  CK(launch_convert<T>(spec, 1, p->spec, sizeof(T) == 8, P, p->stream));
  CK(launch_col<T>(COL_INV, (C2<T>*)p->spec, (C2<T>*)p->q0, nullptr, nullptr, p->N, p->M, tb,
                   nullptr, nullptr, p->stream));
  CK(launch_row_c2r<T>(ROWINV_PLAIN, (C2<T>*)p->q0, nullptr, nullptr, nullptr, (T*)p->w,
                       nullptr, nullptr, 0.0, 1.0, p->N, p->M, tb, nullptr, p->stream));
  CK(launch_convert<T>(p->w, sizeof(T) == 8, x, 1, P, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return OT_OK;
}

extern "C" int ot_fft_forward(ot_plan* p, const double* x, double* spec) {
  if (!p || !x || !spec) return OT_EINVAL;
  CK(cudaSetDevice(p->device));
  return p->precision ? fft_fwd_impl<float>(p, x, spec) : fft_fwd_impl<double>(p, x, spec);
}

extern "C" int ot_fft_inverse(ot_plan* p, const double* spec, double* x) {
  if (!p || !spec || !x) return OT_EINVAL;
  CK(cudaSetDevice(p->device));
  return p->precision ? fft_inv_impl<float>(p, spec, x) : fft_inv_impl<double>(p, spec, x);
}

// ------------------------------------------------------------------------------------------
// Learned warm start: entry points
// ------------------------------------------------------------------------------------------
extern "C" int64_t ot_ws_param_count(void) { return ws_param_count(); }

extern "C" int ot_ws_set_weights(ot_plan* p, const float* params_host, int64_t count) {
  if (!p || !p->ready || !params_host || count != ws_param_count()) return OT_EINVAL;
  CK(cudaSetDevice(p->device));
  if (!p->ws_params) CK(cudaMalloc(&p->ws_params, ws_param_count() * sizeof(float)));
  if (!p->ws_wpack) CK(cudaMalloc(&p->ws_wpack, ws_packed_bytes()));
  RET(alloc_ws(p));
  CK(cudaMemcpyAsync(p->ws_params, params_host, count * sizeof(float), cudaMemcpyHostToDevice,
                     p->stream));
  CK(launch_ws_pack(p->ws_params, p->ws_wpack, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  p->ws_have = 1;
  return OT_OK;
}

static const char kWsMagic[8] = {'O', 'T', 'W', 'S', '0', '0', '0', '1'};

extern "C" int ot_warmstart_load(ot_plan* p, const char* path) {
  if (!p || !path) return OT_EINVAL;
  FILE* fp = fopen(path, "rb");
  if (!fp) return OT_EINVAL;
  char magic[8];
  int64_t count = 0;
  std::vector<float> w;
  bool ok = fread(magic, 1, 8, fp) == 8 && memcmp(magic, kWsMagic, 8) == 0 &&
            fread(&count, sizeof(count), 1, fp) == 1 && count == ws_param_count();
  if (ok) {
    w.resize((size_t)count);
    ok = fread(w.data(), sizeof(float), (size_t)count, fp) == (size_t)count;
  }
  fclose(fp);
  if (!ok) return OT_EINVAL;
  return ot_ws_set_weights(p, w.data(), count);
}

extern "C" int ot_ws_save_weights(const char* path, const float* params_host, int64_t count) {
  if (!path || !params_host || count != ws_param_count()) return OT_EINVAL;
  FILE* fp = fopen(path, "wb");
  if (!fp) return OT_EINVAL;
  bool ok = fwrite(kWsMagic, 1, 8, fp) == 8 && fwrite(&count, sizeof(count), 1, fp) == 1 &&
            fwrite(params_host, sizeof(float), (size_t)count, fp) == (size_t)count;
  ok = (fclose(fp) == 0) && ok;
  return ok ? OT_OK : OT_EINVAL;
}

// translate (or copy) the inputs into the plan's f, g and prefilter g
static int ws_prepare_inputs(ot_plan* p, const double* f, const double* g) {
  const long P = (long)p->N * p->M;
  set_solver_scalars(p);
  CK(cudaMemcpyAsync(p->sc, p->hsc, sizeof(DevScalars), cudaMemcpyHostToDevice, p->stream));
  if (p->translate) {
    LAUNCH(p, OT_PROF_OTHER, -1, 2,
           launch_translate_inputs(f, g, p->f, p->g, p->N, p->M, p->partials, p->sc,
                                   p->stream));
    RET(read_scalars(p));
    if (p->hsc->in_bad) return OT_EINVAL;
  } else {
    CK(cudaMemcpyAsync(p->f, f, P * 8, cudaMemcpyDeviceToDevice, p->stream));
    CK(cudaMemcpyAsync(p->g, g, P * 8, cudaMemcpyDeviceToDevice, p->stream));
  }
  return run_prefilter(p, p->g, p->c);
}

extern "C" int ot_ws_predict(ot_plan* p, const double* f, const double* g, double* phi0,
                             double* alpha_out) {
  if (!p || !p->ready || !f || !g || !phi0 || !p->ws_have) return OT_EINVAL;
  CK(cudaSetDevice(p->device));
  RET(ws_prepare_inputs(p, f, g));
  RET(run_warmstart(p, phi0));
  RET(read_scalars(p));
  if (alpha_out) *alpha_out = p->hsc->ws_alpha;
  if (p->hsc->ws_err) {
    record_kernel_error("tensor-core network: bounded mbarrier wait ran out", __LINE__);
    return OT_ETIMEOUT;
  }
  return OT_OK;
}

extern "C" int ot_ws_features(ot_plan* p, const double* f, const double* g,
                              const double* phi_star, float* X, float* target) {
  if (!p || !p->ready || !f || !g || !X || (phi_star && !target)) return OT_EINVAL;
  CK(cudaSetDevice(p->device));
  const long P = (long)p->N * p->M;
  RET(ws_prepare_inputs(p, f, g));
  RET(run_ws_features(p));
  CK(cudaMemcpyAsync(X, p->ws_X, P * OTGB_WS_K * sizeof(float), cudaMemcpyDeviceToDevice,
                     p->stream));
  if (phi_star)
    LAUNCH(p, OT_PROF_WARMSTART, -1, 2,
           launch_ws_target(phi_star, p->ws_h, p->N, p->M, p->ws_tmp, target, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return OT_OK;
}

extern "C" int ot_ws_mlp_forward(ot_plan* p, const float* X, int64_t rows, float* out) {
  if (!p || !p->ready || !p->ws_have || rows < 0 || (rows > 0 && (!X || !out)))
    return OT_EINVAL;
  CK(cudaSetDevice(p->device));
  CK(cudaMemsetAsync(&p->sc->ws_err, 0, sizeof(int), p->stream));
  const int stall = p->ws_stall;
  p->ws_stall = 0;
  LAUNCH(p, OT_PROF_WARMSTART, -1, 1,
         launch_ws_mlp(p->ws_wpack, p->ws_params, X, rows, out, &p->sc->ws_err, p->sms,
                       p->stream, stall));
  int err = 0;
  CK(cudaMemcpyAsync(&err, &p->sc->ws_err, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  if (err) {
    record_kernel_error("tensor-core network: bounded mbarrier wait ran out", __LINE__);
    return OT_ETIMEOUT;
  }
  return OT_OK;
}

extern "C" int ot_transport_outputs(ot_plan* p, const double* f, const double* phi,
                                    double* dist, double* div_out) {
  if (!p || !p->ready || !f || !phi || !dist) return OT_EINVAL;
  CK(cudaSetDevice(p->device));
  LAUNCH(p, OT_PROF_OTHER, -1, 1,
         launch_transport(f, phi, p->N, p->M, div_out, p->partials,
                          &p->sc->ticket[TK_TRANSPORT], &p->sc->dist, p->stream));
  CK(cudaMemcpyAsync(dist, &p->sc->dist, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return OT_OK;
}

extern "C" int ot_ws_poisson(ot_plan* p, const double* src, int32_t lowpass, double* u) {
  if (!p || !p->ready || !src || !u) return OT_EINVAL;
  CK(cudaSetDevice(p->device));
  RET(alloc_ws(p));
  RET(run_ws_poisson(p, src, u, lowpass != 0));
  CK(cudaStreamSynchronize(p->stream));
  return OT_OK;
}

struct ot_ws_trainer {
  int B = 0, device = 0, t = 0;
  cudaStream_t stream = 0;
  float *params = nullptr, *m = nullptr, *v = nullptr;
  WsTrainBuffers b{};
  std::vector<void*> allocs;
};

extern "C" void ot_ws_trainer_destroy(ot_ws_trainer* tr) {
  if (!tr) return;
  cudaSetDevice(tr->device);
  for (void* q : tr->allocs) cudaFree(q);
  delete tr;
}

extern "C" int ot_ws_trainer_create(ot_ws_trainer** out, int32_t batch,
                                    const float* params_host, int64_t count) {
  if (!out) return OT_EINVAL;
  *out = nullptr;
  if (batch < 64 || batch > (1 << 20) || batch % 64 != 0 || !params_host ||
      count != ws_param_count())
    return OT_EINVAL;
  ot_ws_trainer* tr = new (std::nothrow) ot_ws_trainer();
  if (!tr) return OT_ENOMEM;
  tr->B = batch;
  cudaGetDevice(&tr->device);
  const long n = ws_param_count(), B = batch, H = OTGB_WS_H;
  const long S = (B + WS_ROW_CHUNK - 1) / WS_ROW_CHUNK;
  bool failed = false;
  auto get = [&](size_t bytes) -> void* {
    void* q = nullptr;
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
      failed = true;
      return nullptr;
    }
    tr->allocs.push_back(q);
    return q;
  };
  tr->params = (float*)get(n * 4);
  tr->m = (float*)get(n * 4);
  tr->v = (float*)get(n * 4);
  WsTrainBuffers& b = tr->b;
  b.grad = (float*)get(n * 4);
  b.Xb = (float*)get(B * OTGB_WS_K * 4);
  b.tb = (float*)get(B * 4);
  float** planes[] = {&b.Z0, &b.A0, &b.Z1, &b.A1, &b.Z2, &b.A2, &b.dZ1, &b.dZ2};
  for (float** q : planes) *q = (float*)get(B * H * 4);
  b.dy = (float*)get(B * 4);
  b.part = (float*)get(S * H * H * 4);
  b.loss_part = (double*)get(((B + 7) / 8) * 8);
  b.loss = (double*)get(8);
  if (failed) {
    cudaGetLastError();
    ot_ws_trainer_destroy(tr);
    return OT_ENOMEM;
  }
  if (cudaMemcpy(tr->params, params_host, n * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(tr->m, 0, n * 4) != cudaSuccess || cudaMemset(tr->v, 0, n * 4) != cudaSuccess) {
    ot_ws_trainer_destroy(tr);
    return OT_ECUDA;
  }
  *out = tr;
  return OT_OK;
}

extern "C" int ot_ws_trainer_set_stream(ot_ws_trainer* tr, void* s) {
  if (!tr) return OT_EINVAL;
  tr->stream = (cudaStream_t)s;
  return OT_OK;
}

extern "C" int ot_ws_trainer_grad(ot_ws_trainer* tr, const float* X, const float* t,
                                  const int64_t* idx, float* grad_host, double* loss_host) {
  if (!tr || !X || !t || !idx) return OT_EINVAL;
  CK(cudaSetDevice(tr->device));
  CK(launch_ws_grad(tr->params, X, t, (const long long*)idx, tr->B, tr->b, tr->stream));
  if (grad_host)
    CK(cudaMemcpyAsync(grad_host, tr->b.grad, ws_param_count() * 4, cudaMemcpyDeviceToHost,
                       tr->stream));
  if (loss_host)
    CK(cudaMemcpyAsync(loss_host, tr->b.loss, 8, cudaMemcpyDeviceToHost, tr->stream));
  CK(cudaStreamSynchronize(tr->stream));
  return OT_OK;
}

extern "C" int ot_ws_trainer_step(ot_ws_trainer* tr, const float* X, const float* t,
                                  const int64_t* idx, float lr, double* loss_host) {
  if (!tr || !X || !t || !idx || !(lr > 0.f)) return OT_EINVAL;
  CK(cudaSetDevice(tr->device));
  CK(launch_ws_grad(tr->params, X, t, (const long long*)idx, tr->B, tr->b, tr->stream));
  tr->t += 1;
  CK(launch_ws_adam(tr->params, tr->m, tr->v, tr->b.grad, ws_param_count(), lr, tr->t,
                    tr->stream));
  if (loss_host) {
    CK(cudaMemcpyAsync(loss_host, tr->b.loss, 8, cudaMemcpyDeviceToHost, tr->stream));
    CK(cudaStreamSynchronize(tr->stream));
  }
  return OT_OK;
}

extern "C" int ot_ws_trainer_get_params(ot_ws_trainer* tr, float* params_host, int64_t count) {
  if (!tr || !params_host || count != ws_param_count()) return OT_EINVAL;
  CK(cudaSetDevice(tr->device));
  CK(cudaMemcpyAsync(params_host, tr->params, count * 4, cudaMemcpyDeviceToHost, tr->stream));
  CK(cudaStreamSynchronize(tr->stream));
  return OT_OK;
}

// ------------------------------------------------------------------------------------------
// Plan sets: many problems of uneven sizes in one graph launch.  The problems are grouped
// into size classes; each class is a batched plan (every kernel of the mixed-precision solve
// serves all its pairs at once, gridDim.z = pairs, per-pair masks), and the whole solve of
// every class is one captured graph with one branch per class.
// ------------------------------------------------------------------------------------------
namespace {
struct BatchClass {
  int N = 0, M = 0;
  std::vector<int> idx;        // problem indices of this class
  ot_plan* p = nullptr;        // the batched plan
  double** dtab = nullptr;     // device pointer table: f[B], g[B], phi[B]
  double** htab = nullptr;     // pinned staging of the table
  DevScalars* hsc = nullptr;   // pinned: the pairs' scalars (initial, then final)
};
}  // namespace

struct ot_plan_set {
  int count = 0;
  std::vector<int> N, M;
  double tau = 1.0, tol = 1e-8;
  std::vector<std::pair<int, double>> opts;  // plan options, applied in order
  int tau_retry = 0;
  std::vector<BatchClass> cls;
  cudaStream_t stream = 0;
  cudaStream_t s0 = nullptr;  // origin of the capture
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int device = 0;
};

static void set_free_graph(ot_plan_set* s) {
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  if (s->graph) cudaGraphDestroy(s->graph);
  s->gexec = nullptr;
  s->graph = nullptr;
}

static void set_free_classes(ot_plan_set* s) {
  set_free_graph(s);
  for (auto& c : s->cls) {
    if (c.p) ot_plan_destroy(c.p);
    if (c.dtab) cudaFree(c.dtab);
    if (c.htab) cudaFreeHost(c.htab);
    if (c.hsc) cudaFreeHost(c.hsc);
    c.p = nullptr;
    c.dtab = nullptr;
    c.htab = nullptr;
    c.hsc = nullptr;
  }
}

extern "C" int ot_plan_set_create(ot_plan_set** out, int32_t count, const int32_t* N,
                                  const int32_t* M, double tau, double tol) {
  if (!out) return OT_EINVAL;
  *out = nullptr;
  if (count < 1 || !N || !M || !(tau >= 1.0) || !(tol > 0.0)) return OT_EINVAL;
  for (int k = 0; k < count; ++k)
    if (!size_supported(N[k], M[k])) return OT_EUNSUPPORTED;
  ot_plan_set* s = new (std::nothrow) ot_plan_set();
  if (!s) return OT_ENOMEM;
  s->count = count;
  s->N.assign(N, N + count);
  s->M.assign(M, M + count);
  s->tau = tau;
  s->tol = tol;
  for (int k = 0; k < count; ++k) {
    BatchClass* c = nullptr;
    for (auto& e : s->cls)
      if (e.N == N[k] && e.M == M[k]) c = &e;
    if (!c) {
      s->cls.emplace_back();
      c = &s->cls.back();
      c->N = N[k];
      c->M = M[k];
    }
    c->idx.push_back(k);
  }
  for (auto& c : s->cls)
    if (c.idx.size() > 1024) {
      delete s;
      return OT_EUNSUPPORTED;
    }
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return OT_ECUDA;
  }
  *out = s;
  return OT_OK;
}

extern "C" void ot_plan_set_destroy(ot_plan_set* s) {
  if (!s) return;
  cudaSetDevice(s->device);
  set_free_classes(s);
  if (s->s0) cudaStreamDestroy(s->s0);
  delete s;
}

extern "C" int ot_batch_set_stream(ot_plan_set* s, void* stream) {
  if (!s) return OT_EINVAL;
  s->stream = (cudaStream_t)stream;
  return OT_OK;
}

extern "C" int ot_batch_set_option(ot_plan_set* s, int32_t key, double v) {
  if (!s) return OT_EINVAL;
  switch (key) {
    case OT_OPT_PRECISION:  // the batched solve is the mixed-precision one
      return v == 1 ? OT_OK : OT_EINVAL;
    case OT_OPT_THETA_FP64:  // theta's inverse transforms in double-float
      return v == 2 ? OT_OK : OT_EINVAL;
    case OT_OPT_TAU_RETRY:
      if (!(v >= 0 && v <= 8) || v != (double)(int)v) return OT_EINVAL;
      s->tau_retry = (int)v;
      return OT_OK;
    case OT_OPT_TAU:
      if (!(v >= 1.0)) return OT_EINVAL;
      s->tau = v;
      break;
    case OT_OPT_TOL:
      if (!(v > 0.0)) return OT_EINVAL;
      s->tol = v;
      break;
    case OT_OPT_RESTART:
      if (!(v >= 1 && v <= OTGB_MAXM - 1) || v != (double)(int)v) return OT_EINVAL;
      set_free_classes(s);  // the basis size changes the slabs
      break;
    case OT_OPT_ETA:
      if (!(v > 0.0 && v < 1.0)) return OT_EINVAL;
      break;
    case OT_OPT_MAX_NEWTON:
    case OT_OPT_MAX_RESTARTS:
      if (v < (key == OT_OPT_MAX_NEWTON ? 0 : 1) || v != (double)(int)v) return OT_EINVAL;
      break;
    case OT_OPT_TAU_SWITCH:
      if (!(v >= 0.0)) return OT_EINVAL;
      break;
    case OT_OPT_SAFEGUARD:
    case OT_OPT_TRANSLATE:
    case OT_OPT_SYMBOLS:
    case OT_OPT_FORCING:
    case OT_OPT_OPERATOR:
    case OT_OPT_REORTH:
      if (v != 0 && v != 1) return OT_EINVAL;
      break;
    default:
      return OT_EINVAL;
  }
  s->opts.emplace_back(key, v);
  set_free_graph(s);
  for (auto& c : s->cls)
    if (c.p) RET(ot_plan_set_option(c.p, key, v));
  return OT_OK;
}

// Create the class plans (first use or after a basis-size change) and capture the graph: from
// the capture origin every class forks onto its plan's own stream, gathers its pairs' inputs
// from the pointer table, zeroes the iterates, runs the batched solve and scatters the
// potentials; the branches join at the end.
static int set_build(ot_plan_set* s) {
  for (auto& c : s->cls) {
    if (c.p) continue;
    const int B = (int)c.idx.size();
    RET(ot_plan_create(&c.p, c.N, c.M, s->tau, s->tol));
    RET(ot_plan_set_option(c.p, OT_OPT_PRECISION, 1));
    c.p->autotune = 0;  // the batched passes are the generic kernels
    for (auto& kv : s->opts)
      if (kv.first != OT_OPT_TAU && kv.first != OT_OPT_TOL)
        RET(ot_plan_set_option(c.p, kv.first, kv.second));
    RET(alloc_batch(c.p, B));
    CK(cudaMalloc(&c.dtab, 3 * (size_t)B * sizeof(double*)));
    CK(cudaMallocHost(&c.htab, 3 * (size_t)B * sizeof(double*)));
    CK(cudaMallocHost(&c.hsc, (size_t)B * sizeof(DevScalars)));
    for (int k = 0; k < 4; ++k)
      if (!c.p->cs[k]) CK(cudaStreamCreateWithFlags(&c.p->cs[k], cudaStreamNonBlocking));
  }
  if (s->gexec) return OT_OK;
  if (!s->s0) CK(cudaStreamCreateWithFlags(&s->s0, cudaStreamNonBlocking));
  cudaEvent_t fork = nullptr;
  CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  std::vector<cudaEvent_t> joins(s->cls.size(), nullptr);
  for (auto& e : joins) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  CK(cudaStreamBeginCapture(s->s0, cudaStreamCaptureModeRelaxed));
  int rc = OT_OK;
  cudaError_t e = cudaEventRecord(fork, s->s0);
  for (size_t ci = 0; ci < s->cls.size() && rc == OT_OK && e == cudaSuccess; ++ci) {
    BatchClass& c = s->cls[ci];
    ot_plan* p = c.p;
    const int B = (int)c.idx.size();
    const long P = (long)p->N * p->M;
    p->tau = s->tau;
    p->tol = s->tol;
    p->stream = p->cs[0];
    p->cur_mask = MASK_ALL;
    if ((e = cudaStreamWaitEvent(p->cs[0], fork, 0)) != cudaSuccess) break;
    if ((e = launch_gather(c.dtab, p->f, P, btc(p), p->stream)) != cudaSuccess) break;
    if ((e = launch_gather(c.dtab + B, p->g, P, btc(p), p->stream)) != cudaSuccess) break;
    if ((e = cudaMemset2DAsync(p->u, p->slab, 0, P * 8, B, p->stream)) != cudaSuccess) break;
    rc = capture_solve<float>(p);
    if (rc != OT_OK) break;
    p->cur_mask = MASK_ALL;
    if ((e = launch_scatter(p->uout, c.dtab + 2 * B, P, p->sc, btc(p), p->stream)) !=
        cudaSuccess)
      break;
    if ((e = cudaEventRecord(joins[ci], p->cs[0])) != cudaSuccess) break;
    if ((e = cudaStreamWaitEvent(s->s0, joins[ci], 0)) != cudaSuccess) break;
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(s->s0, &g);
  for (auto& c : s->cls)
    if (c.p) c.p->stream = s->stream;
  cudaEventDestroy(fork);
  for (auto& j : joins) cudaEventDestroy(j);
  if (rc != OT_OK || e != cudaSuccess || e2 != cudaSuccess) {
    if (e != cudaSuccess) record_error(e, __LINE__);
    for (auto& c : s->cls)
      if (c.p) abandon_captures(c.p);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc != OT_OK ? rc : OT_ECUDA;
  }
  s->graph = g;
  e = cudaGraphInstantiate(&s->gexec, g, 0);
  if (e != cudaSuccess) {
    record_error(e, __LINE__);
    set_free_graph(s);
    return OT_ECUDA;
  }
  return OT_OK;
}

// initial scalars of pair k of class c: those of a graph-launched solve with every Arnoldi
// step a plain launch, the pair's tau (doubled per retry) and whether it sits this launch out
static void set_pair_scalars(ot_plan* p, DevScalars* h, double tau, int excluded) {
  const double tau0 = p->tau;
  p->tau = tau;
  graph_scalars(p, h);
  p->tau = tau0;
  h->steps_uncond = p->m;
  h->cycle_done = 1;
  h->excluded = excluded;
}

extern "C" int ot_solve_batched(ot_plan_set* s, int32_t count, const int32_t* N,
                                const int32_t* M, const double* const* f,
                                const double* const* g, double* const* phi, ot_stats* stats) {
  if (!s || count != s->count || !N || !M || !f || !g || !phi) return OT_EINVAL;
  for (int k = 0; k < count; ++k)
    if (N[k] != s->N[k] || M[k] != s->M[k] || !f[k] || !g[k] || !phi[k]) return OT_EINVAL;
  CK(cudaSetDevice(s->device));
  RET(set_build(s));
  cudaStream_t st = s->stream;
  cudaEvent_t ev0, ev1;
  CK(cudaEventCreate(&ev0));
  CK(cudaEventCreate(&ev1));
  CK(cudaEventRecord(ev0, st));
  std::vector<double> tau(count, s->tau);
  std::vector<int> last_status(count, OT_OK), done(count, 0);
  std::vector<DevScalars> fin(count);
  for (auto& c : s->cls) {
    const int B = (int)c.idx.size();
    for (int k = 0; k < B; ++k) {
      c.htab[k] = const_cast<double*>(f[c.idx[k]]);
      c.htab[B + k] = const_cast<double*>(g[c.idx[k]]);
      c.htab[2 * B + k] = phi[c.idx[k]];
    }
    CK(cudaMemcpyAsync(c.dtab, c.htab, 3 * (size_t)B * sizeof(double*), cudaMemcpyHostToDevice,
                       st));
  }
  // attempt 0 solves every pair; each further attempt (OT_OPT_TAU_RETRY) solves again, with
  // twice the tau, only the pairs whose last attempt lost convexity (the others sit it out)
  for (int attempt = 0; attempt <= s->tau_retry; ++attempt) {
    bool any = false;
    for (auto& c : s->cls) {
      const int B = (int)c.idx.size();
      for (int k = 0; k < B; ++k) {
        const int q = c.idx[k];
        const int run = attempt == 0 || (!done[q] && last_status[q] == OT_EDIVERGED);
        if (attempt > 0 && run) tau[q] *= 2.0;
        set_pair_scalars(c.p, &c.hsc[k], tau[q], run ? 0 : 1);
        any |= run != 0;
      }
      CK(cudaMemcpy2DAsync(c.p->sc, c.p->slab, c.hsc, sizeof(DevScalars), sizeof(DevScalars), B,
                           cudaMemcpyHostToDevice, st));
    }
    if (!any) break;
    CK(cudaGraphLaunch(s->gexec, st));
    for (auto& c : s->cls)
      CK(cudaMemcpy2DAsync(c.hsc, sizeof(DevScalars), c.p->sc, c.p->slab, sizeof(DevScalars),
                           c.idx.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (auto& c : s->cls)
      for (size_t k = 0; k < c.idx.size(); ++k) {
        if (c.hsc[k].excluded) continue;
        const int q = c.idx[k];
        fin[q] = c.hsc[k];
        last_status[q] = c.hsc[k].status;
        if (c.hsc[k].status != OT_EDIVERGED) done[q] = 1;
      }
  }
  CK(cudaEventRecord(ev1, st));
  CK(cudaEventSynchronize(ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  int first = OT_OK;
  for (auto& c : s->cls)
    for (size_t k = 0; k < c.idx.size(); ++k) {
      const int q = c.idx[k];
      const DevScalars& h = fin[q];
      if (h.status != OT_OK && first == OT_OK) first = h.status;
      if (!stats) continue;
      ot_stats& o = stats[q];
      memset(&o, 0, sizeof(o));
      o.status = h.status;
      o.newton_iters = h.newton_n;
      o.gmres_iters = h.gmres_iters_total;
      o.gmres_cycles = h.gmres_cycles_total;
      o.step_halvings = h.halvings;
      o.kernel_launches = (int32_t)(c.hsc[0].kcount + c.p->top_kernels);
      o.res_inf = h.res_inf;
      o.res_l2 = sqrt(h.res_l2sum / ((double)c.N * (double)c.M));
      o.min_det = h.min_det;
      o.mean_fn = h.mean_fn;
      o.phi_mean = h.gauge_mean;
      o.ms_total = ms;
      o.ws_alpha = -1.0;
      o.mass_defect_f = h.in_mean[0] - 1.0;
      o.mass_defect_g = h.in_mean[1] - 1.0;
      o.transport_dist = -1.0;
      o.ms_residual = o.ms_fft = o.ms_krylov = o.ms_update = o.ms_other = -1.0;
    }
  return first;
}

// ------------------------------------------------------------------------------------------
// Spectral radius of the inverse of the discretised linearised operator (Sec. 5.1): power
// iteration b_(k+1) = A^{-1} b_k / ||A^{-1} b_k||_2, A^{-1} b = Lbar^{-1} sigma with sigma
// from GMRES(m) on L Lbar^{-1} sigma = b (the Fourier method of Sec. 4.2 at the plan's eta),
// L the linearisation at the iterate phi; b_0 projected to mean zero (the operator acts on
// mean-zero potentials, Sec. 3.1).  Host-driven: one synchronisation per GMRES cycle and per
// iteration.
// ------------------------------------------------------------------------------------------
template <typename T>
static int inverse_radius_impl(ot_plan* p, const double* f, const double* g, const double* phi,
                               const double* b0, int iters, double* rho) {
  const int N = p->N, M = p->M;
  const long P = (long)N * M;
  RET(run_autotune(p));
  set_solver_scalars(p);
  p->hsc->forcing = 0;
  CK(cudaMemcpyAsync(p->sc, p->hsc, sizeof(DevScalars), cudaMemcpyHostToDevice, p->stream));
  if (p->translate) {
    LAUNCH(p, OT_PROF_OTHER, -1, 2,
           launch_translate_inputs(f, g, p->f, p->g, N, M, p->partials, p->sc, p->stream));
  } else {
    CK(cudaMemcpyAsync(p->f, f, P * 8, cudaMemcpyDeviceToDevice, p->stream));
    CK(cudaMemcpyAsync(p->g, g, P * 8, cudaMemcpyDeviceToDevice, p->stream));
    LAUNCH(p, OT_PROF_OTHER, -1, 1,
           launch_input_stats(p->f, p->g, N, M, p->partials, p->sc, p->stream));
  }
  RET(read_scalars(p));
  if (p->hsc->in_bad) return OT_EINVAL;
  RET(run_prefilter(p, p->g, p->c));
  CK(cudaMemcpyAsync(p->u, phi, P * 8, cudaMemcpyDeviceToDevice, p->stream));
  LAUNCH(p, OT_PROF_RESIDUAL, -1, 1,
         residual_launch<T>(p, p->f, p->c, p->u, p->Fraw, nullptr, 0));
  double* b = p->ucand;
  double* th = p->uout;
  CK(cudaMemcpyAsync(b, b0, P * 8, cudaMemcpyDeviceToDevice, p->stream));
  LAUNCH(p, OT_PROF_OTHER, -1, 2,
         launch_subtract_mean(b, N, M, p->partials, p->sc, p->dmean, p->stream));
  LAUNCH(p, OT_PROF_OTHER, -1, 2, launch_normalize(b, P, p->partials, p->sc, p->stream));
  static const double zero = 0.0, one = 1.0;
  for (int k = 0; k < iters; ++k) {
    // right-hand side b: the GMRES start reads (Fraw + shift) / tau
    CK(cudaMemcpyAsync(p->Fraw, b, P * 8, cudaMemcpyDeviceToDevice, p->stream));
    CK(cudaMemcpyAsync(&p->sc->shift, &zero, sizeof(double), cudaMemcpyHostToDevice,
                       p->stream));
    CK(cudaMemcpyAsync(&p->sc->tau, &one, sizeof(double), cudaMemcpyHostToDevice, p->stream));
    RET(run_gmres<T>(p));
    if (sizeof(T) == 4) {
      // theta in double-float from the FP32 sigma (the solve's theta passes)
      LAUNCH(p, OT_PROF_ROW_R2C, -1, 1,
             launch_row_r2c<float>((const float*)p->sigma, 0, nullptr, nullptr,
                                   (C2<float>*)p->spec, N, M, p->tb32, nullptr, p->stream));
      LAUNCH(p, OT_PROF_COL_LBARINV, -1, 1,
             launch_col_lbarinv_dd((const float2*)p->spec, (ddc*)p->q64, N, M, p->tb32,
                                   p->tbdd, p->sc, p->stream));
      LAUNCH(p, OT_PROF_ROW_C2R_UPDATE, -1, 1,
             launch_row_c2r_update_dd((const ddc*)p->q64, nullptr, th, 1.0, N, M, p->tbdd,
                                      nullptr, p->stream));
    } else {
      RET(run_lbar_inv<double>(p, (const double*)p->sigma, nullptr, nullptr, 0.0, th));
    }
    LAUNCH(p, OT_PROF_OTHER, -1, 2, launch_normalize(th, P, p->partials, p->sc, p->stream));
    RET(read_scalars(p));
    rho[k] = p->hsc->pw_norm;
    std::swap(b, th);
  }
  return OT_OK;
}

// ---- finite-difference comparison path (Sec. 4.1), step level ---------------------------
extern "C" int ot_fd_apply(ot_plan* p, const double* coef, const double* x, int32_t transpose,
                           double* y) {
  if (!p || !p->ready || !coef || !x || !y || (transpose != 0 && transpose != 1))
    return OT_EINVAL;
  if (!p->fdv) return OT_EINVAL;  // OT_OPT_LINEAR_SOLVER = 1 allocates the vectors
  CK(cudaSetDevice(p->device));
  CK(cudaMemsetAsync(&p->sc->bicg_done, 0, sizeof(int), p->stream));
  CK(cudaMemsetAsync(&p->sc->bicg_rho, 0, sizeof(double), p->stream));
  CK(launch_fd_apply(coef, x, transpose, y, fdbufs(p).q, p->N, p->M, p->partials, p->sc,
                     p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return OT_OK;
}

extern "C" int ot_fd_bicg(ot_plan* p, const double* coef, const double* h, double eta,
                          int32_t max_iters, double* theta, int32_t* iters, double* relres) {
  if (!p || !p->ready || !coef || !h || !theta || !(eta >= 0.0) || max_iters < 1)
    return OT_EINVAL;
  if (!p->fdv) return OT_EINVAL;
  CK(cudaSetDevice(p->device));
  const long P = (long)p->N * p->M;
  // the plan's coefficient planes and eta are the solve's: stage them
  CK(cudaMemcpyAsync(p->coef, coef, 5 * P * sizeof(double), cudaMemcpyDeviceToDevice,
                     p->stream));
  CK(cudaMemcpyAsync(&p->sc->eta, &eta, sizeof(double), cudaMemcpyHostToDevice, p->stream));
  const int keep = p->max_bicg;
  p->max_bicg = max_iters;
  const int rc = run_bicg(p, h);
  p->max_bicg = keep;
  RET(rc);
  CK(cudaMemcpyAsync(theta, fdbufs(p).x, P * sizeof(double), cudaMemcpyDeviceToDevice,
                     p->stream));
  RET(read_scalars(p));
  const DevScalars* hs = p->hsc;
  if (iters) *iters = hs->bicg_iters;
  if (relres) *relres = hs->bicg_b2 > 0.0 ? sqrt(hs->bicg_r2 / hs->bicg_b2) : 0.0;
  return hs->bicg_status == 0 ? OT_OK : (hs->bicg_status == 1 ? OT_ENOCONV : OT_EDIVERGED);
}

extern "C" int ot_inverse_spectral_radius(ot_plan* p, const double* f, const double* g,
                                          const double* phi, const double* b0, int32_t iters,
                                          double* rho) {
  if (!p || !p->ready || p->slab_base || !f || !g || !phi || !b0 || !rho || iters < 1)
    return OT_EINVAL;
  CK(cudaSetDevice(p->device));
  return p->precision ? inverse_radius_impl<float>(p, f, g, phi, b0, iters, rho)
                      : inverse_radius_impl<double>(p, f, g, phi, b0, iters, rho);
}
