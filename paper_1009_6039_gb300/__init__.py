"""Python binding of libotgb, a GB300 (sm_103a) solver for periodic L2 optimal transport by
the damped-Newton Monge-Ampere method of Saumier, Agueh & Khouider (arXiv:1009.6039).

The functions named ``ot_*`` are thin ctypes wrappers with the same names and arguments as
the C ABI in ``include/otgb.h`` (argument marshalling only; every step runs in the CUDA
kernels of ``libotgb.so``).  ``Plan`` and ``solve`` are conveniences over them that take
torch CUDA tensors (float64, shape (N, M), row index = y, column index = x).

Importing this module loads the library and raises if it is missing: there is no CPU
fallback.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libotgb.so")

OT_OK, OT_EINVAL, OT_ENOCONV, OT_EDIVERGED, OT_ECUDA, OT_ENOMEM, OT_EUNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6
OT_ETIMEOUT = -7
OT_OPT_RESTART, OT_OPT_ETA, OT_OPT_MAX_NEWTON, OT_OPT_MAX_RESTARTS = 1, 2, 3, 4
OT_OPT_PRECISION, OT_OPT_SAFEGUARD, OT_OPT_TRANSLATE, OT_OPT_WARM_START = 5, 6, 7, 8
OT_OPT_TAU, OT_OPT_TOL, OT_OPT_PROFILE, OT_OPT_GRAPH, OT_OPT_REORTH = 9, 10, 11, 12, 13
OT_OPT_THETA_FP64, OT_OPT_AUTOTUNE, OT_OPT_FFT_VARIANT, OT_OPT_SYMBOLS = 14, 15, 16, 17
OT_OPT_FORCING, OT_OPT_TAU_RETRY, OT_OPT_WS_TEST_STALL, OT_OPT_OPERATOR = 18, 19, 20, 21
OT_OPT_PHASE_TIMES, OT_OPT_TRANSPORT, OT_OPT_TAU_SWITCH, OT_OPT_INTERP = 22, 23, 24, 25
OT_OPT_LINEAR_SOLVER, OT_OPT_MAX_BICG, OT_OPT_UNCOND_STEPS = 26, 27, 28
OT_OPT_KRYLOV_BLOCKS, OT_OPT_L2_PERSIST, OT_OPT_FUSED_UPDATE = 29, 30, 31
OT_OPT_THETA_PAIRS = 32
PROF_CLASSES = ["residual", "row_r2c", "col_matvec", "row_c2r_combine", "col_lbarinv",
                "row_c2r_update", "gmres_dots", "gmres_update", "gmres_other", "other",
                "warmstart"]
OT_TIME_WS_NETWORK = 32  # ot_plan_time_kernel only: the warm start's network kernel

EXPORTS = ["ot_plan_create", "ot_plan_set_option", "ot_plan_get_option", "ot_plan_set_stream",
           "ot_solve", "ot_solve_host", "ot_solve_batched", "ot_plan_destroy", "ot_strerror",
           "ot_prefilter", "ot_eval_residual", "ot_apply_operator", "ot_apply_lbar_inverse",
           "ot_fft_forward", "ot_fft_inverse", "ot_plan_get_profile",
           "ot_plan_reset_profile", "ot_plan_time_kernel", "ot_eval_residual_noalloc",
           "ot_last_error", "ot_ws_param_count", "ot_ws_set_weights", "ot_warmstart_load",
           "ot_ws_save_weights", "ot_ws_predict", "ot_ws_features", "ot_ws_mlp_forward",
           "ot_ws_poisson", "ot_transport_outputs", "ot_ws_trainer_create", "ot_ws_trainer_set_stream",
           "ot_ws_trainer_grad", "ot_ws_trainer_step", "ot_ws_trainer_get_params",
           "ot_ws_trainer_destroy", "ot_solve_plans", "ot_plan_set_create",
           "ot_batch_set_option", "ot_batch_set_stream", "ot_plan_set_destroy",
           "ot_inverse_spectral_radius", "ot_fd_apply", "ot_fd_bicg"]


class ot_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("newton_iters", ctypes.c_int32),
                ("gmres_iters", ctypes.c_int32), ("gmres_cycles", ctypes.c_int32),
                ("step_halvings", ctypes.c_int32), ("kernel_launches", ctypes.c_int32),
                ("res_inf", ctypes.c_double), ("res_l2", ctypes.c_double),
                ("min_det", ctypes.c_double), ("mean_fn", ctypes.c_double),
                ("phi_mean", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("ws_alpha", ctypes.c_double), ("mass_defect_f", ctypes.c_double),
                ("mass_defect_g", ctypes.c_double), ("transport_dist", ctypes.c_double),
                ("ms_residual", ctypes.c_double), ("ms_fft", ctypes.c_double),
                ("ms_krylov", ctypes.c_double), ("ms_update", ctypes.c_double),
                ("ms_other", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class OTError(RuntimeError):
    def __init__(self, status, where):
        detail = ot_last_error() if status in (OT_ECUDA, OT_ETIMEOUT) else ""
        super().__init__("%s: %s (%d) %s" % (where, ot_strerror(status), status, detail))
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libotgb.so is not built (run __graft_entry__.build() or "
                          "python -m paper_1009_6039_gb300.build)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    sig = {
        "ot_plan_create": ([ctypes.POINTER(vp), i32, i32, d, d], ctypes.c_int),
        "ot_plan_set_option": ([vp, i32, d], ctypes.c_int),
        "ot_plan_get_option": ([vp, i32, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "ot_plan_set_stream": ([vp, vp], ctypes.c_int),
        "ot_solve": ([vp, vp, vp, vp, ctypes.POINTER(ot_stats)], ctypes.c_int),
        "ot_solve_host": ([vp, vp, vp, vp, ctypes.POINTER(ot_stats)], ctypes.c_int),
        "ot_solve_plans": ([i32, vp, vp, vp, vp, vp], ctypes.c_int),
        "ot_solve_batched": ([vp, i32, vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "ot_plan_set_create": ([ctypes.POINTER(vp), i32, vp, vp, d, d], ctypes.c_int),
        "ot_batch_set_option": ([vp, i32, d], ctypes.c_int),
        "ot_batch_set_stream": ([vp, vp], ctypes.c_int),
        "ot_plan_set_destroy": ([vp], None),
        "ot_inverse_spectral_radius": ([vp, vp, vp, vp, vp, i32, vp], ctypes.c_int),
        "ot_fd_apply": ([vp, vp, vp, i32, vp], ctypes.c_int),
        "ot_fd_bicg": ([vp, vp, vp, d, i32, vp, vp, vp], ctypes.c_int),
        "ot_plan_destroy": ([vp], None),
        "ot_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "ot_prefilter": ([vp, vp, vp], ctypes.c_int),
        "ot_eval_residual": ([vp, vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "ot_apply_operator": ([vp, vp, vp, vp, vp], ctypes.c_int),
        "ot_apply_lbar_inverse": ([vp, vp, vp, vp], ctypes.c_int),
        "ot_fft_forward": ([vp, vp, vp], ctypes.c_int),
        "ot_fft_inverse": ([vp, vp, vp], ctypes.c_int),
        "ot_plan_get_profile": ([vp, vp, vp, i32, vp], ctypes.c_int),
        "ot_plan_reset_profile": ([vp], ctypes.c_int),
        "ot_plan_time_kernel": ([vp, i32, i32, vp], ctypes.c_int),
        "ot_eval_residual_noalloc": ([i32, i32, vp, vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "ot_last_error": ([], ctypes.c_char_p),
        "ot_ws_param_count": ([], ctypes.c_int64),
        "ot_ws_set_weights": ([vp, vp, ctypes.c_int64], ctypes.c_int),
        "ot_warmstart_load": ([vp, ctypes.c_char_p], ctypes.c_int),
        "ot_ws_save_weights": ([ctypes.c_char_p, vp, ctypes.c_int64], ctypes.c_int),
        "ot_ws_predict": ([vp, vp, vp, vp, vp], ctypes.c_int),
        "ot_ws_features": ([vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "ot_ws_mlp_forward": ([vp, vp, ctypes.c_int64, vp], ctypes.c_int),
        "ot_ws_poisson": ([vp, vp, i32, vp], ctypes.c_int),
        "ot_transport_outputs": ([vp, vp, vp, ctypes.POINTER(ctypes.c_double), vp], ctypes.c_int),
        "ot_ws_trainer_create": ([ctypes.POINTER(vp), i32, vp, ctypes.c_int64], ctypes.c_int),
        "ot_ws_trainer_set_stream": ([vp, vp], ctypes.c_int),
        "ot_ws_trainer_grad": ([vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "ot_ws_trainer_step": ([vp, vp, vp, vp, ctypes.c_float, vp], ctypes.c_int),
        "ot_ws_trainer_get_params": ([vp, vp, ctypes.c_int64], ctypes.c_int),
        "ot_ws_trainer_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()


# ---- C ABI, same names ----------------------------------------------------------------
def ot_plan_create(N, M, tau, tol):
    h = ctypes.c_void_p()
    rc = _lib.ot_plan_create(ctypes.byref(h), int(N), int(M), float(tau), float(tol))
    return rc, h


def ot_plan_set_option(plan, key, value):
    return _lib.ot_plan_set_option(plan, int(key), float(value))


def ot_plan_get_option(plan, key, value_ptr):
    return _lib.ot_plan_get_option(plan, int(key), value_ptr)


def ot_plan_set_stream(plan, stream_ptr):
    return _lib.ot_plan_set_stream(plan, ctypes.c_void_p(stream_ptr))


def ot_solve(plan, f_ptr, g_ptr, phi_ptr, stats=None):
    return _lib.ot_solve(plan, f_ptr, g_ptr, phi_ptr,
                         ctypes.byref(stats) if stats is not None else None)


def ot_solve_host(plan, f_ptr, g_ptr, phi_ptr, stats=None):
    return _lib.ot_solve_host(plan, f_ptr, g_ptr, phi_ptr,
                              ctypes.byref(stats) if stats is not None else None)


def ot_solve_plans(count, plans, f_ptrs, g_ptrs, phi_ptrs, stats=None):
    arr = ctypes.c_void_p * count
    return _lib.ot_solve_plans(int(count), arr(*[p.value for p in plans]), arr(*f_ptrs),
                               arr(*g_ptrs), arr(*phi_ptrs),
                               ctypes.cast(stats, ctypes.c_void_p) if stats is not None
                               else None)


def ot_plan_set_create(count, N, M, tau, tol):
    h = ctypes.c_void_p()
    ai = ctypes.c_int32 * count
    rc = _lib.ot_plan_set_create(ctypes.byref(h), int(count), ai(*N), ai(*M), float(tau),
                                 float(tol))
    return rc, h


def ot_batch_set_option(pset, key, value):
    return _lib.ot_batch_set_option(pset, int(key), float(value))


def ot_batch_set_stream(pset, stream_ptr):
    return _lib.ot_batch_set_stream(pset, ctypes.c_void_p(stream_ptr))


def ot_solve_batched(pset, count, N, M, f_ptrs, g_ptrs, phi_ptrs, stats=None):
    ai = ctypes.c_int32 * count
    arr = ctypes.c_void_p * count
    return _lib.ot_solve_batched(pset, int(count), ai(*N), ai(*M), arr(*f_ptrs), arr(*g_ptrs),
                                 arr(*phi_ptrs),
                                 ctypes.cast(stats, ctypes.c_void_p) if stats is not None
                                 else None)


def ot_plan_set_destroy(pset):
    _lib.ot_plan_set_destroy(pset)


def ot_inverse_spectral_radius(plan, f_ptr, g_ptr, phi_ptr, b0_ptr, iters, rho_host_ptr):
    return _lib.ot_inverse_spectral_radius(plan, f_ptr, g_ptr, phi_ptr, b0_ptr, int(iters),
                                           rho_host_ptr)


def ot_fd_apply(plan, coef_ptr, x_ptr, transpose, y_ptr):
    return _lib.ot_fd_apply(plan, coef_ptr, x_ptr, int(transpose), y_ptr)


def ot_fd_bicg(plan, coef_ptr, h_ptr, eta, max_iters, theta_ptr, iters_host_ptr,
               relres_host_ptr):
    return _lib.ot_fd_bicg(plan, coef_ptr, h_ptr, float(eta), int(max_iters), theta_ptr,
                           iters_host_ptr, relres_host_ptr)


def ot_plan_destroy(plan):
    _lib.ot_plan_destroy(plan)


def ot_strerror(status):
    return _lib.ot_strerror(int(status)).decode()


def ot_last_error():
    return _lib.ot_last_error().decode()


def ot_prefilter(plan, g_ptr, c_ptr):
    return _lib.ot_prefilter(plan, g_ptr, c_ptr)


def ot_eval_residual(plan, f_ptr, c_ptr, u_ptr, F_ptr, coef_ptr, scal_host_ptr):
    return _lib.ot_eval_residual(plan, f_ptr, c_ptr, u_ptr, F_ptr, coef_ptr, scal_host_ptr)


def ot_apply_operator(plan, coef_ptr, abar_host_ptr, sigma_ptr, w_ptr):
    return _lib.ot_apply_operator(plan, coef_ptr, abar_host_ptr, sigma_ptr, w_ptr)


def ot_apply_lbar_inverse(plan, abar_host_ptr, sigma_ptr, theta_ptr):
    return _lib.ot_apply_lbar_inverse(plan, abar_host_ptr, sigma_ptr, theta_ptr)


def ot_fft_forward(plan, x_ptr, spec_ptr):
    return _lib.ot_fft_forward(plan, x_ptr, spec_ptr)


def ot_fft_inverse(plan, spec_ptr, x_ptr):
    return _lib.ot_fft_inverse(plan, spec_ptr, x_ptr)


def ot_plan_get_profile(plan, ms_ptr, launches_ptr, n, total_ptr):
    return _lib.ot_plan_get_profile(plan, ms_ptr, launches_ptr, int(n), total_ptr)


def ot_plan_reset_profile(plan):
    return _lib.ot_plan_reset_profile(plan)


def ot_eval_residual_noalloc(N, M, f_ptr, c_ptr, u_ptr, F_ptr, coef_ptr, scal_host_ptr,
                             stream_ptr=0):
    """Allocation-free residual evaluation (no plan; fixed device scratch, N, M <= 2048)."""
    return _lib.ot_eval_residual_noalloc(int(N), int(M), f_ptr, c_ptr, u_ptr, F_ptr, coef_ptr,
                                         scal_host_ptr, ctypes.c_void_p(stream_ptr))


def ot_plan_time_kernel(plan, kernel_class, reps, ms_ptr):
    return _lib.ot_plan_time_kernel(plan, int(kernel_class), int(reps), ms_ptr)


def ot_ws_param_count():
    return int(_lib.ot_ws_param_count())


def ot_ws_set_weights(plan, params_host_ptr, count):
    return _lib.ot_ws_set_weights(plan, params_host_ptr, int(count))


def ot_warmstart_load(plan, path):
    return _lib.ot_warmstart_load(plan, os.fsencode(path))


def ot_ws_save_weights(path, params_host_ptr, count):
    return _lib.ot_ws_save_weights(os.fsencode(path), params_host_ptr, int(count))


def ot_ws_predict(plan, f_ptr, g_ptr, phi0_ptr, alpha_host_ptr=None):
    return _lib.ot_ws_predict(plan, f_ptr, g_ptr, phi0_ptr, alpha_host_ptr)


def ot_ws_features(plan, f_ptr, g_ptr, phi_star_ptr, X_ptr, target_ptr):
    return _lib.ot_ws_features(plan, f_ptr, g_ptr, phi_star_ptr, X_ptr, target_ptr)


def ot_ws_mlp_forward(plan, X_ptr, rows, out_ptr):
    return _lib.ot_ws_mlp_forward(plan, X_ptr, int(rows), out_ptr)


def ot_transport_outputs(plan, f_ptr, phi_ptr, dist_ptr, div_ptr=None):
    return _lib.ot_transport_outputs(plan, f_ptr, phi_ptr, dist_ptr, div_ptr)


def ot_ws_poisson(plan, src_ptr, lowpass, u_ptr):
    return _lib.ot_ws_poisson(plan, src_ptr, int(lowpass), u_ptr)


def ot_ws_trainer_create(batch, params_host_ptr, count):
    h = ctypes.c_void_p()
    rc = _lib.ot_ws_trainer_create(ctypes.byref(h), int(batch), params_host_ptr, int(count))
    return rc, h


def ot_ws_trainer_set_stream(tr, stream_ptr):
    return _lib.ot_ws_trainer_set_stream(tr, ctypes.c_void_p(stream_ptr))


def ot_ws_trainer_grad(tr, X_ptr, t_ptr, idx_ptr, grad_host_ptr, loss_host_ptr):
    return _lib.ot_ws_trainer_grad(tr, X_ptr, t_ptr, idx_ptr, grad_host_ptr, loss_host_ptr)


def ot_ws_trainer_step(tr, X_ptr, t_ptr, idx_ptr, lr, loss_host_ptr=None):
    return _lib.ot_ws_trainer_step(tr, X_ptr, t_ptr, idx_ptr, float(lr), loss_host_ptr)


def ot_ws_trainer_get_params(tr, params_host_ptr, count):
    return _lib.ot_ws_trainer_get_params(tr, params_host_ptr, int(count))


def ot_ws_trainer_destroy(tr):
    _lib.ot_ws_trainer_destroy(tr)


# ---- conveniences over torch tensors ---------------------------------------------------
def _check(rc, where, ok=(OT_OK,)):
    if rc not in ok:
        raise OTError(rc, where)
    return rc


def _dev(t, shape=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("expected shape %s, got %s" % (shape, tuple(t.shape)))
    return ctypes.c_void_p(t.data_ptr())


def _dev32(t, shape):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous() and tuple(t.shape) == tuple(shape)):
        raise TypeError("expected a contiguous float32 CUDA tensor of shape %s" % (shape,))
    return ctypes.c_void_p(t.data_ptr())


class Trainer:
    """Adam trainer of the warm-start network (ot_ws_trainer) over minibatches of `batch`
    rows of device tensors X (rows x 16, float32) and t (rows, float32)."""

    def __init__(self, batch, params, stream=None):
        import numpy as np
        a = np.ascontiguousarray(params, dtype=np.float32)
        rc, h = ot_ws_trainer_create(batch, ctypes.c_void_p(a.ctypes.data), a.size)
        _check(rc, "ot_ws_trainer_create")
        self.h, self.batch = h, batch
        if stream is not None:
            _check(ot_ws_trainer_set_stream(h, stream.cuda_stream if hasattr(stream, "cuda_stream")
                                            else int(stream)), "ot_ws_trainer_set_stream")

    @staticmethod
    def _idx(idx, batch):
        import torch
        if not (isinstance(idx, torch.Tensor) and idx.is_cuda and idx.dtype == torch.int64
                and idx.is_contiguous() and idx.numel() == batch):
            raise TypeError("expected %d int64 CUDA row indices" % batch)
        return ctypes.c_void_p(idx.data_ptr())

    def grad(self, X, t, idx):
        import numpy as np
        g = np.empty(ot_ws_param_count(), dtype=np.float32)
        loss = ctypes.c_double()
        _check(ot_ws_trainer_grad(self.h, _dev32(X, (X.shape[0], 16)), _dev32(t, (t.shape[0],)),
                                  self._idx(idx, self.batch), ctypes.c_void_p(g.ctypes.data),
                                  ctypes.byref(loss)), "ot_ws_trainer_grad")
        return loss.value, g

    def step(self, X, t, idx, lr, want_loss=False):
        loss = ctypes.c_double()
        _check(ot_ws_trainer_step(self.h, _dev32(X, (X.shape[0], 16)), _dev32(t, (t.shape[0],)),
                                  self._idx(idx, self.batch), lr,
                                  ctypes.byref(loss) if want_loss else None),
               "ot_ws_trainer_step")
        return loss.value if want_loss else None

    def params(self):
        import numpy as np
        p = np.empty(ot_ws_param_count(), dtype=np.float32)
        _check(ot_ws_trainer_get_params(self.h, ctypes.c_void_p(p.ctypes.data), p.size),
               "ot_ws_trainer_get_params")
        return p

    def close(self):
        if self.h:
            ot_ws_trainer_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """An ot_plan for N x M grids; options as keyword arguments
    (restart, eta, max_newton, max_restarts, precision ('fp64'|'mixed'), safeguard,
    translate, warm_start)."""

    _keys = {"restart": OT_OPT_RESTART, "eta": OT_OPT_ETA, "max_newton": OT_OPT_MAX_NEWTON,
             "max_restarts": OT_OPT_MAX_RESTARTS, "precision": OT_OPT_PRECISION,
             "safeguard": OT_OPT_SAFEGUARD, "translate": OT_OPT_TRANSLATE,
             "warm_start": OT_OPT_WARM_START, "tau": OT_OPT_TAU, "tol": OT_OPT_TOL,
             "profile": OT_OPT_PROFILE, "graph": OT_OPT_GRAPH, "reorth": OT_OPT_REORTH,
             "theta_fp64": OT_OPT_THETA_FP64, "autotune": OT_OPT_AUTOTUNE,
             "fft_variant": OT_OPT_FFT_VARIANT, "symbols": OT_OPT_SYMBOLS,
             "forcing": OT_OPT_FORCING, "tau_retry": OT_OPT_TAU_RETRY,
             "ws_test_stall": OT_OPT_WS_TEST_STALL, "operator": OT_OPT_OPERATOR,
             "phase_times": OT_OPT_PHASE_TIMES, "transport": OT_OPT_TRANSPORT,
             "tau_switch": OT_OPT_TAU_SWITCH, "interp": OT_OPT_INTERP,
             "linear_solver": OT_OPT_LINEAR_SOLVER, "max_bicg": OT_OPT_MAX_BICG,
             "uncond_steps": OT_OPT_UNCOND_STEPS, "krylov_blocks": OT_OPT_KRYLOV_BLOCKS,
             "l2_persist": OT_OPT_L2_PERSIST, "fused_update": OT_OPT_FUSED_UPDATE,
             "theta_pairs": OT_OPT_THETA_PAIRS}

    def __init__(self, N, M, tau=2.0, tol=1e-8, stream=None, **opts):
        rc, h = ot_plan_create(N, M, tau, tol)
        _check(rc, "ot_plan_create")
        self.h, self.N, self.M = h, N, M
        self.set(**opts)
        if stream is not None:
            _check(ot_plan_set_stream(h, stream.cuda_stream if hasattr(stream, "cuda_stream")
                                      else int(stream)), "ot_plan_set_stream")

    def set(self, **opts):
        for k, v in opts.items():
            if k == "precision" and isinstance(v, str):
                v = {"fp64": 0, "mixed": 1}[v]
            _check(ot_plan_set_option(self.h, self._keys[k], float(v)), "set " + k)
        return self

    def get(self, name):
        v = ctypes.c_double()
        _check(ot_plan_get_option(self.h, self._keys[name], ctypes.byref(v)), "get " + name)
        return v.value

    def solve(self, f, g, phi, raise_on=(OT_EINVAL, OT_ECUDA, OT_ENOMEM)):
        st = ot_stats()
        shp = (self.N, self.M)
        rc = ot_solve(self.h, _dev(f, shp), _dev(g, shp), _dev(phi, shp), st)
        if rc in raise_on:
            raise OTError(rc, "ot_solve")
        return rc, st.as_dict()

    def profile(self):
        """(per-class {name: (ms, launches)}, total kernel launches) since the last reset."""
        import numpy as np
        ms = np.zeros(len(PROF_CLASSES))
        n = np.zeros(len(PROF_CLASSES), dtype=np.int64)
        tot = np.zeros(1, dtype=np.int64)
        _check(ot_plan_get_profile(self.h, ms.ctypes.data_as(ctypes.c_void_p),
                                   n.ctypes.data_as(ctypes.c_void_p), len(PROF_CLASSES),
                                   tot.ctypes.data_as(ctypes.c_void_p)), "profile")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(PROF_CLASSES)}, int(tot[0])

    def time_kernel(self, name, reps=50):
        """Mean ms per launch of one kernel class (a PROF_CLASSES name, or "ws_network"),
        relaunched back to back after a solve."""
        ms = ctypes.c_double()
        cls = OT_TIME_WS_NETWORK if name == "ws_network" else PROF_CLASSES.index(name)
        _check(ot_plan_time_kernel(self.h, cls, reps, ctypes.byref(ms)), "time_kernel")
        return ms.value

    def reset_profile(self):
        _check(ot_plan_reset_profile(self.h), "reset_profile")

    def solve_host(self, f, g, phi, raise_on=(OT_EINVAL, OT_ECUDA, OT_ENOMEM)):
        """ot_solve_host on contiguous float64 numpy arrays (pinned or pageable)."""
        st = ot_stats()
        for a in (f, g, phi):
            if a.dtype.name != "float64" or not a.flags.c_contiguous or a.shape != (self.N, self.M):
                raise TypeError("expected contiguous float64 arrays of shape (N, M)")
        vp = ctypes.c_void_p
        rc = ot_solve_host(self.h, vp(f.ctypes.data), vp(g.ctypes.data), vp(phi.ctypes.data), st)
        if rc in raise_on:
            raise OTError(rc, "ot_solve_host")
        return rc, st.as_dict()

    # ---- learned warm start
    def set_weights(self, params):
        """Upload network parameters (numpy float32, ot_ws_param_count() values)."""
        import numpy as np
        a = np.ascontiguousarray(params, dtype=np.float32)
        _check(ot_ws_set_weights(self.h, ctypes.c_void_p(a.ctypes.data), a.size),
               "ot_ws_set_weights")
        return self

    def load_weights(self, path):
        _check(ot_warmstart_load(self.h, path), "ot_warmstart_load")
        return self

    def ws_predict(self, f, g, phi0):
        """Learned warm start alone: phi0 (float64 CUDA tensor) <- u0; returns alpha."""
        shp = (self.N, self.M)
        a = ctypes.c_double()
        _check(ot_ws_predict(self.h, _dev(f, shp), _dev(g, shp), _dev(phi0, shp),
                             ctypes.byref(a)), "ot_ws_predict")
        return a.value

    def ws_features(self, f, g, X, target=None, phi_star=None):
        """Features (float32 CUDA tensor N*M x 16) and, with phi_star, the target (N*M)."""
        shp = (self.N, self.M)
        _check(ot_ws_features(self.h, _dev(f, shp), _dev(g, shp),
                              _dev(phi_star, shp) if phi_star is not None else None,
                              _dev32(X, (self.N * self.M, 16)),
                              _dev32(target, (self.N * self.M,)) if target is not None
                              else None), "ot_ws_features")

    def ws_mlp_forward(self, X, out):
        rows = X.shape[0]
        _check(ot_ws_mlp_forward(self.h, _dev32(X, (rows, 16)), rows, _dev32(out, (rows,))),
               "ot_ws_mlp_forward")

    def ws_poisson(self, src, u, lowpass=False):
        shp = (self.N, self.M)
        _check(ot_ws_poisson(self.h, _dev(src, shp), lowpass, _dev(u, shp)), "ot_ws_poisson")

    def inverse_spectral_radius(self, f, g, phi, b0, iters=5):
        """Power iteration on the inverse of the linearised operator at phi (Sec. 5.1):
        the norms ||A^{-1} b_k|| (numpy array of iters values)."""
        import numpy as np
        shp = (self.N, self.M)
        rho = np.zeros(int(iters))
        _check(ot_inverse_spectral_radius(self.h, _dev(f, shp), _dev(g, shp), _dev(phi, shp),
                                          _dev(b0, shp), iters,
                                          ctypes.c_void_p(rho.ctypes.data)),
               "ot_inverse_spectral_radius")
        return rho

    def fd_apply(self, coef, x, y, transpose=False):
        """y = A~ x or A~^T x, the finite-difference operator of Sec. 4.1 (needs
        linear_solver=1); coef: device (5, N, M)."""
        shp = (self.N, self.M)
        _check(ot_fd_apply(self.h, _dev(coef, (5,) + shp), _dev(x, shp), int(bool(transpose)),
                           _dev(y, shp)), "ot_fd_apply")

    def fd_bicg(self, coef, h, theta, eta=1e-4, max_iters=20000):
        """BiCG on A~ theta = h (Sec. 4.1): returns (status, iterations, ||r|| / ||h||)."""
        shp = (self.N, self.M)
        it = ctypes.c_int32()
        rr = ctypes.c_double()
        rc = ot_fd_bicg(self.h, _dev(coef, (5,) + shp), _dev(h, shp), eta, max_iters,
                        _dev(theta, shp), ctypes.byref(it), ctypes.byref(rr))
        if rc not in (OT_OK, OT_ENOCONV, OT_EDIVERGED):
            _check(rc, "ot_fd_bicg")
        return rc, it.value, rr.value

    def transport_outputs(self, f, phi, div=None):
        """d(f, g) = mean |grad phi|^2 f (Sec. 5.2); fills div (device N x M) with
        phi_xx + phi_yy when given.  Returns d."""
        shp = (self.N, self.M)
        d = ctypes.c_double()
        _check(ot_transport_outputs(self.h, _dev(f, shp), _dev(phi, shp), ctypes.byref(d),
                                    _dev(div, shp) if div is not None else None),
               "ot_transport_outputs")
        return d.value

    def close(self):
        if self.h:
            ot_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PlanSet:
    """An ot_plan_set: problems of sizes [(N_k, M_k)] solved together (ot_solve_batched) on
    torch float64 CUDA tensors; options as for Plan (the subset the set takes) plus
    tau_retry."""

    def __init__(self, sizes, tau=1.0, tol=1e-8, stream=None, **opts):
        self.N = [int(n) for n, _ in sizes]
        self.M = [int(m) for _, m in sizes]
        rc, h = ot_plan_set_create(len(sizes), self.N, self.M, tau, tol)
        _check(rc, "ot_plan_set_create")
        self.h = h
        self.set(**opts)
        if stream is not None:
            _check(ot_batch_set_stream(h, stream.cuda_stream if hasattr(stream, "cuda_stream")
                                       else int(stream)), "ot_batch_set_stream")

    def set(self, **opts):
        for k, v in opts.items():
            if k == "precision" and isinstance(v, str):
                v = {"fp64": 0, "mixed": 1}[v]
            _check(ot_batch_set_option(self.h, Plan._keys[k], float(v)), "set " + k)
        return self

    def solve(self, fs, gs, phis, raise_on=(OT_EINVAL, OT_ECUDA, OT_ENOMEM)):
        """Solve every problem; returns (rc, [stats dict per problem])."""
        n = len(self.N)
        if not (len(fs) == len(gs) == len(phis) == n):
            raise ValueError("one f, g, phi per problem")
        ptr = []
        for lst in (fs, gs, phis):
            ptr.append([_dev(t, (self.N[k], self.M[k])).value for k, t in enumerate(lst)])
        st = (ot_stats * n)()
        rc = ot_solve_batched(self.h, n, self.N, self.M, ptr[0], ptr[1], ptr[2], st)
        if rc in raise_on:
            raise OTError(rc, "ot_solve_batched")
        return rc, [st[k].as_dict() for k in range(n)]

    def close(self):
        if self.h:
            ot_plan_set_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(f, g, tau=2.0, tol=1e-8, **opts):
    """Solve for the mean-zero potential phi (torch float64 CUDA tensor) with
    g(x + grad phi) det(I + D^2 phi) = f; returns (phi, stats)."""
    import torch
    N, M = f.shape
    plan = Plan(N, M, tau=tau, tol=tol, **opts)
    phi = torch.zeros_like(f)
    rc, st = plan.solve(f, g, phi)
    plan.close()
    return phi, st
