"""FP64 CPU oracle of the damped-Newton Monge-Ampere solver for periodic L2 optimal
transport (Saumier, Agueh & Khouider, arXiv:1009.6039).

TEST INFRASTRUCTURE ONLY.  The plain C implementation lives in ``ot_oracle.c``; this module
builds it with gcc (``build()``) and wraps it with ctypes + numpy.  Only ``tests/``, the
smoke check and the benchmark's CPU-baseline leg may import it.  The CUDA product path
shares no code with it.

Grid convention: arrays are (N, M) float64, row index i is y = i/N, column index j is
x = j/M.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ot_oracle.c")
_LIB = os.path.join(_HERE, "libot_oracle.so")
_lib = None

ORC_OK, ORC_EINVAL, ORC_ENOCONV, ORC_EDIVERGED = 0, -1, -2, -3


class Opts(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("tol", ctypes.c_double), ("eta", ctypes.c_double),
                ("restart", ctypes.c_int), ("max_restarts", ctypes.c_int),
                ("max_newton", ctypes.c_int), ("translate_inputs", ctypes.c_int),
                ("safeguard", ctypes.c_int), ("tau_switch", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("newton_iters", ctypes.c_int),
                ("gmres_iters", ctypes.c_int), ("gmres_cycles", ctypes.c_int),
                ("step_halvings", ctypes.c_int),
                ("res_inf", ctypes.c_double), ("res_l2", ctypes.c_double),
                ("min_det", ctypes.c_double), ("mean_fn", ctypes.c_double),
                ("u_mean", ctypes.c_double)]


def build(force=False):
    """Compile the oracle with gcc (portable flags only: it must build on x86 and Arm)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ot_oracle.h"))):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        _lib.orc_fft2.argtypes = [vp, vp, i, i, i]
        _lib.orc_fft1.argtypes = [vp, vp, i, i]
        _lib.orc_dft2.argtypes = [vp, vp, i, i, i, vp, vp]
        _lib.orc_derivatives.argtypes = [vp, i, i, vp, vp, vp, vp, vp]
        _lib.orc_bspline_coeffs.argtypes = [vp, i, i, vp]
        _lib.orc_bspline_eval.argtypes = [vp, i, i, d, d, vp, vp, vp]
        _lib.orc_residual.argtypes = [vp, vp, vp, i, i, vp, vp, vp]
        _lib.orc_simpson_mean.argtypes = [vp, i, i]
        _lib.orc_simpson_mean.restype = d
        _lib.orc_apply_op.argtypes = [vp, vp, vp, i, i, vp]
        _lib.orc_apply_lbar_inv.argtypes = [vp, vp, i, i, vp]
        _lib.orc_gmres_dense.argtypes = [vp, vp, i, i, d, i, vp, vp, vp, vp]
        _lib.orc_gmres_op.argtypes = [vp, vp, vp, i, i, i, d, i, vp, vp, vp, vp]
        _lib.orc_solve.argtypes = [vp, vp, i, i, ctypes.POINTER(Opts), vp,
                                   ctypes.POINTER(Stats), vp, vp]
        _lib.orc_default_opts.argtypes = [ctypes.POINTER(Opts)]
        _lib.orc_fd_poisson.argtypes = [vp, i, i, i, vp]
        _lib.orc_set_fd_symbols.argtypes = [i]
        _lib.orc_set_simplified.argtypes = [i]
        _lib.orc_set_interp.argtypes = [i]
        _lib.orc_get_interp.restype = i
        _lib.orc_ws_features.argtypes = [vp, vp, vp, vp, i, i, vp]
        _lib.orc_fd_apply.argtypes = [vp, vp, i, i, vp]
        _lib.orc_fd_apply_t.argtypes = [vp, vp, i, i, vp]
        _lib.orc_bicg_dense.argtypes = [vp, vp, i, d, i, vp, vp, vp]
        _lib.orc_bicg_fd.argtypes = [vp, vp, i, i, d, i, vp, vp, vp]
        _lib.orc_set_linear_solver.argtypes = [i, i]
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def fft2(x, inverse=False):
    """Unnormalised 2-D DFT (sign -1 forward, +1 inverse) by the oracle's own FFT."""
    x = np.asarray(x, dtype=np.complex128)
    re, im = _f64(x.real).copy(), _f64(x.imag).copy()
    N, M = x.shape
    lib().orc_fft2(_p(re), _p(im), N, M, 1 if inverse else -1)
    return re + 1j * im


def dft2(x, inverse=False):
    """Brute-force O(P^2) 2-D DFT."""
    x = np.asarray(x, dtype=np.complex128)
    re, im = _f64(x.real), _f64(x.imag)
    N, M = x.shape
    ore, oim = np.empty_like(re), np.empty_like(re)
    lib().orc_dft2(_p(re), _p(im), N, M, 1 if inverse else -1, _p(ore), _p(oim))
    return ore + 1j * oim


def fft1(x, inverse=False):
    x = np.asarray(x, dtype=np.complex128)
    re, im = _f64(x.real).copy(), _f64(x.imag).copy()
    lib().orc_fft1(_p(re), _p(im), x.shape[0], 1 if inverse else -1)
    return re + 1j * im


def derivatives(u):
    """(u_x, u_y, u_xx, u_yy, u_xy) by the 4th-order centred stencils."""
    u = _f64(u)
    N, M = u.shape
    outs = [np.empty_like(u) for _ in range(5)]
    lib().orc_derivatives(_p(u), N, M, *[_p(o) for o in outs])
    return tuple(outs)


def transport_outputs(f, u):
    """Sec. 5.2: the transport distance d(f, g) = int |x - T(x)|^2 f dx = int |grad u|^2 f dx
    with T = x + grad u, as the grid mean of |grad u|^2 f (the periodic trapezoid rule), and
    the divergence of the displacement grad u, u_xx + u_yy; derivatives by the 4th-order
    centred stencils of derivatives().  Returns (d, div)."""
    f = _f64(f)
    ux, uy, uxx, uyy, _ = derivatives(u)
    return float(np.mean((ux * ux + uy * uy) * f)), uxx + uyy


def bspline_coeffs(g):
    g = _f64(g)
    c = np.empty_like(g)
    if lib().orc_bspline_coeffs(_p(g), g.shape[0], g.shape[1], _p(c)) != 0:
        raise ValueError("grid too small")
    return c


def bspline_eval(c, x, y):
    """Interpolant value and gradient at torus points (x along columns, y along rows)."""
    c = _f64(c)
    N, M = c.shape
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    y = np.atleast_1d(np.asarray(y, dtype=np.float64))
    v, gx, gy = np.empty_like(x), np.empty_like(x), np.empty_like(x)
    a, b, e = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    for k in range(x.size):
        lib().orc_bspline_eval(_p(c), N, M, float(x.flat[k]), float(y.flat[k]),
                               ctypes.byref(a), ctypes.byref(b), ctypes.byref(e))
        v.flat[k], gx.flat[k], gy.flat[k] = a.value, b.value, e.value
    return v, gx, gy


def residual(f, c, u):
    """Returns (F, coef[5,N,M], scal) with F = f - f~_n, coef = (a11, a12, a22, b1, b2),
    scal = dict(mean_fn, res_inf, res_l2, min_det, nonfinite)."""
    f, c, u = _f64(f), _f64(c), _f64(u)
    N, M = u.shape
    F = np.empty_like(u)
    coef = np.empty((5, N, M))
    s = np.empty(5)
    lib().orc_residual(_p(f), _p(c), _p(u), N, M, _p(F), _p(coef), _p(s))
    return F, coef, dict(mean_fn=s[0], res_inf=s[1], res_l2=s[2], min_det=s[3],
                         nonfinite=int(s[4]))


def simpson_mean(a):
    a = _f64(a)
    return lib().orc_simpson_mean(_p(a), a.shape[0], a.shape[1])


def apply_op(coef, abar, sigma):
    """w = L Lbar^{-1} sigma."""
    coef, ab, sigma = _f64(coef), _f64(abar), _f64(sigma)
    N, M = sigma.shape
    w = np.empty_like(sigma)
    lib().orc_apply_op(_p(coef), _p(ab), _p(sigma), N, M, _p(w))
    return w


def apply_lbar_inv(abar, sigma):
    """theta = Lbar^{-1} sigma."""
    ab, sigma = _f64(abar), _f64(sigma)
    N, M = sigma.shape
    th = np.empty_like(sigma)
    lib().orc_apply_lbar_inv(_p(ab), _p(sigma), N, M, _p(th))
    return th


def gmres_dense(A, b, m=10, eta=1e-10, max_restarts=50):
    A, b = _f64(A), _f64(b)
    n = b.shape[0]
    x = np.empty(n)
    it, cy, rr = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    st = lib().orc_gmres_dense(_p(A), _p(b), n, m, eta, max_restarts, _p(x), ctypes.byref(it),
                               ctypes.byref(cy), ctypes.byref(rr))
    return x, dict(status=st, iters=it.value, cycles=cy.value, relres=rr.value)


def fd_apply(coef, x, transpose=False):
    """Sec. 4.1: y = A~ x (or A~^T x), A the second-order centred-difference discretisation of
    the linearised operator with the coefficients of residual(), A~ = A + 1 1^T (the extra
    equation sum x = 0 added to every row)."""
    coef, x = _f64(coef), _f64(x)
    N, M = x.shape
    y = np.empty_like(x)
    fn = lib().orc_fd_apply_t if transpose else lib().orc_fd_apply
    fn(_p(coef), _p(x), N, M, _p(y))
    return y


def bicg_dense(A, b, eta=1e-10, max_iters=1000):
    """Unpreconditioned BiCG (Sec. 4.1) on a dense system, from x = 0."""
    A, b = _f64(A), _f64(b)
    n = b.shape[0]
    x = np.empty(n)
    it, rr = ctypes.c_int(), ctypes.c_double()
    st = lib().orc_bicg_dense(_p(A), _p(b), n, eta, max_iters, _p(x), ctypes.byref(it),
                              ctypes.byref(rr))
    return x, dict(status=st, iters=it.value, relres=rr.value)


def bicg_fd(coef, h, eta=1e-4, max_iters=20000):
    """BiCG on A~ theta = h (Sec. 4.1), from theta = 0."""
    coef, h = _f64(coef), _f64(h)
    N, M = h.shape
    t = np.empty_like(h)
    it, rr = ctypes.c_int(), ctypes.c_double()
    st = lib().orc_bicg_fd(_p(coef), _p(h), N, M, eta, max_iters, _p(t), ctypes.byref(it),
                           ctypes.byref(rr))
    return t, dict(status=st, iters=it.value, relres=rr.value)


class fd_bicg:
    """Context manager: the Newton steps of solve() take theta from the finite-difference
    system of Sec. 4.1 solved by BiCG (at most max_iters iterations per step; the stats'
    gmres_iters count BiCG iterations) instead of the Fourier method of Sec. 4.2."""

    def __init__(self, max_iters=20000):
        self.max_iters = max_iters

    def __enter__(self):
        lib().orc_set_linear_solver(1, int(self.max_iters))
        return self

    def __exit__(self, *exc):
        lib().orc_set_linear_solver(0, 0)
        return False


def gmres_op(coef, abar, h, m=10, eta=1e-4, max_restarts=50):
    coef, ab, h = _f64(coef), _f64(abar), _f64(h)
    N, M = h.shape
    s = np.empty_like(h)
    it, cy, rr = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    st = lib().orc_gmres_op(_p(coef), _p(ab), _p(h), N, M, m, eta, max_restarts, _p(s),
                            ctypes.byref(it), ctypes.byref(cy), ctypes.byref(rr))
    return s, dict(status=st, iters=it.value, cycles=cy.value, relres=rr.value)


def solve(f, g, tau=2.0, tol=1e-10, eta=1e-4, restart=10, max_restarts=50, max_newton=200,
          u0=None, translate_inputs=True, safeguard=True, tau_switch=0.0):
    """Damped Newton solve.  Returns (u, stats dict, res history, gmres history)."""
    f, g = _f64(f), _f64(g)
    N, M = f.shape
    o = Opts()
    lib().orc_default_opts(ctypes.byref(o))
    o.tau, o.tol, o.eta, o.restart = tau, tol, eta, restart
    o.max_restarts, o.max_newton = max_restarts, max_newton
    o.translate_inputs, o.safeguard = int(translate_inputs), int(safeguard)
    o.tau_switch = float(tau_switch)
    u = np.zeros((N, M)) if u0 is None else _f64(u0).copy()
    st = Stats()
    hres = np.zeros(max_newton + 1)
    hgm = np.zeros(max_newton + 1, dtype=np.int32)
    lib().orc_solve(_p(f), _p(g), N, M, ctypes.byref(o), _p(u), ctypes.byref(st), _p(hres),
                    _p(hgm))
    d = {k: getattr(st, k) for k, _ in Stats._fields_}
    n = d["newton_iters"]
    return u, d, hres[:n + 1].copy(), hgm[:n].copy()


def inverse_spectral_radius(f, g, u, b0, iters=5, eta=1e-4, restart=10, max_restarts=50,
                            translate_inputs=True):
    """Sec. 5.1: power iteration on the inverse of the discretised linearised operator at the
    iterate u, b_(k+1) = A^{-1} b_k / ||A^{-1} b_k||_2, where A^{-1} b = Lbar^{-1} sigma and
    sigma solves L Lbar^{-1} sigma = b by GMRES(m) (the Fourier method of Sec. 4.2, with the
    symbols the fd_symbols switch selects).  b0 is projected to mean zero (the operator acts on
    mean-zero potentials, Sec. 3.1).  Returns the norms ||A^{-1} b_k|| of the unit b_k."""
    f, g, u = _f64(f), _f64(g), _f64(u)
    if translate_inputs:
        f = f - f.mean() + 1.0
        g = g - g.mean() + 1.0
    c = bspline_coeffs(g)
    _, coef, _ = residual(f, c, u)
    abar = np.array([simpson_mean(coef[q]) for q in range(5)])
    b = _f64(b0) - np.mean(b0)
    b = b / np.linalg.norm(b)
    rho = []
    for _ in range(iters):
        sigma, _ = gmres_op(coef, abar, b, m=restart, eta=eta, max_restarts=max_restarts)
        th = apply_lbar_inv(abar, sigma)
        r = float(np.linalg.norm(th))
        rho.append(r)
        b = th / r
    return np.array(rho)


def fd_poisson(src, lowpass=False):
    """Mean-zero solution of (D_xx + D_yy) out = src - mean(src) (4th-order stencils); with
    lowpass, of the source filtered by exp(-((k1/(M/4))^2 + (k2/(N/4))^2)/2)."""
    src = _f64(src)
    out = np.empty_like(src)
    if lib().orc_fd_poisson(_p(src), src.shape[0], src.shape[1], int(bool(lowpass)),
                            _p(out)) != 0:
        raise ValueError("fft failed")
    return out


def ws_features(f, g, c, h):
    """(N, M, 16) features of the warm-start network at the potential h."""
    f, g, c, h = _f64(f), _f64(g), _f64(c), _f64(h)
    N, M = f.shape
    X = np.empty((N, M, 16))
    lib().orc_ws_features(_p(f), _p(g), _p(c), _p(h), N, M, _p(X))
    return X


class fd_symbols:
    """Context manager: the linear operator (apply_op, apply_lbar_inv, gmres_op, solve) uses
    the Fourier symbols of the 4th-order stencils instead of the spectral ones."""

    def __init__(self, on=True):
        self.on = on

    def __enter__(self):
        lib().orc_set_fd_symbols(int(bool(self.on)))
        return self

    def __exit__(self, *exc):
        lib().orc_set_fd_symbols(0)
        return False


class interpolation:
    """Context manager: g at the displaced points by bilinear (mode 1) or nearest-node
    (mode 2) interpolation of the grid values, grad g by the same rule on the grid's 4th-order
    centred differences (Sec. 4 intro; Sec. 5.2 and 5.3); the solve then skips the B-spline
    prefilter and residual() takes the grid values of g in place of coefficients."""

    def __init__(self, mode):
        self.mode = {"bspline": 0, "bilinear": 1, "nearest": 2}.get(mode, mode)

    def __enter__(self):
        lib().orc_set_interp(int(self.mode))
        return self

    def __exit__(self, *exc):
        lib().orc_set_interp(0)
        return False


def interp_coeffs(g):
    """What residual() takes for g in the current interpolation mode: the B-spline
    coefficients (default) or the grid values themselves (bilinear, nearest)."""
    return bspline_coeffs(g) if lib().orc_get_interp() == 0 else _f64(g).copy()


class simplified_operator:
    """Context manager: the residual's coefficients (and so the operator of apply_op and the
    solve) drop the grad g term, b = 0: the simplified equation g(x + grad u) Tr(Adj(I +
    D^2 u) D^2 theta) = (f - f_n) / tau that Sec. 3.3 reports working in practice."""

    def __init__(self, on=True):
        self.on = on

    def __enter__(self):
        lib().orc_set_simplified(int(bool(self.on)))
        return self

    def __exit__(self, *exc):
        lib().orc_set_simplified(0)
        return False
