"""Pins of the oracle's residual, Strain operator, GMRES and damped-Newton solve against
closed forms, invariants, special cases and an independent 1-D construction (no GPU)."""
import json
import os

import numpy as np
import pytest

import oracle as O
import ot_inputs as I

RNG = np.random.default_rng(99)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid(N, M):
    return np.meshgrid(np.arange(M) / M, np.arange(N) / N, indexing="xy")


# ----------------------------------------------------------------------------------------
# Simpson averages (Sec. 4.2)
# ----------------------------------------------------------------------------------------
def test_simpson_weights_pattern():
    N, M = 6, 8
    assert abs(O.simpson_mean(np.ones((N, M))) - 1.0) < 1e-15
    alt = np.tile((-1.0) ** np.arange(M), (N, 1))  # +1 on even j, -1 on odd j
    # per-axis weights 2/3 (even) and 4/3 (odd), divided by the length
    assert abs(O.simpson_mean(alt) - (2 / 3 - 4 / 3) / 2) < 1e-15
    alt_y = alt.T.copy()
    assert abs(O.simpson_mean(alt_y) - (2 / 3 - 4 / 3) / 2) < 1e-15


def test_simpson_periodic_integral():
    # integral of exp(sin 2 pi x) exp(cos 2 pi y) over the unit square = I0(1)^2
    i0 = 1.2660658777520082
    x, y = _grid(32, 48)
    a = np.exp(np.sin(2 * np.pi * x)) * np.exp(np.cos(2 * np.pi * y))
    assert abs(O.simpson_mean(a) - i0 * i0) < 1e-12


# ----------------------------------------------------------------------------------------
# Residual and coefficients (Eq. ma2, linearmaeq, translation)
# ----------------------------------------------------------------------------------------
def test_residual_at_zero_potential():
    N, M = 16, 24
    f = 1 + 0.3 * RNG.random((N, M))
    g = 1 + 0.3 * RNG.random((N, M))
    c = O.bspline_coeffs(g)
    F, coef, s = O.residual(f, c, np.zeros((N, M)))
    np.testing.assert_allclose(F, f - (g - g.mean() + 1), atol=1e-13)
    np.testing.assert_allclose(coef[0], g, atol=1e-13)
    np.testing.assert_allclose(coef[1], 0.0, atol=1e-13)
    np.testing.assert_allclose(coef[2], g, atol=1e-13)
    x, y = _grid(N, M)
    _, gx, gy = O.bspline_eval(c, x.ravel(), y.ravel())
    np.testing.assert_allclose(coef[3], gx.reshape(N, M), atol=1e-11)
    np.testing.assert_allclose(coef[4], gy.reshape(N, M), atol=1e-11)
    assert s["min_det"] == 1.0
    assert abs(s["mean_fn"] - g.mean()) < 1e-14


def test_residual_transpose_symmetry():
    N, M = 12, 16
    f = 1 + 0.2 * RNG.random((N, M))
    g = 1 + 0.2 * RNG.random((N, M))
    u = 1e-3 * RNG.standard_normal((N, M))
    F, coef, _ = O.residual(f, O.bspline_coeffs(g), u)
    Ft, coeft, _ = O.residual(f.T, O.bspline_coeffs(g.T), u.T)
    np.testing.assert_allclose(Ft, F.T, atol=1e-12)
    for a, b in ((0, 2), (1, 1), (2, 0), (3, 4), (4, 3)):
        np.testing.assert_allclose(coeft[a], coef[b].T, atol=1e-10)


def test_residual_manufactured_fourth_order():
    errs = []
    for N in (16, 32, 64):
        f, g, phi = I.manufactured(N, N)
        F, _, s = O.residual(f, O.bspline_coeffs(g), phi)
        errs.append(s["res_inf"])
        assert abs(F.mean()) < 1e-14 + abs(f.mean() - 1)
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (orders > 3.6).all() and (orders < 4.6).all(), orders


# ----------------------------------------------------------------------------------------
# Strain's operator (Sec. 4.2): closed forms on single Fourier modes
# ----------------------------------------------------------------------------------------
def _mode_closed_form(coef, abar, k1, k2, x, y):
    """L Lbar^{-1} cos(2 pi (k1 x + k2 y)) for non-Nyquist k: with s_p = 2 pi i k_p,
    alpha_pq = Re(s_p s_q rho e^{i phi}), beta_p = Re(s_p rho e^{i phi}),
    rho = 1 / (sum abar_pq s_p s_q + sum bbar_p s_p)."""
    s = [2j * np.pi * k1, 2j * np.pi * k2]
    A = [[abar[0], abar[1]], [abar[1], abar[2]]]
    den = sum(A[p][q] * s[p] * s[q] for p in range(2) for q in range(2)) + \
        abar[3] * s[0] + abar[4] * s[1]
    rho = 1.0 / den
    e = np.exp(2j * np.pi * (k1 * x + k2 * y))
    a = [[coef[0], coef[1]], [coef[1], coef[2]]]
    w = sum(a[p][q] * np.real(s[p] * s[q] * rho * e) for p in range(2) for q in range(2))
    w = w + coef[3] * np.real(s[0] * rho * e) + coef[4] * np.real(s[1] * rho * e)
    theta = np.real(rho * e)
    return w, theta


@pytest.mark.parametrize("k1,k2", [(1, 0), (0, 2), (3, -2), (-5, 4), (7, 5)])
def test_operator_single_mode_closed_form(k1, k2):
    N, M = 12, 16
    x, y = _grid(N, M)
    coef = np.stack([1 + 0.3 * np.sin(2 * np.pi * x), 0.1 * np.cos(2 * np.pi * y),
                     1.2 + 0.2 * np.cos(2 * np.pi * (x + y)), 0.4 * np.sin(2 * np.pi * y),
                     -0.3 * np.cos(2 * np.pi * x)])
    abar = np.array([1.1, 0.05, 1.3, 0.2, -0.15])
    sigma = np.cos(2 * np.pi * (k1 * x + k2 * y))
    w_ref, th_ref = _mode_closed_form(coef, abar, k1, k2, x, y)
    np.testing.assert_allclose(O.apply_op(coef, abar, sigma), w_ref, atol=1e-12)
    np.testing.assert_allclose(O.apply_lbar_inv(abar, sigma), th_ref, atol=1e-14)


def test_operator_nyquist_modes():
    N, M = 8, 12
    x, y = _grid(N, M)
    coef = np.stack([1 + 0.2 * RNG.random((N, M)) for _ in range(5)])
    abar = np.array([1.1, 0.2, 0.9, 0.3, -0.4])
    # x-Nyquist mode (-1)^j: first-derivative symbol 0, second -(pi M)^2
    sig = np.cos(np.pi * M * x)
    rho = 1.0 / (abar[0] * -(np.pi * M) ** 2)
    np.testing.assert_allclose(O.apply_op(coef, abar, sig),
                               coef[0] * -(np.pi * M) ** 2 * rho * sig, atol=1e-12)
    # mixed Nyquist in both axes
    sig = np.cos(np.pi * M * x) * np.cos(np.pi * N * y)
    den = abar[0] * -(np.pi * M) ** 2 + abar[2] * -(np.pi * N) ** 2
    w = (coef[0] * -(np.pi * M) ** 2 + coef[2] * -(np.pi * N) ** 2) / den * sig
    np.testing.assert_allclose(O.apply_op(coef, abar, sig), w, atol=1e-12)
    # the mean is annihilated (rho-bar(0) = 0)
    np.testing.assert_allclose(O.apply_op(coef, abar, np.ones((N, M))), 0.0, atol=1e-13)


def test_operator_identity_for_constant_unit_coefficients():
    N, M = 16, 16
    coef = np.stack([np.ones((N, M)), np.zeros((N, M)), np.ones((N, M)), np.zeros((N, M)),
                     np.zeros((N, M))])
    abar = np.array([1.0, 0.0, 1.0, 0.0, 0.0])
    s = RNG.standard_normal((N, M))
    np.testing.assert_allclose(O.apply_op(coef, abar, s), s - s.mean(), atol=1e-12)


def test_lbar_inverse_is_poisson_solve():
    N, M = 16, 24
    s = RNG.standard_normal((N, M))
    th = O.apply_lbar_inv(np.array([1.0, 0.0, 1.0, 0.0, 0.0]), s)
    k1 = np.fft.fftfreq(M, 1.0 / M)
    k2 = np.fft.fftfreq(N, 1.0 / N)
    lap = -4 * np.pi ** 2 * (k2[:, None] ** 2 + k1[None, :] ** 2)
    lap[0, 0] = 1.0
    sh = np.fft.fft2(s) / lap
    sh[0, 0] = 0.0
    np.testing.assert_allclose(th, np.real(np.fft.ifft2(sh)), atol=1e-15)
    assert abs(th.mean()) < 1e-16


# ----------------------------------------------------------------------------------------
# GMRES(m)
# ----------------------------------------------------------------------------------------
def test_gmres_dense_matches_direct_solve():
    n = 40
    A = np.eye(n) * 4 + RNG.standard_normal((n, n)) * 0.3
    b = RNG.standard_normal(n)
    x, info = O.gmres_dense(A, b, m=10, eta=1e-12, max_restarts=100)
    assert info["status"] == 0
    np.testing.assert_allclose(x, np.linalg.solve(A, b), atol=1e-10)


def test_gmres_full_space_terminates():
    n = 8
    A = RNG.standard_normal((n, n)) + 3 * np.eye(n)
    b = RNG.standard_normal(n)
    x, info = O.gmres_dense(A, b, m=n, eta=1e-13, max_restarts=1)
    assert info["status"] == 0 and info["iters"] <= n
    np.testing.assert_allclose(A @ x, b, atol=1e-11)


def test_gmres_operator_one_step_for_laplacian():
    N, M = 16, 16
    coef = np.stack([np.ones((N, M)), np.zeros((N, M)), np.ones((N, M)), np.zeros((N, M)),
                     np.zeros((N, M))])
    h = RNG.standard_normal((N, M))
    h -= h.mean()
    s, info = O.gmres_op(coef, [1, 0, 1, 0, 0], h, eta=1e-10)
    assert info["iters"] == 1
    np.testing.assert_allclose(s, h, atol=1e-13)


# ----------------------------------------------------------------------------------------
# Damped Newton solve (Sec. 3.1 + 4.2)
# ----------------------------------------------------------------------------------------
def test_equal_densities_give_zero_potential():
    f = I.blob_density(16, 16, 7)
    u, st, hres, _ = O.solve(f, f.copy(), tau=2, tol=1e-12)
    assert st["status"] == 0 and st["newton_iters"] == 0
    assert np.abs(u).max() == 0.0


def test_manufactured_fourth_order_and_paper_orders():
    with open(os.path.join(GOLDEN, "paper_table1.json")) as fh:
        paper = json.load(fh)
    errs = []
    for N in (16, 32, 64):
        f, g, phi = I.manufactured(N, N)
        u, st, hres, hg = O.solve(f, g, tau=2, tol=1e-11, eta=1e-4)
        assert st["status"] == 0
        errs.append(np.sqrt(np.mean((u - (phi - phi.mean())) ** 2)))
        # geometric decrease, at least at the theorem's rate 1 - 1/(2 tau)
        ratios = hres[1:] / hres[:-1]
        assert (ratios < 1 - 1 / (2 * 2.0) + 0.02).all(), ratios
        assert abs(np.median(ratios) - 0.5) < 0.05
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    # the paper prints 4.3521, 4.0035, 3.9965, 3.9990 for its (unstated) constants
    lo, hi = min(paper["observed_order_u"]) - 0.4, max(paper["observed_order_u"]) + 0.3
    assert ((orders > lo) & (orders < hi)).all(), orders


def test_gmres_count_nearly_constant_in_N():
    # Sec. 5.1: GMRES iterations per Newton step nearly independent of the grid (Table 1)
    avgs = []
    for N in (16, 32, 64):
        f, g, _ = I.manufactured(N, N, amp=0.1 / (2 * np.pi) ** 2)
        u, st, hres, hg = O.solve(f, g, tau=1, tol=1e-9, eta=1e-1, max_newton=20)
        avgs.append(np.mean(hg))
    assert max(avgs) / min(avgs) < 1.6, avgs
    assert 1 <= min(avgs) and max(avgs) <= 10, avgs


def test_uniform_target_first_step_is_poisson_solve():
    N = 32
    x, y = _grid(N, N)
    f = 1 + 0.2 * np.sin(2 * np.pi * x) * np.cos(4 * np.pi * y) + 0.1 * np.cos(2 * np.pi * y)
    g = np.ones((N, N))
    tau = 2.0
    u, st, _, hg = O.solve(f, g, tau=tau, tol=1e-14, eta=1e-12, max_newton=1)
    assert st["newton_iters"] == 1 and hg[0] == 1
    ft = f - f.mean() + 1
    k = np.fft.fftfreq(N, 1.0 / N)
    lap = -4 * np.pi ** 2 * (k[:, None] ** 2 + k[None, :] ** 2)
    lap[0, 0] = 1
    uh = np.fft.fft2((ft - 1) / tau) / lap
    uh[0, 0] = 0
    np.testing.assert_allclose(u, np.real(np.fft.ifft2(uh)), atol=1e-14)


def _separable_reference(M, a=0.3, b=0.25):
    """1-D optimal transport on the circle: f = 1 + a sin(2 pi x), g = 1 + b cos(2 pi x).
    With primitives F, G (G(y+1) = G(y) + 1), T(x) = G^{-1}(F(x) + c) and c fixed by
    mean(T - x) = 0; u' = T - x integrated spectrally with mean 0."""
    opt = pytest.importorskip("scipy.optimize")

    def Fp(x):
        return x + a * (1 - np.cos(2 * np.pi * x)) / (2 * np.pi)

    def Gp(y):
        return y + b * np.sin(2 * np.pi * y) / (2 * np.pi)

    def T(xs, c):
        return np.array([opt.brentq(lambda t: Gp(t) - Fp(xv) - c, -2, 3, xtol=1e-15)
                         for xv in xs])

    xq = np.arange(256) / 256
    c = opt.brentq(lambda c: np.mean(T(xq, c) - xq), -0.5, 0.5, xtol=1e-15)
    xs = np.arange(M) / M
    du = T(xs, c) - xs
    k = np.fft.fftfreq(M, 1.0 / M)
    dh = np.fft.fft(du)
    uh = np.zeros_like(dh)
    uh[1:] = dh[1:] / (2j * np.pi * k[1:])
    if M % 2 == 0:
        uh[M // 2] = 0
    f1 = 1 + a * np.sin(2 * np.pi * xs)
    g1 = 1 + b * np.cos(2 * np.pi * xs)
    return f1, g1, np.real(np.fft.ifft(uh))


def test_separable_one_dimensional_reference():
    errs = []
    for M in (32, 64):
        f1, g1, uref = _separable_reference(M)
        f = np.tile(f1, (8, 1))
        g = np.tile(g1, (8, 1))
        u, st, _, _ = O.solve(f, g, tau=2, tol=1e-12, eta=1e-6)
        assert st["status"] == 0
        assert np.abs(u - u[0]).max() < 1e-13  # no y dependence
        errs.append(np.abs(u[0] - uref).max())
    assert errs[1] < errs[0] / 10 and errs[1] < 1e-6, errs


def test_safeguard_recovers_convexity():
    f, g = I.blob_pair(32, 32)
    _, st_plain, _, _ = O.solve(f, g, tau=2, tol=1e-6, eta=1e-2, max_newton=40,
                                safeguard=False)
    assert st_plain["status"] == O.ORC_EDIVERGED
    u, st, hres, _ = O.solve(f, g, tau=2, tol=1e-6, eta=1e-2, max_newton=200)
    assert st["status"] == 0 and st["step_halvings"] >= 1
    assert st["min_det"] > 0
    # the converged potential solves the discrete problem: recheck its residual
    c = O.bspline_coeffs(g - g.mean() + 1)
    F, _, s = O.residual(f - f.mean() + 1, c, u)
    assert s["res_inf"] < 1e-6


def test_invalid_inputs_rejected():
    f = np.ones((16, 16))
    g = np.ones((16, 16))
    g[3, 3] = -5.0
    _, st, _, _ = O.solve(f, g)
    assert st["status"] == O.ORC_EINVAL
    g[3, 3] = np.nan
    _, st, _, _ = O.solve(f, g)
    assert st["status"] == O.ORC_EINVAL
    _, st, _, _ = O.solve(f, np.ones((16, 16)), tau=0.5)
    assert st["status"] == O.ORC_EINVAL


def test_tau_schedule():
    # tau schedule (remarks of Sec. 3.3, the tau study of Sec. 5.1): the damping is tau until
    # max|F| < tau_switch, then 1.  Pins: switch 0 is the fixed-tau solve and a switch above
    # the first residual the tau = 1 solve, step for step; with a switch in between the
    # residual history equals the fixed-tau one up to the first step below the switch, and
    # the solve reaches the same root in fewer steps than the fixed tau
    f, g = I.blob_pair(64, 64, s=1001)
    kw = dict(tol=1e-10, eta=1e-2, max_newton=400)
    with O.fd_symbols():
        u2, s2, h2, _ = O.solve(f, g, tau=2.0, **kw)
        u1, s1, h1, _ = O.solve(f, g, tau=1.0, **kw)
        u0, s0, h0, _ = O.solve(f, g, tau=2.0, tau_switch=0.0, **kw)
        ub, sb, hb, _ = O.solve(f, g, tau=2.0, tau_switch=1e9, **kw)
        us, ss, hs, _ = O.solve(f, g, tau=2.0, tau_switch=0.1, **kw)
    assert np.array_equal(u0, u2) and s0 == s2
    assert np.array_equal(ub, u1) and sb == s1
    k = int(np.argmax(h2 < 0.1))
    assert k > 0 and np.array_equal(hs[:k + 1], h2[:k + 1])
    assert not np.array_equal(hs[k + 1:k + 3], h2[k + 1:k + 3])
    assert ss["status"] == 0 and ss["newton_iters"] < s2["newton_iters"]
    assert np.abs(us - u2).max() <= 1e-10


def test_inverse_spectral_radius_of_the_laplacian():
    # g = 1 at u = 0: the coefficients are a = I, b = 0, so L = Lbar is the Laplacian and the
    # inverse's spectral radius (on mean-zero functions) is 1 / |s2(1)|: 1 / (4 pi^2) with
    # the spectral symbols of Sec. 4.2, 1 / |(-2 cos 2t + 32 cos t - 30) N^2 / 12|, t = 2 pi / N,
    # with the 4th-order stencils' (the largest eigenvalue is that of the four modes k = (+-1,
    # 0), (0, +-1); the next is half of it, so the power iteration gains a bit per step)
    N = 32
    f = I.blob_density(N, N, 3)
    g = np.ones((N, N))
    b0 = I.SplitMix64(77).uniform(N * N).reshape(N, N)
    rho = O.inverse_spectral_radius(f, g, np.zeros((N, N)), b0, iters=45, eta=1e-12)
    assert abs(rho[-1] - 1.0 / (4.0 * np.pi ** 2)) <= 1e-9 * rho[-1]
    t = 2.0 * np.pi / N
    s2 = (-2.0 * np.cos(2 * t) + 32.0 * np.cos(t) - 30.0) * N * N / 12.0
    with O.fd_symbols():
        rho_fd = O.inverse_spectral_radius(f, g, np.zeros((N, N)), b0, iters=45, eta=1e-12)
    assert abs(rho_fd[-1] - 1.0 / abs(s2)) <= 1e-9 * rho_fd[-1]
    assert rho_fd[-1] > rho[-1]  # the stencil symbol is smaller in magnitude at k = 1


def test_inverse_spectral_radius_of_the_manufactured_example():
    # Sec. 5.1 reports about 0.03 for its manufactured example at every Newton step; with this
    # build's constants (g = 1 + 0.5 cos 2 pi x cos 2 pi y, so a ~ g in [0.5, 1.5]) the radius
    # at the solution is of the order of 1 / (4 pi^2 min a): between 0.015 and 0.06
    N = 32
    f, g, phi = I.manufactured(N, N)
    b0 = I.SplitMix64(78).uniform(N * N).reshape(N, N)
    rho = O.inverse_spectral_radius(f, g, phi, b0, iters=8)
    assert 0.015 < rho[-1] < 0.06
    assert abs(rho[-1] - rho[-2]) <= 0.05 * rho[-1]  # settled after a few iterations
