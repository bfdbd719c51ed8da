"""Pins of the stencil-symbol operator option: with the Fourier symbols of the 4th-order
stencils, L is the exact linearisation of the discrete residual F, checked against central
differences of the oracle's independent residual routine."""
import numpy as np
import pytest

import oracle as O
import ot_inputs as I


def smooth(N, M, amp, seed):
    rng = np.random.default_rng(seed)
    x, y = I.grid(N, M)
    u = np.zeros((N, M))
    for _ in range(6):
        k1, k2 = rng.integers(-4, 5, 2)
        u += rng.standard_normal() * np.cos(2 * np.pi * (k1 * x + k2 * y) + rng.random() * 6)
    return amp * u


@pytest.mark.parametrize("N,M", [(24, 32), (32, 32), (16, 48)])
def test_stencil_symbol_operator_is_the_jacobian_of_the_residual(N, M):
    f = I.blob_density(N, M, 5)
    g = I.blob_density(N, M, 6)
    c = O.bspline_coeffs(g)
    u = smooth(N, M, 2e-3, 1)
    _, coef, _ = O.residual(f, c, u)
    abar = np.array([O.simpson_mean(coef[q]) for q in range(5)])
    sigma = np.random.default_rng(2).standard_normal((N, M))
    with O.fd_symbols():
        theta = O.apply_lbar_inv(abar, sigma)
        w = O.apply_op(coef, abar, sigma)
    e = 1e-6
    dF = (O.residual(f, c, u + e * theta)[0] - O.residual(f, c, u - e * theta)[0]) / (2 * e)
    # F = f - (f_n - mean f_n + 1): dF = -(df_n - mean df_n), and L theta = df_n
    lhs, rhs = w - w.mean(), -(dF - dF.mean())
    assert np.abs(lhs - rhs).max() <= 1e-7 * np.abs(rhs).max()
    # the spectral operator differs from the Jacobian at the high frequencies
    w_sp = O.apply_op(coef, abar, sigma)
    assert np.abs(w_sp - w_sp.mean() - rhs).max() > 1e-2 * np.abs(rhs).max()


def test_stencil_symbol_preconditioner_inverts_the_constant_coefficient_operator():
    # a = abar, b = bbar constant: L Lbar^{-1} = identity on mean-zero fields
    N, M = 24, 32
    abar = np.array([1.2, 0.1, 0.8, 0.3, -0.2])
    coef = np.broadcast_to(abar[:, None, None], (5, N, M)).copy()
    sigma = np.random.default_rng(4).standard_normal((N, M))
    with O.fd_symbols():
        w = O.apply_op(coef, abar, sigma)
    assert np.abs(w - (sigma - sigma.mean())).max() < 1e-12


def test_stencil_symbol_solve_reaches_the_same_root():
    N = M = 24
    f, g = I.blob_pair(N, M, s=8)
    u0, st0, h0, _ = O.solve(f, g, tau=2.0, tol=1e-10, eta=1e-1)
    with O.fd_symbols():
        u1, st1, h1, _ = O.solve(f, g, tau=1.0, tol=1e-10, eta=1e-1)
    assert st0["status"] == 0 and st1["status"] == 0
    assert np.abs(u0 - u1).max() < 1e-10
    # exact Newton (tau = 1, consistent Jacobian, accurate inner solves) converges fast
    assert st1["newton_iters"] < st0["newton_iters"]


def test_simplified_operator_drops_only_the_grad_g_term():
    # Sec. 3.3 remark: g(x + grad u) Tr(Adj(I + D^2 u) D^2 theta) = (f - f_n) / tau, i.e. the
    # coefficients b = 0; F and a are untouched, and the root (defined by F alone) is the same
    f, g = I.blob_pair(24, 32, s=11)
    u = 1e-3 * np.random.default_rng(2).standard_normal((24, 32))
    c = O.bspline_coeffs(g)
    F0, a0, s0 = O.residual(f, c, u)
    with O.simplified_operator():
        F1, a1, s1 = O.residual(f, c, u)
    assert np.array_equal(F0, F1) and np.array_equal(a0[:3], a1[:3])
    assert not a1[3:].any() and np.abs(a0[3:]).max() > 1.0
    fm, gm, _ = I.manufactured(32, 32)
    u_full, st_full, _, _ = O.solve(fm, gm, tau=2.0, tol=1e-10, eta=1e-2)
    with O.simplified_operator():
        u_simp, st_simp, _, _ = O.solve(fm, gm, tau=2.0, tol=1e-10, eta=1e-2)
    assert st_full["status"] == 0 and st_simp["status"] == 0
    assert np.abs(u_full - u_simp).max() <= 1e-9
