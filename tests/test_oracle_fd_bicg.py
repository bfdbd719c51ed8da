"""Pins of the oracle's finite-difference comparison path (Sec. 4.1): the second-order
centred-difference operator with the augmented row sum (A~ = A + 1 1^T), its transpose, the
unpreconditioned BiCG solver and the Newton solve that uses them."""
import numpy as np
import pytest

import oracle as O
import ot_inputs as I


def symbols(k, L):
    # Fourier symbols of the second-order centred differences on L points (spacing 1/L):
    # first derivative i L sin t, second derivative L^2 (2 cos t - 2), t = 2 pi k / L
    t = 2.0 * np.pi * k / L
    return 1j * L * np.sin(t), L * L * (2.0 * np.cos(t) - 2.0)


def test_constant_coefficients_act_on_fourier_modes():
    # with constant coefficients every Fourier mode e_k (k != 0) is an eigenvector of A with
    # eigenvalue a11 s2(k1) + 2 a12 s1(k1) s1(k2) + a22 s2(k2) + b1 s1(k1) + b2 s1(k2); its
    # sum is zero, so A~ e_k = A e_k; the transpose has the conjugate eigenvalue; A~ 1 = P 1
    N, M = 12, 16
    a11, a12, a22, b1, b2 = 1.3, -0.4, 0.8, 2.5, -1.7
    coef = np.stack([np.full((N, M), v) for v in (a11, a12, a22, b1, b2)])
    ii, jj = np.meshgrid(np.arange(N), np.arange(M), indexing="ij")
    for k1, k2 in [(1, 0), (0, 1), (3, 2), (M // 2, 1), (5, N // 2), (-2, 3)]:
        s1x, s2x = symbols(k1, M)
        s1y, s2y = symbols(k2, N)
        lam = a11 * s2x + 2 * a12 * s1x * s1y + a22 * s2y + b1 * s1x + b2 * s1y
        e = np.exp(2j * np.pi * (k1 * jj / M + k2 * ii / N))
        for part, take in ((e.real, np.real), (e.imag, np.imag)):
            if np.abs(part).max() < 1e-12:
                continue
            y = O.fd_apply(coef, part)
            assert np.abs(y - take(lam * e)).max() <= 1e-9 * abs(lam), (k1, k2)
            yt = O.fd_apply(coef, part, transpose=True)
            assert np.abs(yt - take(np.conj(lam) * e)).max() <= 1e-9 * abs(lam), (k1, k2)
    one = np.ones((N, M))
    assert np.abs(O.fd_apply(coef, one) - N * M).max() <= 1e-9


def test_transpose_is_the_matrix_transpose():
    # variable coefficients: the matrix assembled from A~ applied to unit vectors, transposed,
    # equals the one assembled from the transpose routine (gather form against scatter form)
    N, M = 6, 8
    rng = np.random.default_rng(11)
    coef = rng.standard_normal((5, N, M))
    E = np.eye(N * M)
    A = np.stack([O.fd_apply(coef, E[k].reshape(N, M)).ravel() for k in range(N * M)], 1)
    At = np.stack([O.fd_apply(coef, E[k].reshape(N, M), transpose=True).ravel()
                   for k in range(N * M)], 1)
    assert np.abs(A.T - At).max() <= 1e-12 * np.abs(A).max()
    # A~ = A + 1 1^T with A's rows summing to zero (A kills constants)
    assert np.abs((A - 1.0).sum(axis=1)).max() <= 1e-10 * np.abs(A).max()


def test_second_order_accuracy_on_smooth_data():
    # smooth variable coefficients and a smooth mean-zero theta: A theta approaches the
    # continuous L theta at second order (error ratio ~4 per grid doubling)
    def case(N):
        x = np.arange(N) / N
        X, Y = np.meshgrid(x, x)  # X along j, Y along i
        tp = 2 * np.pi
        th = np.sin(tp * X) * np.cos(2 * tp * Y)
        tx = tp * np.cos(tp * X) * np.cos(2 * tp * Y)
        ty = -2 * tp * np.sin(tp * X) * np.sin(2 * tp * Y)
        txx = -tp ** 2 * th
        tyy = -(2 * tp) ** 2 * th
        txy = -2 * tp ** 2 * np.cos(tp * X) * np.sin(2 * tp * Y)
        a11 = 1.0 + 0.3 * np.cos(tp * Y)
        a12 = 0.2 * np.sin(tp * (X + Y))
        a22 = 1.2 + 0.1 * np.sin(tp * X)
        b1 = 0.5 * np.cos(tp * X)
        b2 = -0.4 * np.sin(tp * Y)
        exact = a11 * txx + 2 * a12 * txy + a22 * tyy + b1 * tx + b2 * ty
        coef = np.stack([a11, a12, a22, b1, b2])
        return np.abs(O.fd_apply(coef, th) - exact).max()
    e = [case(N) for N in (16, 32, 64)]
    for a, b in zip(e, e[1:]):
        assert 3.6 < a / b < 4.4, e


def test_bicg_dense_systems():
    rng = np.random.default_rng(3)
    for n in (6, 12, 24):
        A = rng.standard_normal((n, n)) + 0.5 * n * np.eye(n)
        b = rng.standard_normal(n)
        x, st = O.bicg_dense(A, b, eta=1e-12, max_iters=200)
        assert st["status"] == 0 and st["relres"] <= 1e-12
        assert np.abs(x - np.linalg.solve(A, b)).max() <= 1e-12 * np.abs(x).max() * n
        # finite termination: at most n steps (in exact arithmetic)
        assert st["iters"] <= n
    # breakdown: (A p, p*) = 0 at the first step
    x, st = O.bicg_dense(np.array([[0.0, 1.0], [1.0, 0.0]]), np.array([1.0, 0.0]))
    assert st["status"] == 2 and st["iters"] == 0
    # the iteration cap
    A = rng.standard_normal((30, 30)) + 3.0 * np.eye(30)
    x, st = O.bicg_dense(A, rng.standard_normal(30), eta=1e-14, max_iters=3)
    assert st["status"] == 1 and st["iters"] == 3


def test_augmented_system_returns_the_mean_zero_solution():
    # the lemma of Sec. 4.1: when b = A x0 lies in A's range and x0 has zero sum, the square
    # system A~ x = b (A~ = A + 1 1^T) has the solution x0 itself (sum x = 0), for the
    # coefficients of a real residual evaluation
    N = 16
    f, g = I.blob_pair(N, N, s=21)
    c = O.bspline_coeffs(g)
    u = 1e-3 * I.SplitMix64(5).uniform(N * N).reshape(N, N)
    u -= u.mean()
    _, coef, _ = O.residual(f, c, u)
    x0 = I.SplitMix64(9).uniform(N * N).reshape(N, N)
    x0 -= x0.mean()
    b = O.fd_apply(coef, x0)  # = A x0 since sum x0 = 0
    x, st = O.bicg_fd(coef, b, eta=1e-13, max_iters=5000)
    assert st["status"] == 0
    assert abs(x.sum()) <= 1e-9 * np.abs(x).sum()
    assert np.abs(x - x0).max() <= 1e-8 * np.abs(x0).max()


def test_fd_newton_reaches_the_fourier_root():
    # the root is defined by F alone (Eq. ma2 with the 4th-order stencils), so the Newton
    # iteration with theta from the finite-difference system reaches the same potential as
    # the Fourier method, with the same linear rate at tau = 2 (both Jacobians are
    # approximations of the stencil F's)
    f, g, _ = I.manufactured(32, 32)
    u0, s0, _, _ = O.solve(f, g, tau=2.0, tol=1e-10, eta=1e-4)
    with O.fd_bicg():
        u1, s1, _, it1 = O.solve(f, g, tau=2.0, tol=1e-10, eta=1e-4)
    assert s0["status"] == 0 and s1["status"] == 0
    assert abs(s1["newton_iters"] - s0["newton_iters"]) <= 2
    assert np.abs(u1 - u0).max() <= 1e-10
    assert s1["gmres_cycles"] == s1["newton_iters"]  # one BiCG run per Newton step
    # leaving the context restores the Fourier method
    u2, s2, _, _ = O.solve(f, g, tau=2.0, tol=1e-10, eta=1e-4)
    assert s2 == s0


@pytest.mark.parametrize("eta", [1e-4])
def test_bicg_iterations_grow_with_the_grid(eta):
    # Table 1's shape: the average BiCG iterations per Newton step grow roughly in
    # proportion to N (14.21, 17.79, 31.11, 63.32, 134.63 for N = 16 ... 256), while the
    # Fourier method's GMRES count stays nearly constant (5.32 ... 8.05)
    avg_b, avg_g = [], []
    for N in (16, 32, 64):
        f, g, _ = I.manufactured(N, N)
        _, s0, _, _ = O.solve(f, g, tau=2.0, tol=1e-10, eta=eta)
        with O.fd_bicg():
            _, s1, _, _ = O.solve(f, g, tau=2.0, tol=1e-10, eta=eta)
        avg_g.append(s0["gmres_iters"] / s0["newton_iters"])
        avg_b.append(s1["gmres_iters"] / s1["newton_iters"])
    assert avg_b[0] < avg_b[1] < avg_b[2] and avg_b[2] / avg_b[0] > 2.5
    assert max(avg_g) / min(avg_g) < 1.2
