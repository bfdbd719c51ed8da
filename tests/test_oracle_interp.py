"""Pins of the oracle's nearest-node and bilinear interpolation of g (Sec. 4 intro:
closest-neighbour interpolation, used for the images of Sec. 5.2; linear interpolation, used
in Sec. 5.3).  Reading: G(T) interpolates the grid values of g and grad G(T) interpolates, by
the same rule, the grid gradient of g by the 4th-order centred differences of Sec. 4."""
import numpy as np
import pytest

import oracle as O
import ot_inputs as I


def smooth(N, M, amp, seed):
    rng = np.random.default_rng(seed)
    x, y = I.grid(N, M)
    u = np.zeros((N, M))
    for _ in range(4):
        k1, k2 = rng.integers(-2, 3, 2)
        u += rng.standard_normal() * np.cos(2 * np.pi * (k1 * x + k2 * y) + rng.random())
    return amp * u


@pytest.mark.parametrize("mode", ["bilinear", "nearest"])
def test_undisplaced_points_take_the_grid_values(mode):
    # u = 0: every displaced point is a node, so G = g and grad G = the grid gradient there
    N, M = 24, 32
    f = I.blob_density(N, M, 1)
    g = I.blob_density(N, M, 2)
    gx, gy, _, _, _ = O.derivatives(g)
    with O.interpolation(mode):
        c = O.interp_coeffs(g)
        F, coef, s = O.residual(f, c, np.zeros((N, M)))
    assert np.array_equal(c, g)
    assert np.array_equal(coef[0], g) and np.array_equal(coef[2], g) and not coef[1].any()
    assert np.array_equal(coef[3], gx) and np.array_equal(coef[4], gy)
    assert np.abs(F - (f - (g - g.mean() + 1.0))).max() <= 1e-14


def test_bilinear_is_exact_on_bilinear_data():
    # g = a + b x + c y + d x y on the grid: away from the periodic wrap the interpolant at a
    # displaced point is the function itself, and the interpolated grid gradient (exact for
    # this g at nodes two or more away from the wrap) is its gradient (b + d y, c + d x)
    N = M = 64
    x, y = I.grid(N, M)
    a, b, c_, d = 2.0, 0.3, -0.2, 0.5
    g = a + b * x + c_ * y + d * x * y
    u = smooth(N, M, 2e-4, 3)
    ux, uy, uxx, uyy, uxy = O.derivatives(u)
    with O.interpolation("bilinear"):
        _, coef, _ = O.residual(np.ones((N, M)), g, u)
    X, Y = x + ux, y + uy
    det = (1 + uxx) * (1 + uyy) - uxy * uxy
    inner = (x > 3.0 / M) & (x < 1 - 4.0 / M) & (y > 3.0 / N) & (y < 1 - 4.0 / N)
    G = coef[0] / (1 + uyy)
    assert np.abs(G - (a + b * X + c_ * Y + d * X * Y))[inner].max() <= 1e-13
    assert np.abs(coef[3] / det - (b + d * Y))[inner].max() <= 1e-12
    assert np.abs(coef[4] / det - (c_ + d * X))[inner].max() <= 1e-12


def test_nearest_takes_the_closest_node():
    # displacements below half a cell keep every point at its own node; a displacement of
    # one cell in x (plus less than half a cell) moves it to the next node
    N = M = 32
    f = I.blob_density(N, M, 5)
    g = I.blob_density(N, M, 6)
    gx, gy, _, _, _ = O.derivatives(g)
    u = smooth(N, M, 1e-4, 7)  # |grad u| << h / 2
    _, _, uxx, uyy, uxy = O.derivatives(u)
    with O.interpolation("nearest"):
        _, coef, _ = O.residual(f, g, u)
    assert np.abs(coef[0] / (1 + uyy) - g).max() <= 1e-14
    det = (1 + uxx) * (1 + uyy) - uxy * uxy
    assert np.abs(coef[3] / det - gx).max() <= 1e-12
    # u = x / M sin-free shift is not periodic; use u = (1.2 / M) sin(2 pi y) / (2 pi) ... in
    # x only: a periodic potential whose x-derivative is exactly one cell on a row
    x, y = I.grid(N, M)
    v = (1.2 / M) * np.sin(2 * np.pi * x) / (2 * np.pi * np.cos(0.0))
    vx, _, vxx, vyy, vxy = O.derivatives(v)
    with O.interpolation("nearest"):
        _, coef, _ = O.residual(f, g, v)
    Gv = coef[0] / (1 + vyy)
    jn = np.floor(np.arange(M)[None, :] + M * vx + 0.5).astype(int) % M
    assert np.array_equal(Gv, g[np.arange(N)[:, None], jn] * (1 + vyy) / (1 + vyy))


def test_manufactured_residual_and_root():
    # At the manufactured phi* the displacement |grad phi*| <= 0.02 / (2 pi) is below half a
    # cell for N <= 128, so the nearest node of x + grad phi* is x itself and F(phi*) is the
    # closed form f - (g det - mean + 1) with the stencils' det; the bilinear interpolant errs
    # by about |grad phi*| h |g''| / 2, first order in h at a fixed sub-cell displacement.
    # The roots of both discrete problems lie within the inverse's size (Sec. 5.1: about
    # 0.03) times max|F(phi*)| of phi*.
    res = {"bilinear": [], "nearest": []}
    for N in (16, 32, 64, 128):
        f, g, phi = I.manufactured(N, N)
        fn, gn = f - f.mean() + 1.0, g - g.mean() + 1.0
        _, _, uxx, uyy, uxy = O.derivatives(phi)
        det = (1 + uxx) * (1 + uyy) - uxy * uxy
        for mode in res:
            with O.interpolation(mode):
                F, _, s = O.residual(fn, O.interp_coeffs(gn), phi)
            res[mode].append(s["res_inf"])
            if mode == "nearest":
                Fc = fn - (gn * det - np.mean(gn * det) + 1.0)
                assert np.abs(F - Fc).max() <= 1e-13
    rates = np.log2(np.array(res["bilinear"][:-1]) / np.array(res["bilinear"][1:]))
    assert 0.8 <= rates.min() and rates.max() <= 1.4, rates
    for mode in res:
        N = 32
        f, g, phi = I.manufactured(N, N)
        with O.interpolation(mode):
            u, st, _, _ = O.solve(f, g, tau=2.0, tol=1e-12, eta=1e-6, max_newton=300)
        assert st["status"] == 0
        assert np.abs(u - phi).max() <= 0.1 * res[mode][1], (mode, np.abs(u - phi).max())
