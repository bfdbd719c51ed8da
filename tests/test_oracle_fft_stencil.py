"""Pins of the oracle's Fourier transform, finite-difference stencils and B-spline
interpolation against definitions, closed forms and library routines (no GPU)."""
import numpy as np
import pytest

import oracle as O

RNG = np.random.default_rng(1234)


@pytest.mark.parametrize("shape", [(8, 8), (12, 12), (16, 24), (24, 24), (32, 32), (6, 10)])
def test_fft2_matches_bruteforce_dft(shape):
    x = RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)
    for inv in (False, True):
        a = O.fft2(x, inverse=inv)
        b = O.dft2(x, inverse=inv)
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


@pytest.mark.parametrize("shape", [(8, 8), (12, 20), (7, 9)])
def test_dft_definition_matches_numpy(shape):
    # the brute-force DFT is the definition; numpy's FFT pins its sign convention
    x = RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)
    np.testing.assert_allclose(O.dft2(x), np.fft.fft2(x), atol=1e-11)
    np.testing.assert_allclose(O.dft2(x, inverse=True), np.fft.ifft2(x) * x.size, atol=1e-11)


@pytest.mark.parametrize("L", [1, 2, 3, 7, 15, 60, 96, 128, 192, 1536])
def test_fft1_lengths_match_numpy(L):
    x = RNG.standard_normal(L) + 1j * RNG.standard_normal(L)
    np.testing.assert_allclose(O.fft1(x), np.fft.fft(x), atol=1e-10 * max(1, L))


def test_fft2_large_matches_numpy():
    x = RNG.standard_normal((192, 256))
    np.testing.assert_allclose(O.fft2(x), np.fft.fft2(x), atol=1e-9)


# ----------------------------------------------------------------------------------------
def _stencil_symbols(theta):
    """Fourier symbols (times h and h^2) of the 4th-order centred first and second
    differences: D1 e^{i k x} = i (8 sin t - sin 2t)/(6h) e^{ikx},
    D2 e^{ikx} = (-2 cos 2t + 32 cos t - 30)/(12 h^2) e^{ikx}."""
    s1 = (8 * np.sin(theta) - np.sin(2 * theta)) / 6.0
    s2 = (-2 * np.cos(2 * theta) + 32 * np.cos(theta) - 30) / 12.0
    return s1, s2


@pytest.mark.parametrize("N,M,kx,ky", [(16, 16, 1, 2), (16, 32, 3, 5), (24, 12, 5, 2)])
def test_stencils_exact_on_fourier_modes(N, M, kx, ky):
    y, x = np.meshgrid(np.arange(N) / N, np.arange(M) / M, indexing="ij")
    tx, ty = 2 * np.pi * kx / M, 2 * np.pi * ky / N
    u = np.sin(2 * np.pi * kx * x) * np.cos(2 * np.pi * ky * y)
    ux, uy, uxx, uyy, uxy = O.derivatives(u)
    s1x, s2x = _stencil_symbols(tx)
    s1y, s2y = _stencil_symbols(ty)
    cx, sx = np.cos(2 * np.pi * kx * x), np.sin(2 * np.pi * kx * x)
    cy, sy = np.cos(2 * np.pi * ky * y), np.sin(2 * np.pi * ky * y)
    np.testing.assert_allclose(ux, s1x * M * cx * cy, atol=1e-11 * M)
    np.testing.assert_allclose(uy, -s1y * N * sx * sy, atol=1e-11 * N)
    np.testing.assert_allclose(uxx, s2x * M * M * sx * cy, atol=1e-10 * M * M)
    np.testing.assert_allclose(uyy, s2y * N * N * sx * cy, atol=1e-10 * N * N)
    np.testing.assert_allclose(uxy, -s1x * s1y * M * N * cx * sy, atol=1e-10 * M * N)


def test_stencils_fourth_order():
    errs = []
    for N in (16, 32, 64):
        y, x = np.meshgrid(np.arange(N) / N, np.arange(N) / N, indexing="ij")
        a, b = 2 * np.pi * x, 2 * np.pi * y
        u = np.exp(np.sin(a) + 0.5 * np.cos(b))
        ex = [u * 2 * np.pi * np.cos(a), u * -np.pi * np.sin(b),
              u * (2 * np.pi) ** 2 * (np.cos(a) ** 2 - np.sin(a)),
              u * (2 * np.pi) ** 2 * (0.25 * np.sin(b) ** 2 - 0.5 * np.cos(b)),
              u * 2 * np.pi * np.cos(a) * -np.pi * np.sin(b)]
        d = O.derivatives(u)
        errs.append([np.abs(d[q] - ex[q]).max() / np.abs(ex[q]).max() for q in range(5)])
    errs = np.array(errs)
    orders = np.log2(errs[:-1] / errs[1:])
    assert (orders > 3.7).all() and (orders < 4.5).all(), orders


# ----------------------------------------------------------------------------------------
def test_bspline_interpolates_nodes():
    g = 1 + RNG.random((12, 20))
    c = O.bspline_coeffs(g)
    N, M = g.shape
    yy, xx = np.meshgrid(np.arange(N) / N, np.arange(M) / M, indexing="ij")
    v, _, _ = O.bspline_eval(c, xx.ravel(), yy.ravel())
    np.testing.assert_allclose(v.reshape(N, M), g, atol=1e-13)


def test_bspline_constant_and_separable():
    N, M = 10, 14
    c = O.bspline_coeffs(np.full((N, M), 2.5))
    np.testing.assert_allclose(c, 2.5, atol=1e-14)
    gx = 1 + RNG.random(M)
    gy = 1 + RNG.random(N)
    c2 = O.bspline_coeffs(np.outer(gy, gx))
    cx = O.bspline_coeffs(np.tile(gx, (4, 1)))[0]
    cy = O.bspline_coeffs(np.tile(gy, (4, 1)))[0]
    np.testing.assert_allclose(c2, np.outer(cy, cx), atol=1e-12)


def test_bspline_matches_scipy_periodic_cubic():
    interp = pytest.importorskip("scipy.interpolate")
    M = 16
    gx = 1 + 0.5 * np.sin(2 * np.pi * np.arange(M) / M) + 0.2 * RNG.random(M)
    g = np.tile(gx, (6, 1))
    c = O.bspline_coeffs(g)
    knots = np.arange(M + 1) / M
    spl = interp.make_interp_spline(knots, np.append(gx, gx[0]), k=3, bc_type="periodic")
    xs = RNG.random(40)
    ys = RNG.random(40)
    v, dx, dy = O.bspline_eval(c, xs, ys)
    np.testing.assert_allclose(v, spl(xs), atol=1e-12)
    np.testing.assert_allclose(dx, spl(xs, 1), atol=1e-10)
    np.testing.assert_allclose(dy, 0.0, atol=1e-10)


def test_bspline_fourth_order_and_gradient():
    def gfun(x, y):
        return 1 + 0.3 * np.sin(2 * np.pi * x) * np.cos(4 * np.pi * y)

    pts = RNG.random((2, 50))
    errs = []
    for N in (16, 32, 64):
        yy, xx = np.meshgrid(np.arange(N) / N, np.arange(N) / N, indexing="ij")
        c = O.bspline_coeffs(gfun(xx, yy))
        v, dx, dy = O.bspline_eval(c, pts[0], pts[1])
        errs.append(np.abs(v - gfun(pts[0], pts[1])).max())
        # gradient equals the derivative of the interpolant itself
        e = 1e-6
        vp, _, _ = O.bspline_eval(c, pts[0] + e, pts[1])
        vm, _, _ = O.bspline_eval(c, pts[0] - e, pts[1])
        np.testing.assert_allclose(dx, (vp - vm) / (2 * e), atol=1e-6)
        vp, _, _ = O.bspline_eval(c, pts[0], pts[1] + e)
        vm, _, _ = O.bspline_eval(c, pts[0], pts[1] - e)
        np.testing.assert_allclose(dy, (vp - vm) / (2 * e), atol=1e-6)
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (orders > 3.6).all(), orders
