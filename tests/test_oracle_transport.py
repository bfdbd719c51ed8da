"""Pins of the oracle's transport outputs (Sec. 5.2: d(f, g) = int |grad u|^2 f dx and the
divergence map u_xx + u_yy), against closed forms built from the stencils' Fourier symbols
rather than from the stencil taps the oracle applies."""
import numpy as np
import pytest

import oracle as O
import ot_inputs as I


def s1(k, L):
    # symbol of the 4th-order first-difference stencil on L points: (8 sin t - sin 2t) L / 6
    t = 2 * np.pi * k / L
    return (8 * np.sin(t) - np.sin(2 * t)) * L / 6


def s2(k, L):
    # symbol of the 4th-order second-difference stencil: (-2 cos 2t + 32 cos t - 30) L^2 / 12
    t = 2 * np.pi * k / L
    return (-2 * np.cos(2 * t) + 32 * np.cos(t) - 30) * L * L / 12


@pytest.mark.parametrize("N,M,k1,k2", [(16, 16, 1, 1), (24, 48, 2, 3), (32, 20, 3, 1)])
def test_single_mode_closed_form(N, M, k1, k2):
    # u = A sin(2 pi k1 x) sin(2 pi k2 y): the stencils act on each factor by their symbols,
    # and the grid mean of cos^2 sin^2 (k < L/2) is 1/4
    A = 1e-3
    x, y = np.arange(M) / M, np.arange(N) / N
    sx, cx = np.sin(2 * np.pi * k1 * x), np.cos(2 * np.pi * k1 * x)
    sy, cy = np.sin(2 * np.pi * k2 * y), np.cos(2 * np.pi * k2 * y)
    u = A * np.outer(sy, sx)
    d, div = O.transport_outputs(np.ones((N, M)), u)
    d_ref = A * A * (s1(k1, M) ** 2 + s1(k2, N) ** 2) / 4
    assert abs(d - d_ref) <= 1e-12 * d_ref
    div_ref = (s2(k1, M) + s2(k2, N)) * u
    assert np.abs(div - div_ref).max() <= 1e-10 * np.abs(div_ref).max()
    # a weight 1 + cos(2 pi 5 x) adds the grid mean of cos(2 pi 5 x) times the squared
    # factors, whose frequencies (0, 2 k1) differ from 5: d is unchanged
    f = 1 + np.outer(np.ones(N), np.cos(2 * np.pi * 5 * x)) if M > 10 else np.ones((N, M))
    d2, _ = O.transport_outputs(f, u)
    assert abs(d2 - d_ref) <= 1e-12 * d_ref


def test_linear_in_f_and_zero_potential():
    f, g = I.blob_pair(32, 48, s=7)
    u = 1e-3 * np.random.default_rng(3).standard_normal((32, 48))
    d1, div1 = O.transport_outputs(f, u)
    d2, div2 = O.transport_outputs(2.5 * f, u)
    assert abs(d2 - 2.5 * d1) <= 1e-14 * d2
    assert np.array_equal(div1, div2)
    d0, div0 = O.transport_outputs(f, np.zeros((32, 48)))
    assert d0 == 0.0 and not div0.any()


def test_manufactured_map_distance():
    # the manufactured potential phi* = A sin 2 pi x sin 2 pi y with f = g(T) det(I + D^2 phi*):
    # d(f, g) = int |grad phi*|^2 f dx with the analytic gradient, by the grid rule on a fine
    # grid (spectrally accurate for this smooth periodic integrand); the stencil value
    # converges to it at order 4
    A = I.MANUFACTURED_A
    n = 512
    fN, _, _ = I.manufactured(n, n)
    xs = np.arange(n) / n
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    ux = 2 * np.pi * A * np.cos(2 * np.pi * X) * np.sin(2 * np.pi * Y)
    uy = 2 * np.pi * A * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)
    d_exact = float(np.mean((ux ** 2 + uy ** 2) * fN))
    errs = []
    for N in (16, 32, 64):
        f, _, ph = I.manufactured(N, N)
        d, _ = O.transport_outputs(f, ph)
        errs.append(abs(d - d_exact))
    assert errs[2] <= 1e-5 * d_exact
    assert errs[0] / errs[1] > 10 and errs[1] / errs[2] > 10  # order ~4 (factor 16)
