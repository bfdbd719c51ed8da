"""Pins of the learned-warm-start oracle (oracle/warmstart.py, orc_fd_poisson,
orc_ws_features) against closed forms, the oracle's independent stencil and B-spline
routines, finite differences and a library bfloat16 conversion."""
import numpy as np
import pytest

import oracle as O
import oracle.warmstart as W
import ot_inputs as I

RNG = np.random.default_rng(11)


def smooth(N, M, amp=1.0, kmax=3, seed=0):
    rng = np.random.default_rng(seed)
    x, y = I.grid(N, M)
    u = np.zeros((N, M))
    for _ in range(5):
        k1, k2 = rng.integers(-kmax, kmax + 1, 2)
        u += rng.standard_normal() * np.cos(2 * np.pi * (k1 * x + k2 * y) + rng.random() * 6)
    return amp * u


@pytest.mark.parametrize("N,M", [(16, 24), (32, 32), (12, 20), (40, 8)])
def test_fd_poisson_inverts_the_stencil_laplacian(N, M):
    src = RNG.standard_normal((N, M))
    u = O.fd_poisson(src)
    d = O.derivatives(u)
    lap = d[2] + d[3]
    assert abs(u.mean()) < 1e-14
    assert np.abs(lap - (src - src.mean())).max() < 1e-11 * np.abs(src).max()
    assert np.abs(O.fd_poisson(np.full((N, M), 3.0))).max() < 1e-15


def test_fd_poisson_lowpass_on_single_modes():
    # a Fourier mode is an eigenfunction of both the stencil Laplacian and the filter
    N, M = 32, 48
    x, y = I.grid(N, M)
    for k1, k2 in ((1, 0), (3, -2), (12, 8), (24, 16), (0, 16)):
        mode = np.cos(2 * np.pi * (k1 * x + k2 * y))
        u = O.fd_poisson(mode, lowpass=True)
        d = O.derivatives(u)
        w = np.exp(-0.5 * ((k1 / (M / 4)) ** 2 + (k2 / (N / 4)) ** 2))
        assert np.abs(d[2] + d[3] - w * mode).max() < 1e-11
    src = RNG.standard_normal((N, M))
    assert np.abs(O.fd_poisson(src, lowpass=True)).max() < np.abs(O.fd_poisson(src)).max()


def test_features_with_uniform_target():
    # g = 1: G(T) = 1 (the B-spline reproduces constants), so log G, grad G vanish; the
    # Laplacian feature equals the Poisson source up to its mean
    N, M = 32, 48
    f, _ = W.normalise(I.blob_density(N, M, 3), np.ones((N, M)))
    g = np.ones((N, M))
    X, h, src = W.features(f, g)
    X = X.reshape(N, M, 16)
    hx, hy, hxx, hyy, hxy = O.derivatives(h)
    det = np.maximum((1 + hxx) * (1 + hyy) - hxy ** 2, W.FLOOR)
    assert np.abs(X[..., 0] - np.log(f)).max() < 1e-15
    assert np.abs(X[..., 1]).max() < 1e-15
    for k in (2, 10, 11, 12):
        assert np.abs(X[..., k]).max() < 1e-12, k
    assert np.abs(X[..., 3] - (np.log(f) - np.log(det))).max() < 1e-12
    assert np.abs(X[..., 4] - (src - src.mean())).max() < 1e-10
    assert np.abs(X[..., 5] - (hxx - hyy)).max() < 1e-14
    assert np.abs(X[..., 6] - 2 * hxy).max() < 1e-14
    assert np.abs(X[..., 7] - (hxx * hyy - hxy ** 2)).max() < 1e-14
    assert np.abs(X[..., 8] - 10 * hx).max() < 1e-14 and np.abs(X[..., 9] - 10 * hy).max() < 1e-14
    assert np.abs(X[..., 13] - ((hxx - hyy) ** 2 + 4 * hxy ** 2)).max() < 1e-14
    assert np.abs(X[..., 14] - X[..., 3] * X[..., 4]).max() < 1e-14
    assert np.all(X[..., 15] == 0)


def test_features_with_equal_densities():
    # f = g: h = 0, T = x, so G(T) = g at the nodes and every h-dependent feature is 0;
    # grad log G is the interpolant's gradient, close to the analytic one for a smooth g
    N, M = 64, 64
    x, y = I.grid(N, M)
    g = 1 + 0.3 * np.cos(2 * np.pi * x) * np.cos(2 * np.pi * y)
    X, h, src = W.features(g / g.mean(), g / g.mean())
    X = X.reshape(N, M, 16)
    gn = g / g.mean()
    assert np.abs(h).max() == 0.0
    for k in (0, 1, 2):
        assert np.abs(X[..., k] - np.log(gn)).max() < 1e-13
    for k in (3, 4, 5, 6, 7, 8, 9, 12, 13, 14):
        assert np.abs(X[..., k]).max() < 1e-13, k
    gx = -0.3 * 2 * np.pi * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    gy = -0.3 * 2 * np.pi * np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y)
    assert np.abs(X[..., 10] - 0.1 * gx / g).max() < 1e-4
    assert np.abs(X[..., 11] - 0.1 * gy / g).max() < 1e-4


def test_exact_source_recovers_the_potential():
    # with the exact correction s* (and no low-pass) h + P(s*) is phi* itself
    N, M = 48, 32
    f, g = W.normalise(*I.blob_pair(N, M, s=7))
    h, src = W.linear_potential(f, g)
    phi = smooth(N, M, amp=1e-3, seed=4)
    s = W.target(phi, h).reshape(N, M)
    u = O.fd_poisson(src + s)
    assert np.abs(u - (phi - phi.mean())).max() < 1e-12
    assert np.abs(h + O.fd_poisson(s) - (phi - phi.mean())).max() < 1e-12


def test_silu_and_its_derivative():
    z = np.linspace(-30, 30, 1001)
    assert np.all(np.abs(W.silu(np.array([0.0]))) == 0)
    assert np.abs(W.silu(np.array([40.0])) - 40.0).max() < 1e-12
    e = 1e-6
    fd = (W.silu(z + e) - W.silu(z - e)) / (2 * e)
    assert np.abs(fd - W.silu_grad(z)).max() < 1e-8


def test_forward_closed_form_with_zero_weights():
    p = np.zeros(W.N_PARAMS)
    W0, b0, W1, b1, W2, b2, w3, b3 = W.unpack(p)
    b2[:] = np.linspace(-2, 2, W.H)
    w3[:] = np.linspace(1, 3, W.H)
    b3[0] = 0.25
    y, _ = W.mlp_forward(p, RNG.standard_normal((7, 16)))
    expect = 0.25 + np.sum(w3 * b2 / (1 + np.exp(-b2)))
    assert np.abs(y - expect).max() < 1e-12


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(5)
    p = I.ws_init_params(9).astype(np.float64)
    p[-W.H - 1:] *= 10.0  # a larger output layer so that every term matters
    X = rng.standard_normal((40, 16))
    t = rng.standard_normal(40)
    loss, g = W.loss_and_grad(p, X, t)
    idx = np.concatenate([rng.choice(W.N_PARAMS - W.H - 1, 48, replace=False),
                          np.arange(W.N_PARAMS - W.H - 1, W.N_PARAMS, 16), [W.N_PARAMS - 1]])
    for i in idx:
        e = 1e-6
        q = p.copy()
        q[i] += e
        lp = W.loss_and_grad(q, X, t)[0]
        q[i] -= 2 * e
        lm = W.loss_and_grad(q, X, t)[0]
        fd = (lp - lm) / (2 * e)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_adam_first_steps_closed_form():
    # bias correction makes the first step -lr g / (|g| + eps); with a constant gradient
    # every later step is the same
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p0 = np.array([1.0, 2.0, 3.0, 4.0])
    m = v = np.zeros(4)
    p1, m, v = W.adam_step(p0, m, v, g, 1, 0.01)
    assert np.abs(p1 - (p0 - 0.01 * g / (np.abs(g) + W.ADAM_EPS))).max() < 1e-15
    p2, m, v = W.adam_step(p1, m, v, g, 2, 0.01)
    assert np.abs((p2 - p1) - (p1 - p0)).max() < 1e-13


def test_bf16_rounding_matches_library_conversion():
    torch = pytest.importorskip("torch")
    x = np.concatenate([RNG.standard_normal(5000) * 10.0 ** RNG.integers(-6, 6, 5000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -1.0 - 2 ** -8, 0.0, 65504.0]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(W.bf16_round(x), ref)
    assert W.bf16_round(np.array([1.0 + 2 ** -8]))[0] == 1.0          # tie to even
    assert W.bf16_round(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6


def test_admissible_scale():
    N, M = 32, 32
    u = smooth(N, M, amp=1.0, kmax=2, seed=2)
    _, _, uxx, uyy, uxy = O.derivatives(u)
    a = W.admissible_scale(u)
    det = lambda s: ((1 + s * uxx) * (1 + s * uyy) - (s * uxy) ** 2).min()
    if a > 0:
        assert det(a) > 0
    if a < 1.0:
        assert det(2 * a if a > 0 else W.ALPHAS[-1]) <= 0
    assert W.admissible_scale(np.zeros((N, M))) == 1.0


def test_batch_rows_in_range_and_deterministic():
    a = I.ws_batch_rows(3, 7, 1000, 4096)
    assert a.dtype == np.int64 and a.min() >= 0 and a.max() < 1000
    assert np.array_equal(a, I.ws_batch_rows(3, 7, 1000, 4096))
    assert not np.array_equal(a, I.ws_batch_rows(3, 8, 1000, 4096))
