"""FP64 oracle of the learned warm start (TEST INFRASTRUCTURE ONLY: only tests/, the smoke
check and the benchmark's CPU-baseline leg may import it).

The paper starts Newton from u0 = 0 and notes only that the iteration needs an admissible
(convex) start, det(I + D^2 u0) > 0 (Theorem convproof).  The warm start here is a learned
map (f, g) -> u0 built on the paper's quantities:

  1. h   = P(log f - log g), P = the mean-zero inverse of the 4th-order stencil Laplacian
           (the linearisation of log det(I + D^2 u) + log G(x + grad u) = log f about u = 0);
  2. X   = 16 per-point features at h (``oracle.ws_features``: the Monge-Ampere log-residual
           at h, the Hessian of h, the displacement grad h, grad log G at T = x + grad h ...);
  3. s   = a per-point MLP 16 -> 128 -> 128 -> 128 -> 1 (SiLU) of X, trained to predict the
           source correction s* = Lap_h(phi* - h) of the converged potential phi*;
  4. u0  = alpha (h + P(G s)), G the Gaussian low-pass exp(-((k1/(M/4))^2 + (k2/(N/4))^2)/2)
           on the network's output, alpha the largest of 1, 1/2, 1/4, 1/8 with
           det(I + alpha D^2 u0) > 0 everywhere (else 0: the zero start).

Without the low-pass, s = s* would return phi* itself.  The low-pass keeps the network's
pointwise errors out of the high frequencies, where the damped iteration's contraction
(spectral operator against stencil residual) is slowest.  Network parameters are one flat vector:
W0[H,16], b0[H], W1[H,H], b1[H], W2[H,H], b2[H], w3[H], b3[1] (row-major, H = 128).

Inference on the GPU runs the matrix products in BF16 with FP32 accumulation: the network
input X and the hidden activations a0, a1 (the MMA operands) and the weights W0, W1, W2 are
rounded to BF16 (round to nearest even), everything else stays FP32.  ``mlp_forward(...,
bf16=True)`` applies exactly these roundings, in FP64 otherwise.
"""
import numpy as np

import oracle as O

K, H = 16, 128
N_PARAMS = H * K + H + 2 * (H * H + H) + H + 1
FLOOR = 1e-3
ALPHAS = (1.0, 0.5, 0.25, 0.125)
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def unpack(params):
    """Views (W0, b0, W1, b1, W2, b2, w3, b3) of the flat parameter vector."""
    p = np.asarray(params, dtype=np.float64)
    assert p.size == N_PARAMS
    out, o = [], 0
    for shape in ((H, K), (H,), (H, H), (H,), (H, H), (H,), (H,), (1,)):
        n = int(np.prod(shape))
        out.append(p[o:o + n].reshape(shape))
        o += n
    return out


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64.  The value is
    first rounded to float32 (as the GPU holds it), then the low 16 bits of the float32
    pattern are rounded away."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = a.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = ((b + 0x7FFF + lsb) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64).reshape(a.shape)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def mlp_forward(params, X, bf16=False):
    """Network output y (rows,) for features X (rows, 16); also the cache for backward."""
    W0, b0, W1, b1, W2, b2, w3, b3 = unpack(params)
    r = bf16_round if bf16 else (lambda a: a)
    X = np.asarray(X, dtype=np.float64).reshape(-1, K)
    z0 = r(X) @ r(W0).T + b0
    a0 = silu(z0)
    z1 = r(a0) @ r(W1).T + b1
    a1 = silu(z1)
    z2 = r(a1) @ r(W2).T + b2
    a2 = silu(z2)
    y = a2 @ w3 + b3[0]
    return y, (X, z0, a0, z1, a1, z2, a2)


def loss_and_grad(params, X, t):
    """Mean squared error of the FP64 network on (X, t) and its gradient (flat), by
    reverse-mode differentiation of mlp_forward."""
    W0, b0, W1, b1, W2, b2, w3, b3 = unpack(params)
    y, (X, z0, a0, z1, a1, z2, a2) = mlp_forward(params, X)
    t = np.asarray(t, dtype=np.float64).reshape(-1)
    B = y.size
    e = y - t
    loss = float(np.mean(e * e))
    dy = 2.0 * e / B
    g_w3 = a2.T @ dy
    g_b3 = np.array([dy.sum()])
    dz2 = np.outer(dy, w3) * silu_grad(z2)
    g_W2, g_b2 = dz2.T @ a1, dz2.sum(0)
    dz1 = (dz2 @ W2) * silu_grad(z1)
    g_W1, g_b1 = dz1.T @ a0, dz1.sum(0)
    dz0 = (dz1 @ W1) * silu_grad(z0)
    g_W0, g_b0 = dz0.T @ X, dz0.sum(0)
    grad = np.concatenate([a.reshape(-1) for a in
                           (g_W0, g_b0, g_W1, g_b1, g_W2, g_b2, g_w3, g_b3)])
    return loss, grad


def adam_step(params, m, v, grad, t, lr):
    """One Adam update (Kingma & Ba, Algorithm 1) at step t >= 1; returns new (params, m, v)."""
    m = ADAM_B1 * m + (1.0 - ADAM_B1) * grad
    v = ADAM_B2 * v + (1.0 - ADAM_B2) * grad * grad
    mh = m / (1.0 - ADAM_B1 ** t)
    vh = v / (1.0 - ADAM_B2 ** t)
    return params - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v


def normalise(f, g):
    """The solver's input translation (Eq. translation): d <- d - mean(d) + 1."""
    f = np.asarray(f, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    return f - f.mean() + 1.0, g - g.mean() + 1.0


def linear_potential(f, g):
    """(h, src): src = log f - log g and h = P(src)."""
    src = np.log(f) - np.log(g)
    return O.fd_poisson(src), src


def features(f, g):
    """(X (N*M, 16), h, src) for normalised f, g."""
    h, src = linear_potential(f, g)
    X = O.ws_features(f, g, O.bspline_coeffs(g), h)
    return X.reshape(-1, K), h, src


def target(phi_star, h):
    """s* = (D_xx + D_yy)(phi* - h), per point."""
    d = O.derivatives(np.asarray(phi_star) - h)
    return (d[2] + d[3]).reshape(-1)


def admissible_scale(u):
    """Largest alpha in ALPHAS with det(I + alpha D^2 u) > 0 at every point, else 0."""
    _, _, uxx, uyy, uxy = O.derivatives(u)
    for a in ALPHAS:
        if np.min((1.0 + a * uxx) * (1.0 + a * uyy) - (a * uxy) ** 2) > 0.0:
            return a
    return 0.0


def predict(params, f, g, bf16=True):
    """(u0, alpha, s): the warm start for the raw densities f, g (translated here)."""
    f, g = normalise(f, g)
    X, h, src = features(f, g)
    s, _ = mlp_forward(params, X, bf16=bf16)
    u = h + O.fd_poisson(s.reshape(f.shape), lowpass=True)
    a = admissible_scale(u)
    return a * u, a, s.reshape(f.shape)
