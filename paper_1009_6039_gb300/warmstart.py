"""Training driver of the learned warm start (OT_OPT_WARM_START = 2).

train() solves the given density pairs with the library (zero start, mixed precision),
computes each pair's features and target s* = (D_xx + D_yy)(phi* - h) with ot_ws_features,
and fits the network with the library's Adam trainer (FP32 forward/backward kernels) on
random minibatches of grid points.  Everything runs on the current CUDA device; the result
is the FP32 parameter vector for Plan.set_weights / ot_ws_save_weights.
"""
import math

import numpy as np

from . import Plan, Trainer, ot_ws_param_count

K, H = 16, 128


def init_params(seed):
    """Uniform +-1/sqrt(fan_in) weights (output layer x 0.1), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((H, K), (H, H), (H, H)):
        parts += [rng.uniform(-1, 1, fan_out * fan_in) / math.sqrt(fan_in), np.zeros(fan_out)]
    parts += [rng.uniform(-1, 1, H) * 0.1 / math.sqrt(H), np.zeros(1)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == ot_ws_param_count()
    return p


def training_data(pairs, N, M, tau=2.0, tol=1e-8, eta=0.1, max_newton=400, symbols=0):
    """(X, t): features (n*N*M x 16) and targets (n*N*M) as float32 CUDA tensors, from the
    converged potentials of the pairs (numpy float64 (N, M) arrays); pairs whose solve does
    not converge are skipped.  The solver settings change the path, not the root (the
    target): symbols = 1 (the stencils' symbols) converges in fewer steps."""
    import torch
    P = N * M
    plan = Plan(N, M, tau=tau, tol=tol, eta=eta, precision="mixed", max_newton=max_newton,
                symbols=symbols)
    Xs, ts = [], []
    for f, g in pairs:
        fd = torch.from_numpy(np.ascontiguousarray(f, dtype=np.float64)).cuda()
        gd = torch.from_numpy(np.ascontiguousarray(g, dtype=np.float64)).cuda()
        phi = torch.zeros((N, M), dtype=torch.float64, device="cuda")
        rc, st = plan.solve(fd, gd, phi)
        if rc != 0:
            continue
        X = torch.empty((P, K), dtype=torch.float32, device="cuda")
        t = torch.empty(P, dtype=torch.float32, device="cuda")
        plan.ws_features(fd, gd, X, t, phi_star=phi)
        Xs.append(X)
        ts.append(t)
    plan.close()
    if not Xs:
        raise RuntimeError("no training pair converged")
    return torch.cat(Xs), torch.cat(ts)


def fit(X, t, steps=2000, batch=16384, lr=2e-3, seed=0, params=None):
    """Adam on the mean squared error over random minibatches of rows of (X, t), cosine
    learning-rate decay; the target is scaled to unit RMS during training and the output
    layer rescaled after.  Returns the FP32 parameters."""
    import torch
    rms = float(torch.sqrt(torch.mean(t.double() ** 2)).item()) or 1.0
    ts = (t / rms).contiguous()
    p0 = init_params(seed) if params is None else np.array(params, dtype=np.float32)
    if params is not None:
        p0[-H - 1:] /= rms
    tr = Trainer(batch, p0)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    n = X.shape[0]
    for s in range(steps):
        idx = torch.randint(0, n, (batch,), device="cuda", generator=gen, dtype=torch.int64)
        lr_s = lr * 0.5 * (1.0 + math.cos(math.pi * s / steps)) + 1e-6
        tr.step(X, ts, idx, lr_s)
    p = tr.params()
    tr.close()
    p[-H - 1:] *= rms
    return p


def train(pairs, N, M, steps=2000, batch=16384, lr=2e-3, seed=0, tau=2.0, tol=1e-8, eta=0.1):
    """Solve the pairs, build the training set, fit the network; returns the parameters."""
    X, t = training_data(pairs, N, M, tau=tau, tol=tol, eta=eta)
    return fit(X, t, steps=steps, batch=batch, lr=lr, seed=seed)
