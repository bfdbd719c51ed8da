"""GPU parity of the learned warm start against its FP64 oracle (oracle/warmstart.py), and
the gain of a trained network over the zero start.

Tolerances:
  - FD Poisson solve: FP64 mode (FP64 FFTs) 1e-12 of the result's scale; mixed mode
    (FP32 forward transforms, division and inverse transforms in double-float) 5e-6: the
    forward transforms' FP32 round-off, ~2^-24 sqrt(log2 P) relative to the source's
    coefficients, passes through the division by the Laplacian's eigenvalues as a relative
    error of the same size in the result (a few 1e-7), plus the FP32 eigenvalues and
    low-pass factors (1e-7 relative).
  - Features (FP64 stencils and interpolation, FP32 logarithms, stored as FP32): 1e-5 of
    each feature's scale (FP32 logf and storage rounding, a few 1e-7 relative, plus FP64
    stencil round-off amplified by M^2); the two features holding log det(I + D^2 h) are
    weighted by det (clamped to [1e-3, 1]), since an error in det enters them divided by
    det.
  - Network on the tensor cores vs the oracle with the same BF16 roundings: FP32 instead of
    FP64 accumulation and __expf differ by ~1e-6 relative; where that moves a value across a
    BF16 rounding boundary the activation changes by one BF16 ulp (2^-8 relative), so single
    outputs may move by ~1e-3 of the output scale and the mean by much less.
  - Gradient (FP32 sums over 4096 rows): 1e-4 of the largest gradient of each layer.
"""
import numpy as np
import pytest

import oracle as O
import oracle.warmstart as W
import ot_inputs as I
from gpu_util import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ot():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1009_6039_gb300 as m
    return m


def tdev32(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def random_params(seed, scale=1.0):
    p = I.ws_init_params(seed).astype(np.float64)
    rng = np.random.default_rng(seed)
    p[-W.H - 1:] *= 10.0 * scale
    p[W.H * W.K:W.H * W.K + W.H] = 0.3 * rng.standard_normal(W.H)  # nonzero b0
    return p.astype(np.float32)


@pytest.mark.parametrize("N,M", [(16, 24), (64, 96), (256, 256), (12, 512)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("lowpass", [False, True])
def test_fd_poisson(ot, N, M, prec, lowpass):
    _check_fd_poisson(ot, N, M, prec, lowpass)


@pytest.mark.parametrize("N,M", [(1024, 512), (256, 2048), (2048, 64)])
@pytest.mark.parametrize("lowpass", [False, True])
def test_fd_poisson_on_pairs(ot, N, M, lowpass):
    # the mixed mode's double-float passes on column / row pairs (columns of 256 .. 2048
    # points, rows of 512 .. 2048 points)
    _check_fd_poisson(ot, N, M, "mixed", lowpass)


def _check_fd_poisson(ot, N, M, prec, lowpass):
    src = np.random.default_rng(N * M).standard_normal((N, M))
    p = ot.Plan(N, M, precision=prec)
    u = dev(np.zeros((N, M)))
    p.ws_poisson(dev(src), u, lowpass=lowpass)
    ref = O.fd_poisson(src, lowpass=lowpass)
    rel = 1e-12 if prec == "fp64" else 5e-6
    assert np.abs(u.cpu().numpy() - ref).max() <= rel * np.abs(ref).max()
    p.close()


@pytest.mark.parametrize("N,M", [(32, 48), (128, 128), (192, 384)])
def test_features_and_target(ot, N, M):
    import torch
    f, g = I.blob_pair(N, M, s=21)
    fn, gn = W.normalise(f, g)
    X_ref, h, _ = W.features(fn, gn)
    phi = 1e-3 * np.cos(2 * np.pi * I.grid(N, M)[0]) * np.sin(4 * np.pi * I.grid(N, M)[1])
    t_ref = W.target(phi, h)
    p = ot.Plan(N, M, precision="mixed")
    X = torch.zeros((N * M, 16), dtype=torch.float32, device="cuda")
    t = torch.zeros(N * M, dtype=torch.float32, device="cuda")
    p.ws_features(dev(f), dev(g), X, t, phi_star=dev(phi))
    Xg = X.cpu().numpy()
    # features 3 (r = log f - log G - log det) and 14 (r times the Laplacian of h) carry
    # log max(det, 1e-3), det = det(I + D^2 h) = 1 + X4 + X7, whose error is the error of det
    # over det: where h is close to losing convexity the (FP32-forward) error of h is
    # amplified by up to 1e3, so those two are compared weighted by the clamped det
    det = np.clip(1.0 + X_ref[:, 4] + X_ref[:, 7], 1e-3, 1.0)
    for k in range(16):
        scale = np.abs(X_ref[:, k]).max() + 1e-30
        wk = det if k in (3, 14) else 1.0
        assert np.max(np.abs(Xg[:, k] - X_ref[:, k]) * wk) <= 1e-5 * max(scale, 1e-3), k
    assert np.abs(t.cpu().numpy() - t_ref).max() <= 1e-5 * np.abs(t_ref).max()
    p.close()


@pytest.mark.parametrize("rows", [1, 127, 128, 1000, 128 * 311 + 77])
def test_network_tensor_cores_match_oracle(ot, rows):
    import torch
    params = random_params(3)
    rng = np.random.default_rng(rows)
    X = rng.standard_normal((rows, 16)).astype(np.float32)
    X[:, 15] = 0.0
    p = ot.Plan(16, 16, precision="mixed").set_weights(params)
    out = torch.zeros(rows, dtype=torch.float32, device="cuda")
    p.ws_mlp_forward(tdev32(X), out)
    y_ref, _ = W.mlp_forward(params.astype(np.float64), X.astype(np.float64), bf16=True)
    y = out.cpu().numpy()
    scale = np.abs(y_ref).max()
    assert np.all(np.isfinite(y))
    assert np.abs(y - y_ref).max() <= 2e-3 * scale
    assert np.abs(y - y_ref).mean() <= 2e-4 * scale
    p.close()


def test_network_full_grid_sampled(ot):
    # the launch the 1024^2 solve uses (all SMs, many tiles per CTA), checked on sampled rows
    import torch
    params = random_params(4)
    P = 1024 * 1024
    X = torch.randn((P, 16), dtype=torch.float32, device="cuda", generator=torch.Generator(
        device="cuda").manual_seed(5))
    X[:, 15] = 0
    p = ot.Plan(1024, 1024, precision="mixed").set_weights(params)
    out = torch.zeros(P, dtype=torch.float32, device="cuda")
    p.ws_mlp_forward(X, out)
    idx = I.ws_batch_rows(17, 0, P, 4096)
    Xs = X.cpu().numpy()[idx].astype(np.float64)
    y_ref, _ = W.mlp_forward(params.astype(np.float64), Xs, bf16=True)
    y = out.cpu().numpy()[idx]
    scale = np.abs(y_ref).max()
    assert np.abs(y - y_ref).max() <= 2e-3 * scale
    assert np.abs(y - y_ref).mean() <= 2e-4 * scale
    p.close()


def test_gradient_matches_oracle(ot):
    import torch
    params = random_params(6)
    rng = np.random.default_rng(8)
    n = 20000
    X = rng.standard_normal((n, 16)).astype(np.float32)
    t = rng.standard_normal(n).astype(np.float32)
    B = 4096
    idx = I.ws_batch_rows(2, 0, n, B)
    tr = ot.Trainer(B, params)
    loss, g = tr.grad(tdev32(X), tdev32(t), torch.from_numpy(idx).cuda())
    loss_ref, g_ref = W.loss_and_grad(params.astype(np.float64), X[idx].astype(np.float64),
                                      t[idx].astype(np.float64))
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    o = 0
    for size in (W.H * W.K, W.H, W.H * W.H, W.H, W.H * W.H, W.H, W.H, 1):
        a, b = g[o:o + size], g_ref[o:o + size]
        assert np.abs(a - b).max() <= 1e-4 * np.abs(b).max() + 1e-12, o
        o += size
    # the parameters did not move
    assert np.array_equal(tr.params(), params)
    tr.close()


def test_adam_steps_match_oracle(ot):
    import torch
    params = random_params(7)
    rng = np.random.default_rng(9)
    n, B, lr = 8192, 1024, 1e-3
    X = rng.standard_normal((n, 16)).astype(np.float32)
    t = rng.standard_normal(n).astype(np.float32)
    tr = ot.Trainer(B, params)
    Xd, td = tdev32(X), tdev32(t)
    p_ref = params.astype(np.float64)
    m = np.zeros_like(p_ref)
    v = np.zeros_like(p_ref)
    well = np.ones(p_ref.size, dtype=bool)
    for step in range(3):
        idx = I.ws_batch_rows(11, step, n, B)
        tr.step(Xd, td, torch.from_numpy(idx).cuda(), lr)
        _, g = W.loss_and_grad(p_ref, X[idx].astype(np.float64), t[idx].astype(np.float64))
        well &= np.abs(g) > 1e-2 * np.abs(g).max()
        p_ref, m, v = W.adam_step(p_ref, m, v, g, step + 1, lr)
    p = tr.params().astype(np.float64)
    # every Adam step moves a parameter by at most ~lr; where the gradient is well above its
    # FP32 round-off the GPU steps equal the oracle's
    assert np.abs(p - p_ref).max() <= 2 * 3 * lr + 1e-6
    assert np.abs(p - p_ref)[well].max() <= 1e-2 * lr
    tr.close()


def test_predict_matches_oracle(ot):
    N = M = 64
    f, g = I.noise_blob_pair(N, M, s=3100)
    params = random_params(12, scale=0.01)
    u_ref, a_ref, _ = W.predict(params.astype(np.float64), f, g)
    p = ot.Plan(N, M, precision="mixed").set_weights(params)
    u = dev(np.zeros((N, M)))
    a = p.ws_predict(dev(f), dev(g), u)
    assert a == a_ref
    assert np.abs(u.cpu().numpy() - u_ref).max() <= 1e-3 * np.abs(u_ref).max()
    p.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_warm_started_solve(ot, prec):
    # the warm start changes the start, not the root: both solves reach the tolerance and
    # agree; graph and host-driven solves agree bit for bit
    N = M = 64
    f, g = I.noise_blob_pair(N, M, s=3200)
    params = random_params(13, scale=0.01)
    tol = 1e-10 if prec == "fp64" else 1e-8
    out = {}
    for mode, graph in ((0, 1), (2, 1), (2, 0)):
        p = ot.Plan(N, M, tau=2.0, tol=tol, precision=prec, eta=0.1, graph=graph)
        if mode == 2:
            p.set_weights(params).set(warm_start=2)
        phi = dev(np.zeros((N, M)))
        rc, st = p.solve(dev(f), dev(g), phi)
        assert rc == 0, st
        assert (st["ws_alpha"] == -1.0) == (mode == 0)
        out[(mode, graph)] = (phi.cpu().numpy(), st)
        p.close()
    a, b = out[(0, 1)][0], out[(2, 1)][0]
    assert np.abs(a - b).max() <= (1e-9 if prec == "fp64" else 1e-6)
    assert np.array_equal(out[(2, 1)][0], out[(2, 0)][0])
    assert out[(2, 1)][1]["newton_iters"] == out[(2, 0)][1]["newton_iters"]


def test_network_kernel_timing_class(ot):
    # ot_plan_time_kernel(OT_TIME_WS_NETWORK) relaunches the network kernel on the solve's
    # features: a positive time, and a later solve is unchanged (only workspace is written);
    # a plan without weights refuses the class
    import ctypes
    N = M = 64
    f, g = I.noise_blob_pair(N, M, s=3300)
    p = ot.Plan(N, M, tau=2.0, tol=1e-8, precision="mixed", eta=0.1)
    p.set_weights(random_params(13, scale=0.01)).set(warm_start=2)
    phi1 = dev(np.zeros((N, M)))
    assert p.solve(dev(f), dev(g), phi1)[0] == 0
    ms = p.time_kernel("ws_network", reps=5)
    assert 0.0 < ms < 50.0
    phi2 = dev(np.zeros((N, M)))
    assert p.solve(dev(f), dev(g), phi2)[0] == 0
    assert np.array_equal(phi1.cpu().numpy(), phi2.cpu().numpy())
    q = ot.Plan(N, M, tau=2.0, tol=1e-8, precision="mixed", eta=0.1)
    assert q.solve(dev(f), dev(g), dev(np.zeros((N, M))))[0] == 0
    out = ctypes.c_double()
    assert ot.ot_plan_time_kernel(q.h, ot.OT_TIME_WS_NETWORK, 5, ctypes.byref(out)) == \
        ot.OT_EINVAL
    assert ot.ot_plan_time_kernel(q.h, 11, 5, ctypes.byref(out)) == ot.OT_EINVAL
    p.close()
    q.close()


def test_weights_file_round_trip(ot, tmp_path):
    params = random_params(14)
    path = str(tmp_path / "w.otws")
    assert ot.ot_ws_save_weights(path, params.ctypes.data, params.size) == 0
    p1 = ot.Plan(32, 32, precision="mixed").load_weights(path)
    p2 = ot.Plan(32, 32, precision="mixed").set_weights(params)
    import torch
    X = tdev32(np.random.default_rng(1).standard_normal((500, 16)))
    o1 = torch.zeros(500, dtype=torch.float32, device="cuda")
    o2 = torch.zeros(500, dtype=torch.float32, device="cuda")
    p1.ws_mlp_forward(X, o1)
    p2.ws_mlp_forward(X, o2)
    assert torch.equal(o1, o2)
    bad = str(tmp_path / "bad.otws")
    open(bad, "wb").write(b"OTWS0001" + b"\0" * 8)
    assert ot.ot_warmstart_load(p1.h, bad) == ot.OT_EINVAL
    assert ot.ot_warmstart_load(p1.h, str(tmp_path / "missing")) == ot.OT_EINVAL
    # warm_start = 2 needs weights
    p3 = ot.Plan(32, 32)
    assert ot.ot_plan_set_option(p3.h, ot.OT_OPT_WARM_START, 2) == ot.OT_EINVAL
    for p in (p1, p2, p3):
        p.close()


def test_trained_network_saves_newton_steps(ot):
    # train on solved pairs, then compare warm and zero starts on held-out pairs of the same
    # generator: every warm solve reaches the tolerance at the same root, in fewer steps on
    # average
    import torch
    from paper_1009_6039_gb300 import warmstart as WS
    N = M = 128
    train = [I.noise_blob_pair(N, M, s=10000 + k) for k in range(24)]
    held = [I.noise_blob_pair(N, M, s=90000 + k) for k in range(4)]
    params = WS.train(train, N, M, steps=600, batch=8192, seed=1, tau=2.0, tol=1e-8, eta=0.1)
    cold, warm = [], []
    for f, g in held:
        res = {}
        for mode in (0, 2):
            p = ot.Plan(N, M, tau=2.0, tol=1e-8, eta=0.1, precision="mixed")
            if mode == 2:
                p.set_weights(params).set(warm_start=2)
            phi = dev(np.zeros((N, M)))
            rc, st = p.solve(dev(f), dev(g), phi)
            assert rc == 0
            res[mode] = (phi.cpu().numpy(), st)
            p.close()
        assert np.abs(res[0][0] - res[2][0]).max() <= 1e-6
        cold.append(res[0][1]["newton_iters"])
        warm.append(res[2][1]["newton_iters"])
    assert np.mean(warm) < np.mean(cold), (cold, warm)


def test_network_wait_timeout_is_reported_and_recoverable(ot):
    # the bounded mbarrier wait of the tensor-core kernel runs out (one MMA group is not
    # issued); the call reports it, the error flag clears, and the next call is correct
    import torch
    params = random_params(15)
    rows = 5000
    X = tdev32(np.random.default_rng(3).standard_normal((rows, 16)))
    p = ot.Plan(32, 32, precision="mixed").set_weights(params)
    out = torch.zeros(rows, dtype=torch.float32, device="cuda")
    p.set(ws_test_stall=1)
    assert ot.ot_ws_mlp_forward(p.h, ctypes_ptr(X), rows, ctypes_ptr(out)) == ot.OT_ETIMEOUT
    assert "mbarrier wait" in ot.ot_last_error()
    p.ws_mlp_forward(X, out)
    y_ref, _ = W.mlp_forward(params.astype(np.float64), X.cpu().numpy().astype(np.float64),
                             bf16=True)
    assert np.abs(out.cpu().numpy() - y_ref).max() <= 2e-3 * np.abs(y_ref).max()
    p.close()


def ctypes_ptr(t):
    import ctypes
    return ctypes.c_void_p(t.data_ptr())


def test_network_timeout_inside_a_solve_falls_back_to_zero_start(ot):
    # the same failure inside a solve: the admissibility step takes the zero start, the
    # stats report ws_alpha = -2 and ot_last_error names the warm start; the solve reaches
    # the root of the zero-start solve
    N = M = 64
    f, g = I.noise_blob_pair(N, M, s=3600)
    kw = dict(tau=1.0, tol=1e-8, eta=1e-2, precision="mixed", symbols=1, graph=0)
    p0 = ot.Plan(N, M, **kw)
    phi0 = dev(np.zeros((N, M)))
    rc0, st0 = p0.solve(dev(f), dev(g), phi0)
    p0.close()
    p = ot.Plan(N, M, **kw).set_weights(random_params(16))
    p.set(warm_start=2, ws_test_stall=1)
    phi = dev(np.zeros((N, M)))
    rc, st = p.solve(dev(f), dev(g), phi)
    assert rc == 0 and rc0 == 0
    assert st["ws_alpha"] == -2.0
    assert "warm start" in ot.ot_last_error()
    assert st["newton_iters"] == st0["newton_iters"]
    assert np.abs(phi.cpu().numpy() - phi0.cpu().numpy()).max() <= 1e-9
    # the hook reset itself: the next solve uses the network again
    rc2, st2 = p.solve(dev(f), dev(g), phi)
    assert rc2 == 0 and st2["ws_alpha"] >= 0.0
    p.close()
