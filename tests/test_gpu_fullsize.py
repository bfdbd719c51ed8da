"""GPU parity at the benchmarked sizes against stored oracle results.

The expected values come from tests/golden/make_golden.py, which runs only the CPU oracle
(its FP64 Newton solve, Sec. 3.1, with the Fourier linear solver of Sec. 4.2) and stores
the Newton/GMRES counts and the potential at 512 seeded grid points.  The solves here run
the library's graph-launched path with the settings each file lists.

Bounds:
  - FP64 path, same settings as the oracle: the same Newton steps (the convergence test
    max|F| < tol sees the same iterates up to round-off) and ||phi - phi_oracle||_inf <=
    1e-10 on the samples.
  - mixed path (FP32 FFTs and Krylov vectors, FP64-accurate residual and update): the
    residual reaches the same tolerance, so the root agrees with the oracle's to about
    ||J^-1|| 2 tol plus the refinement's round-off: <= 1e-6 on the samples.
"""
import json
import os

import numpy as np
import pytest

import ot_inputs as I
from gpu_util import dev

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def ot():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1009_6039_gb300 as m
    return m


def golden(name):
    path = os.path.join(GOLDEN, name + ".json")
    if not os.path.exists(path):
        pytest.fail("missing stored oracle result %s (python tests/golden/make_golden.py %s)"
                    % (path, name))
    with open(path) as fh:
        return json.load(fh)


def inputs(case):
    if "batch_index" in case:
        n, s = I.batch_workload(512)[case["batch_index"]]
        return I.blob_pair(n, n, s=s)
    gen = {"blob_pair": I.blob_pair, "noise_blob_pair": I.noise_blob_pair}[case["kind"]]
    return gen(case["N"], case["M"], s=case["seed"])


def sample_err(phi, gold):
    ii, jj = np.array(gold["sample_i"]), np.array(gold["sample_j"])
    return float(np.abs(phi[ii, jj] - np.array(gold["phi_samples"])).max())


def solve(ot, gold, precision, **kw):
    case = gold["case"]
    f, g = inputs(case)
    N, M = f.shape
    opts = dict(tau=case["tau"], tol=case["tol"], eta=case["eta"],
                symbols=case.get("symbols", 0), max_newton=case.get("max_newton", 300))
    opts.update(kw)
    p = ot.Plan(N, M, precision=precision, **opts)
    phi = dev(np.zeros((N, M)))
    rc, st = p.solve(dev(f), dev(g), phi)
    return p, rc, st, phi.cpu().numpy(), (f, g)


def test_noise1024_fp64_same_steps_as_oracle(ot):
    # the timed workload's pair and settings (stencil symbols, tau = 1, eta = 0.01, tol 1e-8)
    # on the plain FP64 path: the oracle's 13 Newton steps, 91 GMRES iterations and 7 step
    # halvings, and its root within 1e-10
    gold = golden("noise1024")
    p, rc, st, phi, _ = solve(ot, gold, "fp64")
    p.close()
    ref = gold["stats"]
    assert rc == 0 and st["res_inf"] < gold["case"]["tol"]
    assert st["newton_iters"] == ref["newton_iters"]
    assert st["gmres_iters"] == ref["gmres_iters"]
    assert st["step_halvings"] == ref["step_halvings"]
    assert sample_err(phi, gold) <= 1e-10


def test_noise1024_mixed_learned_warm_start(ot):
    # the benchmarked configuration: mixed precision and the learned warm start (a network
    # trained here on two other pairs of the generator); Newton still runs to max|F| < 1e-8,
    # so the result is the oracle's root within the mixed-mode bound
    from paper_1009_6039_gb300 import warmstart as WS
    gold = golden("noise1024")
    case = gold["case"]
    N = M = 1024
    pairs = [I.noise_blob_pair(N, M, s=10000 + k) for k in range(2)]
    X, t = WS.training_data(pairs, N, M, tau=1.0, tol=1e-8, eta=0.1)
    params = WS.fit(X, t, steps=300, batch=32768, seed=1)
    del X, t
    f, g = inputs(case)
    p = ot.Plan(N, M, precision="mixed", tau=case["tau"], tol=case["tol"], eta=case["eta"],
                symbols=1)
    p.set_weights(params).set(warm_start=2)
    phi = dev(np.zeros((N, M)))
    rc, st = p.solve(dev(f), dev(g), phi)
    p.close()
    assert rc == 0 and st["res_inf"] < case["tol"]
    assert st["ws_alpha"] >= 0.0
    assert sample_err(phi.cpu().numpy(), gold) <= 1e-6


def test_noise2048_mixed(ot):
    # the largest benchmarked grid, mixed precision from the zero start
    gold = golden("noise2048")
    p, rc, st, phi, _ = solve(ot, gold, "mixed")
    p.close()
    assert rc == 0 and st["res_inf"] < gold["case"]["tol"]
    assert sample_err(phi, gold) <= 1e-6


def test_blob256_fp64(ot):
    # the 256^2 blob-mixture pair on the plain FP64 path (tau = 4: at tau = 2 the oracle's
    # iteration stalls on this pair, see the oracle run stored beside it).  A run of 180
    # safeguarded steps with eta = 0.1 may take a slightly different path (one borderline
    # GMRES stop moves theta at the eta level), so the Newton count is compared within 3;
    # the root is unique and compared at 1e-10.
    gold = golden("blob256")
    p, rc, st, phi, _ = solve(ot, gold, "fp64", max_newton=400)
    p.close()
    ref = gold["stats"]
    assert rc == 0 and st["res_inf"] < gold["case"]["tol"]
    assert abs(st["newton_iters"] - ref["newton_iters"]) <= 3
    assert sample_err(phi, gold) <= 1e-10
