"""GPU tests of the plan set (ot_solve_batched): many problems of uneven sizes in one graph
launch, each size class running every kernel for all its pairs with per-pair loop control.

Bounds: the batched solve is the mixed-precision solve (FP32 transforms and Krylov vectors,
FP64-accurate residual and update), so a converged pair matches the FP64 oracle's root within
the mixed-mode bound 1e-6 (on the oracle's stored samples), and a single-problem mixed solve
of the same pair within the distance of two roots with max|F| < tol (about ||J^-1|| 2 tol).
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import ot_inputs as I
from gpu_util import dev

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
# the batched workload's settings (stencil symbols, tau = 1, eta = 0.1, tol 1e-8)
SETTINGS = dict(tau=1.0, tol=1e-8)
OPTS = dict(eta=0.1, symbols=1, max_newton=1000, tau_retry=2)


@pytest.fixture(scope="module")
def ot():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1009_6039_gb300 as m
    return m


def batch_pairs(indices):
    work = I.batch_workload(512)
    out = []
    for k in indices:
        n, s = work[k]
        f, g = I.blob_pair(n, n, s=s)
        out.append((k, n, f, g))
    return out


def solve_set(ot, pairs, **kw):
    import torch
    opts = dict(OPTS)
    opts.update(kw)
    ps = ot.PlanSet([(f.shape[0], f.shape[1]) for f, _ in pairs], **SETTINGS, **opts)
    fs = [dev(f) for f, _ in pairs]
    gs = [dev(g) for _, g in pairs]
    phis = [torch.zeros_like(t) for t in fs]
    rc, st = ps.solve(fs, gs, phis, raise_on=())
    ps.close()
    return rc, st, [p.cpu().numpy() for p in phis]


def test_batched_pairs_match_the_oracle(ot):
    # pairs of the batched workload (ot_inputs.batch_workload), the first of each size with a
    # stored oracle solve, plus others of the same sizes so that every size class has several
    # pairs, and the two 512^2 pairs that the oracle solves at tau = 1 (batch200, batch297)
    with_gold = [0, 2, 5, 7, 9, 200, 297]
    others = [1, 3, 6, 8, 12, 13, 15, 19]
    pairs = batch_pairs(with_gold + others)
    rc, st, phis = solve_set(ot, [(f, g) for _, _, f, g in pairs])
    for (k, n, f, g), s, phi in zip(pairs, st, phis):
        assert s["status"] == 0 and s["res_inf"] < SETTINGS["tol"], (k, s)
        assert abs(phi.mean()) < 1e-14
        if k in with_gold:
            with open(os.path.join(GOLDEN, "batch%d.json" % k)) as fh:
                gold = json.load(fh)
            ii, jj = np.array(gold["sample_i"]), np.array(gold["sample_j"])
            err = np.abs(phi[ii, jj] - np.array(gold["phi_samples"])).max()
            assert err <= 1e-6, (k, err)
    assert rc == 0


def test_batched_equals_single_problem_solves(ot):
    # uneven sizes, two pairs of one size: each pair reaches the root of its own
    # single-problem mixed solve
    sizes = [(32, 32), (48, 96), (32, 32), (64, 64), (24, 48)]
    pairs = [I.blob_pair(N, M, s=4100 + k) for k, (N, M) in enumerate(sizes)]
    rc, st, phis = solve_set(ot, pairs, tau_retry=0)
    assert rc == 0
    for (f, g), s, phi in zip(pairs, st, phis):
        N, M = f.shape
        p = ot.Plan(N, M, precision="mixed", **SETTINGS, **{k: v for k, v in OPTS.items()
                                                             if k != "tau_retry"})
        ref = dev(np.zeros((N, M)))
        rc1, s1 = p.solve(dev(f), dev(g), ref)
        p.close()
        assert rc1 == 0 and s["status"] == 0
        assert np.abs(phi - ref.cpu().numpy()).max() <= 1e-9
        assert abs(s["newton_iters"] - s1["newton_iters"]) <= 1
        # the statistics of the batched solve
        assert s["res_inf"] < SETTINGS["tol"] and s["gmres_iters"] > 0
        assert abs(s["mass_defect_f"]) < 1e-13 and s["kernel_launches"] > 0


def test_batched_retry_solves_only_the_diverged_pairs(ot):
    # without the safeguard one 32^2 blob pair loses convexity at tau = 1 (the oracle's plain
    # Eq. linma does too); with OT_OPT_TAU_RETRY the set solves it again with 2 tau, 4 tau
    # while the other pairs sit the rounds out, keeping their first results
    f0, g0 = I.blob_pair(32, 32)
    _, st_ref, _, _ = O.solve(f0, g0, tau=1.0, tol=1e-8, eta=1e-2, max_newton=400,
                              safeguard=False)
    # the other pairs: manufactured ones that converge at tau = 1 without the safeguard
    pairs = [(f0, g0)] + [I.manufactured(32, 32, amp=a * I.MANUFACTURED_A)[:2]
                          for a in (0.5, 1.0, 1.5)]
    base = dict(safeguard=0, symbols=0, eta=1e-2, max_newton=400)
    rc0, st0, ph0 = solve_set(ot, pairs, tau_retry=0, **base)
    rc, st, ph = solve_set(ot, pairs, tau_retry=3, **base)
    if st_ref["status"] == O.ORC_EDIVERGED:
        assert st0[0]["status"] == ot.OT_EDIVERGED
    assert st[0]["status"] == 0 and st[0]["res_inf"] < 1e-8
    for k in range(1, 4):
        assert st0[k]["status"] == st[k]["status"]
        assert np.array_equal(ph0[k], ph[k])
    u_ref, s_ref, _, _ = O.solve(f0, g0, tau=4.0, tol=1e-10, eta=1e-2, max_newton=400)
    assert s_ref["status"] == 0
    assert np.abs(ph[0] - u_ref).max() <= 1e-6


def test_batched_invalid_pair_and_api_checks(ot):
    import torch
    f, g = I.blob_pair(32, 32, s=7)
    bad = f.copy()
    bad[3, 4] = np.nan
    rc, st, _ = solve_set(ot, [(f, g), (bad, g)], tau_retry=0)
    assert st[0]["status"] == 0 and st[1]["status"] == ot.OT_EINVAL
    assert rc == ot.OT_EINVAL
    # sizes must repeat the set's
    ps = ot.PlanSet([(32, 32), (32, 32)], **SETTINGS)
    z = dev(np.zeros((32, 32)))
    p = ctypes_ptr(z)
    assert ot.ot_solve_batched(ps.h, 2, [32, 64], [32, 64], [p, p], [p, p], [p, p]) == \
        ot.OT_EINVAL
    assert ot.ot_solve_batched(ps.h, 1, [32], [32], [p], [p], [p]) == ot.OT_EINVAL
    # the set is the mixed-precision solve; options outside its set are refused
    assert ot.ot_batch_set_option(ps.h, ot.OT_OPT_PRECISION, 0) == ot.OT_EINVAL
    assert ot.ot_batch_set_option(ps.h, ot.OT_OPT_WARM_START, 2) == ot.OT_EINVAL
    assert ot.ot_batch_set_option(ps.h, ot.OT_OPT_TAU, 0.5) == ot.OT_EINVAL
    ps.close()
    rc, h = ot.ot_plan_set_create(2, [32, 30], [32, 30], 1.0, 1e-8)
    assert rc == ot.OT_EUNSUPPORTED
    del torch


def ctypes_ptr(t):
    return t.data_ptr()
