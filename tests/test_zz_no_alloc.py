"""The allocation-free residual entry point (for callers that cannot allocate device memory:
code whose device memory is all owned by its own pool, or latency-critical loops that cannot
afford cudaMalloc's implicit synchronisation) agrees with the plan-based ot_eval_residual.

Kept in a file of its own that pytest collects last, so a run stopping at the first failure
has already run every other test.  It builds what it needs itself, so it also passes alone in
a fresh process."""
import ctypes

import numpy as np
import pytest

import oracle as O
import ot_inputs as I

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


def _field(N, M, seed):
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid(np.arange(N) / N, np.arange(M) / M, indexing="ij")
    u = np.zeros((N, M))
    for _ in range(5):
        k1, k2 = rng.integers(-3, 4, 2)
        u += 1e-3 * rng.standard_normal() * np.cos(2 * np.pi * (k1 * x + k2 * y) + rng.random())
    return u


# (2048, 2048) fills the fixed scratch exactly (4096 tiles of 32 x 32, 10 partials each);
# (2048, 48) and (48, 2048) have ragged edge tiles along one axis
@pytest.mark.parametrize("N,M,on_stream", [(64, 96, False), (256, 256, False),
                                           (256, 256, True), (2048, 48, False),
                                           (48, 2048, False), (2048, 2048, True)])
def test_noalloc_matches_plan_entry_point_twice(ot, N, M, on_stream):
    import torch

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    def ptr(t):
        return ctypes.c_void_p(t.data_ptr())

    plan = ot.Plan(N, M, precision="fp64")
    # on_stream: both entry points run on a non-default torch stream, passed by handle
    stream = torch.cuda.Stream() if on_stream else None
    handle = stream.cuda_stream if on_stream else 0
    if on_stream:
        assert ot.ot_plan_set_stream(plan.h, handle) == 0
    for call, seed in enumerate((1, 2)):  # two calls in a row on the shared scratch
        f = I.blob_density(N, M, 40 + seed)
        g = I.blob_density(N, M, 50 + seed)
        u = _field(N, M, seed)
        fd, ud = dev(f), dev(u)
        cd = dev(O.bspline_coeffs(g))
        F_ref, coef_ref = dev(np.zeros((N, M))), dev(np.zeros((5, N, M)))
        F_new, coef_new = dev(np.zeros((N, M))), dev(np.zeros((5, N, M)))
        s_ref, s_new = np.zeros(10), np.zeros(10)
        assert ot.ot_eval_residual(plan.h, ptr(fd), ptr(cd), ptr(ud), ptr(F_ref),
                                   ptr(coef_ref), s_ref.ctypes.data_as(ctypes.c_void_p)) == 0
        torch.cuda.synchronize()
        assert ot.ot_eval_residual_noalloc(N, M, ptr(fd), ptr(cd), ptr(ud), ptr(F_new),
                                           ptr(coef_new),
                                           s_new.ctypes.data_as(ctypes.c_void_p),
                                           handle) == 0
        # the tolerance of the residual parity test (rounding bound of the stencils)
        eps = np.finfo(float).eps
        tol = 32 * eps * np.abs(u).max() * max(N, M) ** 2 * max(1, np.abs(g).max()) + 1e-13
        assert np.abs(F_new.cpu().numpy() - F_ref.cpu().numpy()).max() <= tol, call
        cscale = max(1.0, float(coef_ref.abs().max()))
        assert np.abs(coef_new.cpu().numpy() - coef_ref.cpu().numpy()).max() <= tol * cscale
        assert np.abs(s_new - s_ref).max() <= tol * cscale, (s_new, s_ref)
    plan.close()


def test_noalloc_rejects_oversized_grid(ot):
    z = ctypes.c_void_p(8)  # never dereferenced: the size check comes first
    assert ot.ot_eval_residual_noalloc(4096, 4096, z, z, z, z, z, None) == ot.OT_EUNSUPPORTED
    assert ot.ot_eval_residual_noalloc(4, 64, z, z, z, z, z, None) == ot.OT_EINVAL
