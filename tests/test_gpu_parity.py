"""GPU parity: every stage of the CUDA path, called through the C ABI, against the CPU
oracle on the same seeded inputs.

Tolerances: FP64 stages are compared to the oracle's FP64 result within a few hundred ulps
of the result's scale (different summation order, FMA contraction and FFT factorisation);
FP32 (mixed-mode) stages within 2e-5 of the scale (FP32 round-off, 2^-24 ~ 6e-8, grown
by the log2 P stages of the FFT and the symbol magnitudes).  Solves: ||phi_gpu -
phi_oracle||_inf <= 1e-10 for the FP64 path after the same Newton steps, <= 1e-6 for the
mixed path at the same residual tolerance.
"""
import numpy as np
import pytest

import oracle as O
import ot_inputs as I
from gpu_util import dev, hptr, pack_spectrum, ptr, unpack_spectrum

pytestmark = pytest.mark.gpu

SIZES = [(8, 16), (12, 24), (16, 16), (24, 48), (128, 48), (64, 96), (12, 512), (192, 384),
         (256, 256)]
RNG = np.random.default_rng(7)


@pytest.fixture(scope="module")
def ot():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1009_6039_gb300 as m
    return m


def plan(ot, N, M, precision="fp64", **kw):
    return ot.Plan(N, M, precision=precision, **kw)


def smooth_field(N, M, amp=1.0, kmax=4):
    y, x = np.meshgrid(np.arange(N) / N, np.arange(M) / M, indexing="ij")
    u = np.zeros((N, M))
    for _ in range(6):
        k1, k2 = RNG.integers(-kmax, kmax + 1, 2)
        ph = RNG.random() * 2 * np.pi
        u += RNG.standard_normal() * np.cos(2 * np.pi * (k1 * x + k2 * y) + ph)
    return amp * u


# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("N,M", SIZES)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fft_forward_inverse(ot, N, M, prec):
    x = RNG.standard_normal((N, M))
    p = plan(ot, N, M, prec)
    xd = dev(x)
    sd = dev(np.zeros((N, M)))
    assert ot.ot_fft_forward(p.h, ptr(xd), ptr(sd)) == 0
    half = unpack_spectrum(sd.cpu().numpy(), N, M)
    ref = O.fft2(x)[:, :M // 2 + 1]
    tol = (2e-13 if prec == "fp64" else 2e-5) * np.abs(ref).max()
    assert np.abs(half - ref).max() <= tol
    # inverse (unnormalised) of the oracle's spectrum returns N M x
    sd2 = dev(pack_spectrum(ref, N, M))
    xo = dev(np.zeros((N, M)))
    assert ot.ot_fft_inverse(p.h, ptr(sd2), ptr(xo)) == 0
    back = xo.cpu().numpy() / (N * M)
    assert np.abs(back - x).max() <= (2e-13 if prec == "fp64" else 2e-5) * np.abs(x).max()
    p.close()


@pytest.mark.parametrize("N,M", [(8, 16), (12, 24), (16, 16), (24, 48), (128, 48), (192, 384),
                                 (256, 256), (1024, 1024)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_prefilter(ot, N, M, prec):
    # FP64 recursions, or (mixed) the same recursions in double-float: both to FP64-level
    # accuracy against the oracle's exact periodic inverse (|c| ~ 1.5, dd unit round-off 2^-48)
    g = 1 + 0.5 * RNG.random((N, M))
    p = plan(ot, N, M, prec)
    gd, cd = dev(g), dev(np.zeros((N, M)))
    assert ot.ot_prefilter(p.h, ptr(gd), ptr(cd)) == 0
    assert np.abs(cd.cpu().numpy() - O.bspline_coeffs(g)).max() <= 1e-13
    p.close()


@pytest.mark.parametrize("N,M", [(16, 16), (24, 48), (128, 48), (64, 96), (192, 384),
                                 (256, 256)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_residual_and_coefficients(ot, N, M, prec):
    f = I.blob_density(N, M, 11)
    g = I.blob_density(N, M, 12)
    u = smooth_field(N, M, amp=2e-3)
    c = O.bspline_coeffs(g)
    F_ref, coef_ref, s_ref = O.residual(f, c, u)
    p = plan(ot, N, M, prec)
    fd, cd, ud = dev(f), dev(c), dev(u)
    Fd, coefd = dev(np.zeros((N, M))), dev(np.zeros((5, N, M)))
    scal = np.zeros(10)
    assert ot.ot_eval_residual(p.h, ptr(fd), ptr(cd), ptr(ud), ptr(Fd), ptr(coefd),
                               hptr(scal)) == 0
    # F and the scalars are FP64 values in both modes; the mixed mode computes them in
    # double-float arithmetic (FP32 pairs, unit round-off 2^-48) instead of FP64 (2^-52).
    # Rounding bound: the second-difference stencils cancel, so their rounding error is
    # ~ (sum of |taps| = 64) eps max|u| L^2 / 12 per derivative, times |G| in f_n = G det(...)
    eps = np.finfo(float).eps if prec == "fp64" else 2.0 ** -48
    tol = 32 * eps * np.abs(u).max() * max(N, M) ** 2 * max(1, np.abs(g).max())
    # plus the interpolated value G (|G| <~ max|g|): ~20 multiply-adds of the 16-tap gather
    # and the products det, G det, each within 2 eps relative -> 64 eps max|g| (below 1e-13
    # in FP64, which the fixed 1e-13 covers)
    tol += 1e-13 if prec == "fp64" else 64 * eps * max(1, np.abs(g).max())
    assert np.abs(Fd.cpu().numpy() - F_ref).max() <= tol
    assert abs(scal[0] - s_ref["mean_fn"]) <= tol
    assert abs(scal[1] - s_ref["res_inf"]) <= tol
    assert abs(scal[2] - s_ref["res_l2"]) <= tol
    assert abs(scal[3] - s_ref["min_det"]) <= tol
    assert scal[4] == 0
    abar_ref = [O.simpson_mean(coef_ref[q]) for q in range(5)]
    # mixed mode: the gradient of the interpolant (b1, b2; Jacobian only) is FP32
    atol = tol if prec == "fp64" else 1e-6
    assert np.abs(scal[5:] - abar_ref).max() <= atol * max(1, np.abs(coef_ref).max())
    ctol = (tol if prec == "fp64" else 1e-6 * np.abs(coef_ref).max()) * max(1, np.abs(coef_ref).max())
    assert np.abs(coefd.cpu().numpy() - coef_ref).max() <= ctol
    p.close()


@pytest.mark.parametrize("N,M", [(16, 16), (24, 48), (128, 48), (64, 96), (192, 384),
                                 (256, 256)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("symbols", [0, 1])
def test_operator_and_lbar_inverse(ot, N, M, prec, symbols):
    f = I.blob_density(N, M, 21)
    g = I.blob_density(N, M, 22)
    u = smooth_field(N, M, amp=2e-3)
    _, coef, _ = O.residual(f, O.bspline_coeffs(g), u)
    abar = np.array([O.simpson_mean(coef[q]) for q in range(5)])
    sigma = RNG.standard_normal((N, M))
    with O.fd_symbols(symbols):
        w_ref = O.apply_op(coef, abar, sigma)
        th_ref = O.apply_lbar_inv(abar, sigma)
    p = plan(ot, N, M, prec, symbols=symbols)
    cd, sd, wd, td = dev(coef), dev(sigma), dev(np.zeros((N, M))), dev(np.zeros((N, M)))
    assert ot.ot_apply_operator(p.h, ptr(cd), hptr(abar), ptr(sd), ptr(wd)) == 0
    assert ot.ot_apply_lbar_inverse(p.h, hptr(abar), ptr(sd), ptr(td)) == 0
    r = 1e-12 if prec == "fp64" else 5e-6
    assert np.abs(wd.cpu().numpy() - w_ref).max() <= r * np.abs(w_ref).max()
    assert np.abs(td.cpu().numpy() - th_ref).max() <= r * np.abs(th_ref).max()
    if prec == "mixed":
        assert np.linalg.norm(wd.cpu().numpy() - w_ref) <= 2e-6 * np.linalg.norm(w_ref)
    p.close()


@pytest.mark.parametrize("N,M", [(16, 16), (24, 48), (128, 48), (192, 384), (256, 256),
                                 (1024, 1024)])
def test_transport_outputs(ot, N, M):
    # Sec. 5.2 outputs: d = mean |grad u|^2 f and div = u_xx + u_yy, in double-float on the
    # GPU.  d: the stencils' rounding (2^-48 relative to max|u| times sum|taps| M / 12) is
    # far below the value (|grad u| ~ 2 pi k |u|), plus a log2(P)-deep double-float sum:
    # 1e-11 relative.  div: the second-difference stencils cancel, 64 eps max|u| max(N,M)^2.
    f = I.blob_density(N, M, 41)
    u = smooth_field(N, M, amp=2e-3)
    d_ref, div_ref = O.transport_outputs(f, u)
    p = plan(ot, N, M, "mixed")
    div = dev(np.zeros((N, M)))
    d = p.transport_outputs(dev(f), dev(u), div)
    assert abs(d - d_ref) <= 1e-11 * d_ref
    tol = 64 * 2.0 ** -48 * np.abs(u).max() * max(N, M) ** 2
    assert np.abs(div.cpu().numpy() - div_ref).max() <= tol
    # without the map: the distance alone
    assert abs(p.transport_outputs(dev(f), dev(u)) - d) <= 1e-15 * d
    p.close()


@pytest.mark.parametrize("N,M", [(2048, 32), (32, 2048), (1536, 48), (48, 1536)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_longest_transforms(ot, N, M, prec):
    # the longest supported transform lengths (columns N <= 2048, rows M <= 2048, and a
    # radix-3 length): the launch configurations at their largest blocks (the default variants
    # at these shapes include the concurrent column pass and the two-warp row transforms),
    # through the operator and Lbar^-1
    f = I.blob_density(N, M, 61)
    g = I.blob_density(N, M, 62)
    u = smooth_field(N, M, amp=2e-3)
    _, coef, _ = O.residual(f, O.bspline_coeffs(g), u)
    abar = np.array([O.simpson_mean(coef[q]) for q in range(5)])
    sigma = RNG.standard_normal((N, M))
    w_ref = O.apply_op(coef, abar, sigma)
    th_ref = O.apply_lbar_inv(abar, sigma)
    p = plan(ot, N, M, prec)
    cd, sd, wd, td = dev(coef), dev(sigma), dev(np.zeros((N, M))), dev(np.zeros((N, M)))
    assert ot.ot_apply_operator(p.h, ptr(cd), hptr(abar), ptr(sd), ptr(wd)) == 0
    assert ot.ot_apply_lbar_inverse(p.h, hptr(abar), ptr(sd), ptr(td)) == 0
    r = 1e-12 if prec == "fp64" else 5e-6
    assert np.abs(wd.cpu().numpy() - w_ref).max() <= r * np.abs(w_ref).max()
    assert np.abs(td.cpu().numpy() - th_ref).max() <= r * np.abs(th_ref).max()
    p.close()


@pytest.mark.parametrize("N,M", [(24, 48), (128, 48), (192, 384), (256, 256), (512, 512),
                                 (1024, 1024)])
@pytest.mark.parametrize("variant", [0, 0 + 4 * 1 + 16 * 1, 2 + 4 * 2 + 16 * 2,
                                     3 + 4 * 3 + 16 * 3, 2 + 4 * 0 + 16 * 1, 64, 128,
                                     3 + 4 * 3 + 16 * 3 + 256, 63 + 256 + 512,
                                     63 + 256 + 512 + 1024])
def test_fp32_kernel_variants(ot, N, M, variant):
    # every FP32 transform kernel variant the autotuner can pick computes the same operator
    # (at 1024^2 the concurrent column pass, launched first, needs more shared memory than
    # the warp column pass, which has the same signature: each kernel's own limit is raised)
    f = I.blob_density(N, M, 23)
    g = I.blob_density(N, M, 24)
    u = smooth_field(N, M, amp=2e-3)
    _, coef, _ = O.residual(f, O.bspline_coeffs(g), u)
    abar = np.array([O.simpson_mean(coef[q]) for q in range(5)])
    sigma = RNG.standard_normal((N, M))
    w_ref = O.apply_op(coef, abar, sigma)
    p = plan(ot, N, M, "mixed", fft_variant=variant)
    cd, sd, wd = dev(coef), dev(sigma), dev(np.zeros((N, M)))
    assert ot.ot_apply_operator(p.h, ptr(cd), hptr(abar), ptr(sd), ptr(wd)) == 0
    assert np.abs(wd.cpu().numpy() - w_ref).max() <= 5e-6 * np.abs(w_ref).max()
    assert np.linalg.norm(wd.cpu().numpy() - w_ref) <= 2e-6 * np.linalg.norm(w_ref)
    p.close()


@pytest.mark.parametrize("N,M", [(64, 128), (128, 2048), (1024, 128), (256, 512),
                                 (512, 256), (1024, 1024)])
def test_register_resident_matvec(ot, N, M):
    # the register-resident passes on the transposed spectrum (OT_OPT_FFT_VARIANT bit 128)
    # at every length they cover (N and M/2 powers of two in 64..1024), rectangular grids
    # included: the same operator as the oracle within the FP32 bounds of the other variants,
    # and the kernels in use read back through the option
    f = I.blob_density(N, M, 25)
    g = I.blob_density(N, M, 26)
    u = smooth_field(N, M, amp=2e-3)
    _, coef, _ = O.residual(f, O.bspline_coeffs(g), u)
    abar = np.array([O.simpson_mean(coef[q]) for q in range(5)])
    sigma = RNG.standard_normal((N, M))
    for symbols in (0, 1):
        with O.fd_symbols(symbols):
            w_ref = O.apply_op(coef, abar, sigma)
        p = plan(ot, N, M, "mixed", fft_variant=128, symbols=symbols)
        assert int(p.get("fft_variant")) & 128
        cd, sd, wd = dev(coef), dev(sigma), dev(np.zeros((N, M)))
        assert ot.ot_apply_operator(p.h, ptr(cd), hptr(abar), ptr(sd), ptr(wd)) == 0
        assert np.abs(wd.cpu().numpy() - w_ref).max() <= 5e-6 * np.abs(w_ref).max()
        assert np.linalg.norm(wd.cpu().numpy() - w_ref) <= 2e-6 * np.linalg.norm(w_ref)
        p.close()


@pytest.mark.parametrize("N,M", [(256, 24), (256, 512), (512, 256), (1024, 64), (2048, 128),
                                 (8, 512), (12, 1024), (48, 2048)])
def test_column_pair_pass(ot, N, M):
    # the column matvec pass on column pairs and the combine pass on row pairs, with packed
    # FP32 arithmetic (OT_OPT_FFT_VARIANT bits 256 and 512), at every length they cover
    # (columns of 256 .. 2048, rows of 512 .. 2048 points; the pair with the packed DC /
    # Nyquist column included; sizes that only one of them covers take another variant for
    # the other pass), both symbol sets: the oracle's operator within the FP32 bounds of the
    # other variants, and the choice read back through the option
    f = I.blob_density(N, M, 27)
    g = I.blob_density(N, M, 28)
    u = smooth_field(N, M, amp=2e-3)
    _, coef, _ = O.residual(f, O.bspline_coeffs(g), u)
    abar = np.array([O.simpson_mean(coef[q]) for q in range(5)])
    sigma = RNG.standard_normal((N, M))
    for symbols in (0, 1):
        with O.fd_symbols(symbols):
            w_ref = O.apply_op(coef, abar, sigma)
        p = plan(ot, N, M, "mixed", fft_variant=63 + 256 + 512, symbols=symbols)
        assert int(p.get("fft_variant")) & 768 == 768
        cd, sd, wd = dev(coef), dev(sigma), dev(np.zeros((N, M)))
        assert ot.ot_apply_operator(p.h, ptr(cd), hptr(abar), ptr(sd), ptr(wd)) == 0
        assert np.abs(wd.cpu().numpy() - w_ref).max() <= 5e-6 * np.abs(w_ref).max()
        assert np.linalg.norm(wd.cpu().numpy() - w_ref) <= 2e-6 * np.linalg.norm(w_ref)
        p.close()


def test_autotuned_solve_matches_fixed_variant(ot):
    f, g = I.blob_pair(256, 256, s=41)
    out = []
    for kw in ({"autotune": 1}, {"fft_variant": 0}):
        p = plan(ot, 256, 256, "mixed", tau=4.0, tol=1e-8, eta=1e-1, max_newton=400, **kw)
        phi = dev(np.zeros((256, 256)))
        rc, st = p.solve(dev(f), dev(g), phi)
        # the variants in use read back in the encoding the option takes
        v = p.get("fft_variant")
        assert v == 0 if "fft_variant" in kw else 0 <= v <= 2047
        assert p.get("tau") == 4.0 and p.get("precision") == 1
        p.close()
        assert rc == 0 and st["status"] == 0
        out.append(phi.cpu().numpy())
    # both converge to ||res||_inf <= 1e-8; the potentials agree to the mixed-mode bound
    assert np.abs(out[0] - out[1]).max() <= 1e-6


# ---------------------------------------------------------------------------------------
def _gpu_solve(ot, f, g, prec="fp64", tau=2.0, tol=1e-10, **kw):
    N, M = f.shape
    p = plan(ot, N, M, prec, tau=tau, tol=tol, **kw)
    fd, gd = dev(f), dev(g)
    phi = dev(np.zeros((N, M)))
    rc, st = p.solve(fd, gd, phi)
    p.close()
    return rc, st, phi.cpu().numpy()


@pytest.mark.parametrize("N", [16, 32, 64])
def test_solve_manufactured_fp64_matches_oracle(ot, N):
    f, g, phi_star = I.manufactured(N, N)
    u_ref, st_ref, hres, hgm = O.solve(f, g, tau=2.0, tol=1e-10, eta=1e-4)
    rc, st, phi = _gpu_solve(ot, f, g, "fp64", eta=1e-4)
    assert rc == 0 and st_ref["status"] == 0
    assert st["newton_iters"] == st_ref["newton_iters"]
    assert abs(st["gmres_iters"] - st_ref["gmres_iters"]) <= 2
    assert np.abs(phi - u_ref).max() <= 1e-10
    assert st["res_inf"] < 1e-10
    assert abs(st["res_l2"] - st_ref["res_l2"]) <= 1e-11


@pytest.mark.parametrize("N", [32, 64])
def test_solve_manufactured_mixed(ot, N):
    f, g, _ = I.manufactured(N, N)
    u_ref, st_ref, _, _ = O.solve(f, g, tau=2.0, tol=1e-10, eta=1e-4)
    rc, st, phi = _gpu_solve(ot, f, g, "mixed", eta=1e-4)
    assert rc == 0 and st["res_inf"] < 1e-10
    assert np.abs(phi - u_ref).max() <= 1e-6
    # the mixed result certifies itself through the oracle's FP64 residual
    F, _, s = O.residual(f, O.bspline_coeffs(g), phi)
    assert s["res_inf"] < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_simplified_operator(ot, prec):
    # OT_OPT_OPERATOR = 1 (Sec. 3.3 remark): the coefficients lose the grad g term (b = 0),
    # F and a are unchanged; the solve follows another Newton path to the oracle's root
    N, M = 64, 96
    f = I.blob_density(N, M, 51)
    g = I.blob_density(N, M, 52)
    u = smooth_field(N, M, amp=2e-3)
    c = O.bspline_coeffs(g)
    with O.simplified_operator():
        F_ref, coef_ref, _ = O.residual(f, c, u)
    p = plan(ot, N, M, prec, operator=1)
    assert p.get("operator") == 1
    fd, cd, ud = dev(f), dev(c), dev(u)
    Fd, coefd = dev(np.zeros((N, M))), dev(np.zeros((5, N, M)))
    scal = np.zeros(10)
    assert ot.ot_eval_residual(p.h, ptr(fd), ptr(cd), ptr(ud), ptr(Fd), ptr(coefd),
                               hptr(scal)) == 0
    cg = coefd.cpu().numpy()
    assert not cg[3:].any()
    rel = 1e-12 if prec == "fp64" else 1e-6
    assert np.abs(cg[:3] - coef_ref[:3]).max() <= rel * np.abs(coef_ref[:3]).max()
    p.close()
    fm, gm, _ = I.manufactured(32, 32)
    u_full, st_full, _, _ = O.solve(fm, gm, tau=2.0, tol=1e-10, eta=1e-2)
    with O.simplified_operator():
        u_simp, st_simp, _, _ = O.solve(fm, gm, tau=2.0, tol=1e-10, eta=1e-2)
    rc, st, phi = _gpu_solve(ot, fm, gm, prec, eta=1e-2, operator=1)
    assert st_full["status"] == 0 and st_simp["status"] == 0
    assert rc == 0 and st["res_inf"] < 1e-10
    if prec == "fp64":
        # the oracle's solve on the same (simplified) Newton path: the same steps, and the
        # iterate within the FP64 bound of the other FP64 parity tests
        assert st["newton_iters"] == st_simp["newton_iters"]
        assert np.abs(phi - u_simp).max() <= 1e-10
    # against the full operator's root (another Newton path): both iterates have max|F| <
    # 1e-10, so they differ by at most ||J^-1|| 2e-10 (the oracle's two solves are 1.2e-12
    # apart; the inverse's size is ~0.03, Sec. 5.1): 1e-10 in FP64; mixed: the refinement's
    # bound 1e-6
    assert np.abs(phi - u_full).max() <= (1e-10 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("symbols", [0, 1])
def test_solve_uniform_target_breakdown_path(ot, prec, symbols):
    # g = 1: at u = 0 the coefficients are a = I, b = 0, so L = Lbar and the preconditioned
    # operator is the identity.  The first Arnoldi step then has w in span(v_0): the
    # single-reduction step finds ||w||^2 - h^2 at round-off level, ends the cycle without a
    # convergence claim, and the restart's explicit residual (zero) finishes the linear solve.
    # The solve must still reach the oracle's root.
    N = 64
    f = I.blob_density(N, N, 31)
    g = np.ones((N, N))
    with O.fd_symbols(symbols):
        u_ref, st_ref, _, _ = O.solve(f, g, tau=2.0, tol=1e-10, eta=1e-4)
    rc, st, phi = _gpu_solve(ot, f, g, prec, eta=1e-4, symbols=symbols)
    assert st_ref["status"] == 0 and rc == 0 and st["res_inf"] < 1e-10
    assert np.abs(phi - u_ref).max() <= (1e-10 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("N,M", [(32, 32), (48, 64), (64, 48)])
def test_solve_blob_pair_fp64_with_safeguard(ot, N, M):
    # Long safeguarded runs with an inexact inner solve (eta = 1e-2) may take a different
    # path: one borderline GMRES stop changes theta at the eta level.  The converged
    # potential is unique (it is the root of the discrete residual), so it is compared;
    # two roots with max|F| < tol differ by about ||J^-1|| 2 tol ~ 0.06 tol.
    f, g = I.blob_pair(N, M, s=1000 + N + M)
    u_ref, st_ref, _, _ = O.solve(f, g, tau=2.0, tol=1e-10, eta=1e-2, max_newton=400)
    rc, st, phi = _gpu_solve(ot, f, g, "fp64", tol=1e-10, eta=1e-2, max_newton=400)
    assert st_ref["status"] == 0 and rc == 0
    assert np.abs(phi - u_ref).max() <= 1e-10
    assert abs(st["newton_iters"] - st_ref["newton_iters"]) <= 3
    assert st_ref["step_halvings"] >= 1 and st["step_halvings"] >= 1


def test_safeguard_off_diverges_like_oracle(ot):
    f, g = I.blob_pair(32, 32)
    _, st_ref, _, _ = O.solve(f, g, tau=2.0, tol=1e-6, eta=1e-2, max_newton=40,
                              safeguard=False)
    rc, st, _ = _gpu_solve(ot, f, g, "fp64", tol=1e-6, eta=1e-2, max_newton=40, safeguard=0)
    assert st_ref["status"] == O.ORC_EDIVERGED and rc == ot.OT_EDIVERGED
    assert st["newton_iters"] == st_ref["newton_iters"]


def test_equal_densities_and_invalid_inputs(ot):
    f = I.blob_density(32, 32, 5)
    rc, st, phi = _gpu_solve(ot, f, f.copy(), "fp64")
    assert rc == 0 and st["newton_iters"] == 0 and np.abs(phi).max() == 0
    bad = f.copy()
    bad[4, 7] = -10.0
    with pytest.raises(ot.OTError):
        _gpu_solve(ot, bad, f)
    bad[4, 7] = np.nan
    with pytest.raises(ot.OTError):
        _gpu_solve(ot, f, bad)
    rc, h = ot.ot_plan_create(30, 30, 2.0, 1e-8)
    assert rc == ot.OT_EUNSUPPORTED
    rc, h = ot.ot_plan_create(32, 32, 0.5, 1e-8)
    assert rc == ot.OT_EINVAL


def test_max_newton_cap(ot):
    f, g, _ = I.manufactured(32, 32)
    rc, st, _ = _gpu_solve(ot, f, g, "fp64", max_newton=3)
    assert rc == ot.OT_ENOCONV and st["newton_iters"] == 3


def test_solve_host_buffers_equal_device(ot):
    import ctypes
    f, g = I.blob_pair(64, 64, s=77)
    rc, st, phi = _gpu_solve(ot, f, g, "mixed", tol=1e-8, eta=1e-2)
    p = plan(ot, 64, 64, "mixed", tau=2.0, tol=1e-8, eta=1e-2)
    fh, gh = np.ascontiguousarray(f), np.ascontiguousarray(g)
    ph = np.zeros((64, 64))
    sth = ot.ot_stats()
    rc2 = ot.ot_solve_host(p.h, hptr(fh), hptr(gh), hptr(ph), sth)
    p.close()
    assert rc == rc2 == 0
    assert np.array_equal(ph, phi)


def test_batched_uneven_sizes(ot):
    import ctypes
    import torch
    sizes = [(32, 32), (48, 96), (64, 64), (24, 48)]
    plans, fs, gs, phis, refs = [], [], [], [], []
    for k, (N, M) in enumerate(sizes):
        f, g = I.blob_pair(N, M, s=4000 + k)
        refs.append(_gpu_solve(ot, f, g, "mixed", tol=1e-8, eta=1e-2)[2])
        plans.append(plan(ot, N, M, "mixed", tau=2.0, tol=1e-8, eta=1e-2))
        fs.append(dev(f))
        gs.append(dev(g))
        phis.append(dev(np.zeros((N, M))))
    stats = (ot.ot_stats * len(sizes))()
    rc = ot.ot_solve_plans(len(sizes), [p.h for p in plans], [t.data_ptr() for t in fs],
                             [t.data_ptr() for t in gs], [t.data_ptr() for t in phis],
                             stats)
    assert rc == 0
    for k in range(len(sizes)):
        assert stats[k].status == 0
        assert np.array_equal(phis[k].cpu().numpy(), refs[k])
    for p in plans:
        p.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_solve_equals_host_driven_solve(ot, prec):
    # the captured graph runs the same kernels in the same order as the host-driven loop;
    # every reduction is deterministic, so the results agree bit for bit
    for (N, M), gen in (((32, 32), lambda: I.manufactured(32, 32)[:2]),
                        ((48, 64), lambda: I.blob_pair(48, 64, s=99))):
        f, g = gen()
        out = []
        for graph in (1, 0):
            p = plan(ot, N, M, prec, tau=2.0, tol=1e-10, eta=1e-2, max_newton=300, graph=graph)
            phi = dev(np.zeros((N, M)))
            rc, st = p.solve(dev(f), dev(g), phi)
            out.append((rc, st, phi.cpu().numpy()))
            # a second solve on the same plan reuses the captured graph
            phi2 = dev(np.zeros((N, M)))
            rc2, st2 = p.solve(dev(f), dev(g), phi2)
            assert rc2 == rc and np.array_equal(phi2.cpu().numpy(), out[-1][2])
            p.close()
        (r1, s1, a1), (r0, s0, a0) = out
        assert r1 == r0 == 0
        for k in ("newton_iters", "gmres_iters", "gmres_cycles", "step_halvings"):
            assert s1[k] == s0[k], k
        # the host loop also launches the no-op steps of finished cycles; the graph does not
        assert 0 < s1["kernel_launches"] <= s0["kernel_launches"]
        assert np.array_equal(a1, a0)


def test_warm_start_from_solution_takes_no_step(ot):
    f, g = I.blob_pair(32, 32, s=5)
    rc, st, phi = _gpu_solve(ot, f, g, "fp64", tol=1e-9, eta=1e-2, max_newton=300)
    p = plan(ot, 32, 32, "fp64", tau=2.0, tol=1e-9, eta=1e-2, warm_start=1)
    phid = dev(phi)
    rc2, st2 = p.solve(dev(f), dev(g), phid)
    p.close()
    assert rc == rc2 == 0 and st2["newton_iters"] == 0
    assert np.abs(phid.cpu().numpy() - phi).max() < 1e-15


@pytest.mark.parametrize("N,M,variant", [(256, 256, 0), (192, 384, 0), (1024, 1024, 0),
                                         (1024, 1024, 128), (1024, 1024, 63 + 256 + 512),
                                         (2048, 256, 63 + 256), (256, 2048, 63 + 512)])
def test_fp32_operator_norm_accuracy(ot, N, M, variant):
    # The FP32 operator must stay at FP32 round-off in the 2-norm (a few 1e-7 per FFT pass,
    # ~1e-6 for the whole matvec), also for inputs whose spectrum spans many decades
    # (a smooth field plus small high-frequency noise, like a Newton residual late in the
    # iteration): the k1 = 0 and k1 = M/2 channels share one complex column and must not
    # swamp each other.
    f = I.blob_density(N, M, 31)
    g = I.blob_density(N, M, 32)
    u = smooth_field(N, M, amp=2e-3)
    c = O.bspline_coeffs(g)
    p64, p32 = plan(ot, N, M, "fp64"), plan(ot, N, M, "mixed", fft_variant=variant)
    fd, cd, ud = dev(f), dev(c), dev(u)
    coefd, scal = dev(np.zeros((5, N, M))), np.zeros(10)
    assert ot.ot_eval_residual(p64.h, ptr(fd), ptr(cd), ptr(ud), ptr(dev(np.zeros((N, M)))),
                               ptr(coefd), hptr(scal)) == 0
    abar = scal[5:].copy()
    rng = np.random.default_rng(3)
    inputs = [rng.standard_normal((N, M)),
              smooth_field(N, M, amp=1.0, kmax=3) + 1e-4 * rng.standard_normal((N, M))]
    for x in inputs:
        xd = dev(x)
        w64, w32 = dev(np.zeros((N, M))), dev(np.zeros((N, M)))
        t64, t32 = dev(np.zeros((N, M))), dev(np.zeros((N, M)))
        assert ot.ot_apply_operator(p64.h, ptr(coefd), hptr(abar), ptr(xd), ptr(w64)) == 0
        assert ot.ot_apply_operator(p32.h, ptr(coefd), hptr(abar), ptr(xd), ptr(w32)) == 0
        assert ot.ot_apply_lbar_inverse(p64.h, hptr(abar), ptr(xd), ptr(t64)) == 0
        assert ot.ot_apply_lbar_inverse(p32.h, hptr(abar), ptr(xd), ptr(t32)) == 0
        ew = float((w32 - w64).norm() / w64.norm())
        et = float((t32 - t64).norm() / t64.norm())
        assert ew <= 2e-6 and et <= 2e-6, (ew, et)
    p64.close()
    p32.close()


def test_theta_precision_modes(ot):
    # theta's inverse transforms in double-float (default), FP64 or FP32: all reach the
    # tolerance at the same root; double-float and FP64 take the same Newton path
    N = M = 128
    f, g = I.noise_blob_pair(N, M, s=3300)
    out = {}
    for theta in (2, 1, 0):
        p = plan(ot, N, M, "mixed", tau=1.0, tol=1e-8, eta=0.1, theta_fp64=theta,
                 max_newton=300)
        phi = dev(np.zeros((N, M)))
        rc, st = p.solve(dev(f), dev(g), phi)
        p.close()
        assert rc == 0 and st["res_inf"] < 1e-8
        out[theta] = (phi.cpu().numpy(), st)
    assert abs(out[2][1]["newton_iters"] - out[1][1]["newton_iters"]) <= 1
    assert np.abs(out[2][0] - out[1][0]).max() <= 1e-9
    assert np.abs(out[0][0] - out[1][0]).max() <= 1e-6



@pytest.mark.parametrize("N,M", [(256, 256), (512, 1024), (2048, 64)])
def test_theta_pairs_keep_the_root(ot, N, M):
    # theta's double-float passes on column / row pairs (OT_OPT_THETA_PAIRS, the default)
    # against one column / row per thread group: the double-float inverse transforms are the
    # same arithmetic and only the FP32 forward column transform rounds differently, so both
    # take the same Newton path to the same root (within the double-float / FP64 bound of the
    # theta modes)
    f, g = I.noise_blob_pair(N, M, s=3710)
    out = {}
    for pairs in (1, 0):
        p = plan(ot, N, M, "mixed", tau=1.0, tol=1e-8, eta=1e-2, symbols=1, theta_pairs=pairs,
                 max_newton=300)
        assert p.get("theta_pairs") == pairs
        phi = dev(np.zeros((N, M)))
        rc, st = p.solve(dev(f), dev(g), phi)
        p.close()
        assert rc == 0 and st["res_inf"] < 1e-8
        out[pairs] = (phi.cpu().numpy(), st)
    assert abs(out[1][1]["newton_iters"] - out[0][1]["newton_iters"]) <= 1
    assert np.abs(out[1][0] - out[0][0]).max() <= 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_stencil_symbol_solve_matches_oracle(ot, prec):
    # with the stencils' symbols the operator is the exact linearisation of F; at tau = 1
    # the FP64 path takes the oracle's Newton steps and both reach the same root
    N = M = 32
    f, g = I.blob_pair(N, M, s=8)
    with O.fd_symbols():
        u_ref, st_ref, _, _ = O.solve(f, g, tau=1.0, tol=1e-10, eta=1e-1)
    p = plan(ot, N, M, prec, tau=1.0, tol=1e-10 if prec == "fp64" else 1e-8, eta=1e-1,
             symbols=1, max_newton=300)
    phi = dev(np.zeros((N, M)))
    rc, st = p.solve(dev(f), dev(g), phi)
    p.close()
    assert rc == 0 and st_ref["status"] == 0
    if prec == "fp64":
        assert st["newton_iters"] == st_ref["newton_iters"]
        assert np.abs(phi.cpu().numpy() - u_ref).max() <= 1e-10
    else:
        assert np.abs(phi.cpu().numpy() - u_ref).max() <= 1e-6


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_eisenstat_walker_forcing(ot, prec):
    # adaptive GMRES tolerance: same root as the fixed tolerance, graph = host-driven
    N = M = 64
    f, g = I.noise_blob_pair(N, M, s=3400)
    out = []
    for forcing, graph in ((0, 1), (1, 1), (1, 0)):
        p = plan(ot, N, M, prec, tau=1.0, tol=1e-9, eta=1e-2, symbols=1, forcing=forcing,
                 graph=graph, max_newton=300)
        phi = dev(np.zeros((N, M)))
        rc, st = p.solve(dev(f), dev(g), phi)
        p.close()
        assert rc == 0 and st["res_inf"] < 1e-9
        out.append((phi.cpu().numpy(), st))
    assert np.abs(out[0][0] - out[1][0]).max() <= (1e-10 if prec == "fp64" else 1e-6)
    assert np.array_equal(out[1][0], out[2][0])
    assert out[1][1]["newton_iters"] == out[2][1]["newton_iters"]


def test_tau_retry_after_divergence(ot):
    # without the safeguard the blob pair diverges at tau = 2 (as in the oracle); with
    # OT_OPT_TAU_RETRY the solve restarts with twice tau until it converges to the root
    f, g = I.blob_pair(32, 32)
    rc0, st0, _ = _gpu_solve(ot, f, g, "fp64", tol=1e-6, eta=1e-2, max_newton=400,
                             safeguard=0)
    assert rc0 == ot.OT_EDIVERGED
    rc, st, phi = _gpu_solve(ot, f, g, "fp64", tol=1e-9, eta=1e-2, max_newton=400,
                             safeguard=0, tau_retry=4)
    assert rc == 0
    # an independent safeguarded oracle solve reaches the same root
    u_ref, st_ref, _, _ = O.solve(f, g, tau=4.0, tol=1e-10, eta=1e-2, max_newton=400)
    assert st_ref["status"] == 0
    assert np.abs(phi - u_ref).max() <= 1e-8


@pytest.mark.parametrize("graph", [1, 0])
def test_solve_fills_every_stats_field(ot, graph):
    # mass defects of the inputs (Eq. translation), the transport distance of Sec. 5.2 at the
    # returned potential, and the device time per phase (stamps at the phase changes, in the
    # graph-launched and the host-driven solve alike)
    N = M = 64
    f, g = I.noise_blob_pair(N, M, s=3700)
    f2, g2 = 1.3 * f, 0.8 * g
    p = plan(ot, N, M, "mixed", tau=1.0, tol=1e-8, eta=1e-2, symbols=1, graph=graph,
             phase_times=1, transport=1)
    phi = dev(np.zeros((N, M)))
    rc, st = p.solve(dev(f2), dev(g2), phi)
    assert rc == 0
    assert abs(st["mass_defect_f"] - (f2.mean() - 1.0)) <= 1e-13
    assert abs(st["mass_defect_g"] - (g2.mean() - 1.0)) <= 1e-13
    ph = phi.cpu().numpy()
    d_ref, _ = O.transport_outputs(f2 - f2.mean() + 1.0, ph)
    assert abs(st["transport_dist"] - d_ref) <= 1e-10 * d_ref
    ms = [st[k] for k in ("ms_residual", "ms_fft", "ms_krylov", "ms_update", "ms_other")]
    assert all(m > 0.0 for m in ms), ms
    assert sum(ms) <= 1.05 * st["ms_total"] + 0.02, (ms, st["ms_total"])
    # the same solve without the options: same result, the fields read -1
    p.set(phase_times=0, transport=0)
    phi2 = dev(np.zeros((N, M)))
    rc2, st2 = p.solve(dev(f2), dev(g2), phi2)
    p.close()
    assert rc2 == 0 and np.array_equal(phi2.cpu().numpy(), ph)
    assert st2["transport_dist"] == -1.0 and st2["ms_fft"] == -1.0 and st2["ms_other"] == -1.0
    assert st2["mass_defect_f"] == st["mass_defect_f"]


def test_per_class_device_times(ot):
    # OT_OPT_PHASE_TIMES = 2: stamps at every change of kernel class; the profile returns
    # the device ms per class of the last (graph-launched) solve, the phase fields are the
    # sums of their classes, and the result is that of the unstamped solve
    N = M = 64
    f, g = I.noise_blob_pair(N, M, s=3701)
    p = plan(ot, N, M, "mixed", tau=1.0, tol=1e-8, eta=1e-2, symbols=1, phase_times=2)
    phi = dev(np.zeros((N, M)))
    rc, st = p.solve(dev(f), dev(g), phi)
    assert rc == 0
    prof, _ = p.profile()
    for k in ("residual", "row_r2c", "col_matvec", "row_c2r_combine", "gmres_dots",
              "gmres_update", "col_lbarinv", "row_c2r_update"):
        assert prof[k][0] > 0.0, (k, prof)
    fft = prof["row_r2c"][0] + prof["col_matvec"][0] + prof["row_c2r_combine"][0]
    assert abs(st["ms_fft"] - fft) <= 1e-9 + 1e-9 * fft
    assert abs(st["ms_residual"] - prof["residual"][0]) <= 1e-9
    assert sum(v[0] for v in prof.values()) <= 1.05 * st["ms_total"] + 0.02
    p.set(phase_times=0)
    phi2 = dev(np.zeros((N, M)))
    rc2, st2 = p.solve(dev(f), dev(g), phi2)
    p.close()
    assert rc2 == 0 and np.array_equal(phi2.cpu().numpy(), phi.cpu().numpy())


def test_graph_shape_options_keep_the_result(ot):
    # OT_OPT_UNCOND_STEPS (plain Arnoldi steps before the WHILE tail) and OT_OPT_L2_PERSIST
    # change the graph, not the arithmetic: bit-identical potentials and counts;
    # OT_OPT_KRYLOV_BLOCKS changes the block partial sums of the Krylov reductions: the same
    # root within the mixed-mode bound
    N = M = 128
    f, g = I.noise_blob_pair(N, M, s=3702)
    base = dict(tau=1.0, tol=1e-8, eta=1e-2, symbols=1)
    results = {}
    for key, val in (("uncond_steps", 4), ("uncond_steps", 0), ("uncond_steps", 7),
                     ("uncond_steps", 10), ("l2_persist", 1), ("krylov_blocks", 1),
                     ("krylov_blocks", 4)):
        p = plan(ot, N, M, "mixed", **base, **{key: val})
        phi = dev(np.zeros((N, M)))
        rc, st = p.solve(dev(f), dev(g), phi)
        p.close()
        assert rc == 0 and st["res_inf"] < 1e-8, (key, val, st)
        results[(key, val)] = (phi.cpu().numpy(), st["newton_iters"], st["gmres_iters"])
    ref = results[("uncond_steps", 4)]
    for k in (("uncond_steps", 0), ("uncond_steps", 7), ("uncond_steps", 10),
              ("l2_persist", 1)):
        assert np.array_equal(results[k][0], ref[0]) and results[k][1:] == ref[1:], k
    for k in (("krylov_blocks", 1), ("krylov_blocks", 4)):
        assert np.abs(results[k][0] - ref[0]).max() <= 1e-6, k


@pytest.mark.parametrize("N,M", [(128, 128), (48, 64), (64, 256), (64, 512), (16, 2048)])
@pytest.mark.parametrize("variant", [0, 3, 3 + 1024])
def test_fused_update_keeps_the_result(ot, N, M, variant):
    # OT_OPT_FUSED_UPDATE: the Arnoldi update fused with the next product's row pass (row
    # pass variant 0: 8 elements per thread, 3: 4, + 1024: on row pairs where the row length
    # allows, else 4) against the two separate launches:
    # bit-identical potentials and counts, graph and host-driven, over several restart
    # cycles (eta 1e-4, m = 5: cycles end at their last step as well as on convergence)
    f, g = I.noise_blob_pair(N, M, s=3703)
    base = dict(tau=1.0, tol=1e-8, eta=1e-4, symbols=1, restart=5, fft_variant=variant)
    results = {}
    for fused in (1, 0):
        for graph in (1, 0):
            p = plan(ot, N, M, "mixed", graph=graph, fused_update=fused, **base)
            phi = dev(np.zeros((N, M)))
            rc, st = p.solve(dev(f), dev(g), phi)
            assert rc == 0 and st["res_inf"] < 1e-8, (fused, graph, st)
            if fused and graph:
                assert p.time_kernel("gmres_update", reps=3) > 0.0
            p.close()
            results[(fused, graph)] = (phi.cpu().numpy(), st["newton_iters"],
                                       st["gmres_iters"], st["step_halvings"])
    ref = results[(0, 1)]
    assert ref[2] > 5 * ref[1]  # cycles restarted
    for k, r in results.items():
        assert np.array_equal(r[0], ref[0]) and r[1:] == ref[1:], k


def test_untranslated_inputs_are_checked(ot):
    # OT_OPT_TRANSLATE = 0: inputs are used as given, so they must be positive as they are;
    # the statistics still report the mass defects
    N = M = 32
    f = I.blob_density(N, N, 5)
    for graph in (1, 0):
        rc, st, phi = _gpu_solve(ot, f, f.copy(), "fp64", translate=0, graph=graph)
        assert rc == 0 and st["newton_iters"] == 0
        assert abs(st["mass_defect_f"]) <= 1e-14
        bad = f.copy()
        bad[3, 3] = -0.5
        with pytest.raises(ot.OTError):
            _gpu_solve(ot, bad, f, "fp64", translate=0, graph=graph)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_inverse_spectral_radius_matches_oracle(ot, prec):
    # Sec. 5.1's power iteration on the inverse of the linearised operator, at the
    # manufactured solution and at a blob pair's start, from the same seeded b0 (uniform in
    # [0, 1] like the paper's): the norms follow the oracle's step for step (FP64: the GMRES
    # solves agree to round-off; mixed: FP32 Krylov vectors and transforms, 1e-5)
    cases = [(I.manufactured(32, 32)[:2], I.manufactured(32, 32)[2]),
             (I.blob_pair(48, 64, s=1001), np.zeros((48, 64)))]
    for (f, g), u in cases:
        N, M = f.shape
        b0 = I.SplitMix64(80).uniform(N * M).reshape(N, M)
        for symbols in (0, 1):
            with O.fd_symbols(symbols):
                ref = O.inverse_spectral_radius(f, g, u, b0, iters=6, eta=1e-6)
            p = plan(ot, N, M, prec, eta=1e-6, symbols=symbols)
            rho = p.inverse_spectral_radius(dev(f), dev(g), dev(u), dev(b0), iters=6)
            p.close()
            tol = 1e-9 if prec == "fp64" else 1e-5
            assert np.abs(rho - ref).max() <= tol * ref.max(), (rho, ref)


@pytest.mark.parametrize("prec,graph", [("fp64", 1), ("fp64", 0), ("mixed", 1)])
def test_tau_schedule_matches_oracle(ot, prec, graph):
    # OT_OPT_TAU_SWITCH: tau = 2 until max|F| < 0.1, then 1 (the oracle's schedule); the FP64
    # path takes the oracle's Newton steps, both reach its root
    f, g = I.blob_pair(64, 64, s=1001)
    with O.fd_symbols():
        u_ref, st_ref, _, _ = O.solve(f, g, tau=2.0, tol=1e-10, eta=1e-2, max_newton=400,
                                      tau_switch=0.1)
    rc, st, phi = _gpu_solve(ot, f, g, prec, tau=2.0, tol=1e-10, eta=1e-2, symbols=1,
                             max_newton=400, tau_switch=0.1, graph=graph)
    assert st_ref["status"] == 0 and rc == 0
    if prec == "fp64":
        assert st["newton_iters"] == st_ref["newton_iters"]
        assert np.abs(phi - u_ref).max() <= 1e-10
    else:
        assert np.abs(phi - u_ref).max() <= 1e-6


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_interpolation_modes_residual_and_solve(ot, mode, prec):
    # OT_OPT_INTERP 1 (bilinear) / 2 (nearest node): g and its grid gradient interpolated at
    # the displaced points (Sec. 4 intro, Sec. 5.2, 5.3), against the oracle's modes.  The
    # displacement of u spans several cells so that cell and node choices vary.  Residual: as
    # test_residual_and_coefficients (FP64 round-off; mixed: double-float value, FP32
    # gradient); nearest: the node decision is taken in FP64 on both sides, so a disagreement
    # could only come from a tie within round-off (none in these fields)
    N, M = 64, 96
    f = I.blob_density(N, M, 61)
    g = I.blob_density(N, M, 62)
    u = smooth_field(N, M, amp=3e-3, kmax=3)
    name = {1: "bilinear", 2: "nearest"}[mode]
    with O.interpolation(name):
        F_ref, coef_ref, s_ref = O.residual(f, g, u)
    p = plan(ot, N, M, prec, interp=mode)
    fd, gd, ud = dev(f), dev(g), dev(u)
    Fd, coefd = dev(np.zeros((N, M))), dev(np.zeros((5, N, M)))
    scal = np.zeros(10)
    assert ot.ot_eval_residual(p.h, ptr(fd), ptr(gd), ptr(ud), ptr(Fd), ptr(coefd),
                               hptr(scal)) == 0
    p.close()
    eps = np.finfo(float).eps if prec == "fp64" else 2.0 ** -48
    tol = 32 * eps * np.abs(u).max() * max(N, M) ** 2 * np.abs(g).max() + 64 * eps * 10
    assert np.abs(Fd.cpu().numpy() - F_ref).max() <= tol
    assert abs(scal[3] - s_ref["min_det"]) <= tol
    cs = np.abs(coef_ref).max()
    ctol = (1e-12 if prec == "fp64" else 2e-6) * cs
    assert np.abs(coefd.cpu().numpy() - coef_ref).max() <= ctol
    # a blob pair in the mode: bilinear reaches the oracle's root; with the nearest node the
    # residual is piecewise constant in u and the iteration stalls near its floor, so (as the
    # paper's image runs, a fixed number of steps) both take 4 Newton steps and the iterates
    # are compared
    fb, gb = I.blob_pair(48, 64, s=1005)
    kw = dict(tau=1.0, tol=1e-9, eta=1e-2, max_newton=300 if mode == 1 else 4)
    with O.interpolation(name), O.fd_symbols():
        u_ref, st_ref, _, _ = O.solve(fb, gb, **kw)
    rc, st, phi = _gpu_solve(ot, fb, gb, prec, symbols=1, interp=mode, **kw)
    if mode == 1:
        assert st_ref["status"] == 0 and rc == 0
    else:
        assert st_ref["status"] == O.ORC_ENOCONV and rc == ot.OT_ENOCONV
        assert st["newton_iters"] == 4
    assert np.abs(phi - u_ref).max() <= (1e-10 if prec == "fp64" else 1e-6)
