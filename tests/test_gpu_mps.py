"""Mixed precision solves (MPS, Sec. 5.3: mplu(A; onthefly = true)) on the GPU.

The correction d = s U^{-1} L^{-1} P r is evaluated in TW = binary64 on the
binary32 factors promoted exactly (k_trsv64.cu), r is not scaled by ||r||.
Checked against the oracle's ir_solve(solve="mps"): the same status, the
iteration count within one, and x within the parity bar of both the oracle's
MPS result and x_ref; the residual history the paper prints for
mplu(A; onthefly = true) in Sec. 2.2.1 reproduced; exact factors give A^{-1} b
in one step; TW = binary32 (solves in binary32 with no scaling).
"""
import numpy as np
import pytest
import torch

import irgen
import oracle as O
import parity as P
from gpu_util import dev_colmajor, dev_vec
from paper_2311_14616_gb300 import ir

pytestmark = pytest.mark.gpu


def _cases():
    # systems where the oracle's own MPS refinement meets the bar (kappa u_F < 1 for
    # the factorization precision; binary16 factors of I - 800 G do not converge)
    yield "green_a800_N520_f32", lambda: irgen.case_green_sine(520)[:2], O.F32
    yield "green_a100_N700_f16", lambda: irgen.case_green(700, 100.0), O.F16
    yield "gauss_N700_bf16", lambda: irgen.case_gaussian(700, 19), O.BF16
    yield "gauss_N1000_tf32", lambda: irgen.case_gaussian(1000, 14), O.TF32
    yield "random_N300_f32", lambda: irgen.case_random(300, 13), O.F32
    yield "green_a1_N129_f16", lambda: irgen.case_green(129, 1.0), O.F16
    yield "gauss_N1_f32", lambda: irgen.case_gaussian(1, 3), O.F32
    yield "gauss_N5000_f16", lambda: irgen.case_gaussian(5000, 15), O.F16


@pytest.mark.parametrize("name,make,tf", list(_cases()), ids=[c[0] for c in _cases()])
def test_mps_matches_oracle(ctx, name, make, tf):
    A, b = make()
    f = ctx.factor(dev_colmajor(A), tf=O.DTYPE_NAMES[tf], onthefly=True)
    x, rep = f.solve(dev_vec(b))
    x = x.cpu().numpy()
    ref = O.ir_solve(A, b, tf, nb=64, solve="mps")
    xr = O.reference_solution(A, b)
    tol = P.bar(O.cond_inf(A) if A.shape[0] <= 2000 else float(np.linalg.cond(A, np.inf)))
    assert rep.status == O.STATUS_NAMES[ref.status], (rep.rhist, ref.rhist)
    assert abs(rep.iters - ref.iters) <= 1
    assert rep.rhist[0] == ref.rhist[0]
    assert O.rel_err_inf(ref.x, xr) <= tol          # the oracle meets the bar: compare
    assert O.rel_err_inf(x, ref.x) <= tol, O.rel_err_inf(x, ref.x)
    assert O.rel_err_inf(x, xr) <= tol, O.rel_err_inf(x, xr)


def test_mps_reproduces_paper_onthefly_history(ctx, golden):
    """Sec. 2.2.1: mplu(A; onthefly = true) for A = I - Gmat(4096) (trapezoid),
    b = A 1.  The binary32 factors are bitwise the oracle's (and the paper's).
    The first correction's residual is set by the factorization error alone and
    is the printed one to the printed digits; from the second step on the
    residual is ~1e-11 out of |A||x| ~ 2, so its own rounding (the summation
    order of r = b - A x, a fixed split-K order here, the BLAS order in the
    paper and in the oracle) shows in the 4th digit; the loop takes the printed
    number of steps to eps."""
    g = golden("paper_values.json")["ir_double_single_onthefly_alpha1_N4096"]
    A, _ = irgen.case_green(4096, 1.0, rule="trapezoid")
    n = A.shape[0]
    b = -O.residual(A, np.zeros(n), np.ones(n))
    f = ctx.factor(dev_colmajor(A), tf="f32", onthefly=True)
    x, rep = f.solve(dev_vec(b))
    assert rep.status == "converged"
    got = [float("%.5e" % v) for v in rep.rhist]
    assert got[:2] == g["rhist"][:2], got
    assert abs(rep.rhist[2] / g["rhist"][2] - 1) < 1e-2, rep.rhist
    assert rep.rhist[3] <= 2 * g["rhist"][3], rep.rhist
    assert len(rep.rhist) == len(g["rhist"]) and rep.rhist[-1] <= 4 * 2.0 ** -52
    # against the solution of the rounded b (b = A 1 carries its own rounding, so
    # x = 1 is not the exact solution; the oracle, whose residual sums in the
    # order b was formed in, sees r(1) = 0 and returns 1)
    # within what the binary64 residual itself resolves (sqrt(n) u |A||x| times ||A^-1||)
    xr = O.reference_solution(A, b)
    assert O.rel_err_inf(x.cpu().numpy(), xr) <= 2 * np.sqrt(n) * 2.0 ** -52 * O.cond_inf(A)
    # binary32 solves of the same factors take another path
    g32 = ctx.factor(dev_colmajor(A), tf="f32")
    _, rep32 = g32.solve(dev_vec(b))
    assert [float("%.5e" % v) for v in rep32.rhist][:2] != g["rhist"][:2]


def test_mps_exact_factors_solve_in_one_step(ctx):
    """Diagonal A with powers of two: L = I and U = A exactly in every TF, so the
    binary64 solve gives A^{-1} b exactly and IR stops after one step with a
    zero residual; the binary32 solve of fl32(r / ||r||) cannot (b has more
    bits than binary32)."""
    n = 300
    g = np.random.Generator(np.random.PCG64(5))
    d = 2.0 ** g.integers(-3, 4, size=n)
    A = np.asfortranarray(np.diag(d))
    b = g.standard_normal(n)
    for tf in ("f32", "f16"):
        f = ctx.factor(dev_colmajor(A), tf=tf, onthefly=True)
        x, rep = f.solve(dev_vec(b))
        np.testing.assert_array_equal(x.cpu().numpy(), b / d)
        assert rep.iters == 1 and rep.status == "converged" and rep.rhist[1] == 0.0
        f_lps = ctx.factor(dev_colmajor(A), tf=tf)
        _, rep_lps = f_lps.solve(dev_vec(b))
        assert rep_lps.iters > 1


def test_mps_single_precision_working_type(ctx):
    """TW = binary32 (TR = binary64 wider): r rounded to binary32, binary32 solves
    with no scaling; same status as the oracle's MPS, result within its bound."""
    n = 384
    A, b = irgen.case_svd(n, 1004, kappa=1e4)
    f = ctx.factor(dev_colmajor(A), tf="f32", onthefly=True)
    x, rep = f.solve(dev_vec(b))
    ref = O.ir_solve(A, b, O.F32, solve="mps")
    assert rep.status == O.STATUS_NAMES[ref.status]
    xp = O.reference_solution(A, b)
    bound = 4 * (n + 1) * O.cond_inf(A) * 2.0 ** -53 + 2.0 ** -24
    assert x.dtype == torch.float32
    assert O.rel_err_inf(x.cpu().numpy(), xp) <= bound


def test_mps_host_entry_point_and_many_rhs(ctx):
    A, b = irgen.case_green(640, 100.0)
    xh, rep = ctx.solve_host(torch.from_numpy(A), torch.from_numpy(b), tf="f16", onthefly=True)
    ref = O.ir_solve(A, b, O.F16, nb=64, solve="mps")
    assert rep.status == O.STATUS_NAMES[ref.status]
    assert O.rel_err_inf(xh.numpy(), O.reference_solution(A, b)) <= P.bar(O.cond_inf(A))
    f = ctx.factor(dev_colmajor(A), tf="f16", onthefly=True)
    B = np.stack([b, 2 * b, np.zeros_like(b)], axis=1)
    X, reps = f.solve_many(torch.from_numpy(B).cuda())
    X = X.cpu().numpy()
    assert reps[2].status == "converged" and reps[2].iters == 0
    assert O.rel_err_inf(X[:, 0], xh.numpy()) <= 1e-14


@pytest.mark.parametrize("name,make,tf", [
    ("green_a100_N700_f16", lambda: irgen.case_green(700, 100.0), O.F16),
    ("gauss_N700_bf16", lambda: irgen.case_gaussian(700, 19), O.BF16),
], ids=["green_a100_N700_f16", "gauss_N700_bf16"])
def test_mps_on_factors_kept_in_two_bytes(ctx, name, make, tf):
    """Mixed precision solves on factors kept in TF (store_tf): the oracle rounds
    its factors to TF once and promotes them in its binary64 solves; the GPU's
    status, steps (within one) and x agree with it."""
    A, b = make()
    f = ctx.factor(dev_colmajor(A), tf=O.DTYPE_NAMES[tf], onthefly=True, store_tf=True)
    x, rep = f.solve(dev_vec(b))
    x = x.cpu().numpy()
    ref = O.ir_solve(A, b, tf, nb=64, solve="mps", store_tf=True)
    xr = O.reference_solution(A, b)
    tol = P.bar(O.cond_inf(A))
    assert rep.status == O.STATUS_NAMES[ref.status], (rep.rhist, ref.rhist)
    assert abs(rep.iters - ref.iters) <= 1
    assert O.rel_err_inf(ref.x, xr) <= tol
    assert O.rel_err_inf(x, ref.x) <= tol, O.rel_err_inf(x, ref.x)
    assert O.rel_err_inf(x, xr) <= tol, O.rel_err_inf(x, xr)
