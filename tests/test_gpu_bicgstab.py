"""Parity of the CUDA BiCGSTAB-IR (Sec. 2.3, 4.2) with the oracle's BiCGSTAB-IR."""
import numpy as np
import pytest

import irgen
import oracle as O
from gpu_util import dev_colmajor, dev_vec
from paper_2311_14616_gb300 import ir

pytestmark = pytest.mark.gpu

OK = ("converged", "stagnated")


def _cases():
    yield "green_a800_N512_f16", lambda: irgen.case_green(512, 800.0), O.F16
    yield "green_a800_N700_bf16", lambda: irgen.case_green(700, 800.0), O.BF16
    yield "gauss_N1000_f16", lambda: irgen.case_gaussian(1000, 12), O.F16
    yield "random_N300_f32", lambda: irgen.case_random(300, 3), O.F32
    yield "green_a800_N4097_f16", lambda: irgen.case_green(4097, 800.0), O.F16   # two rows per thread
    yield "gauss_N7_f16", lambda: irgen.case_gaussian(7, 5), O.F16


@pytest.mark.parametrize("name,make,tf", list(_cases()), ids=[c[0] for c in _cases()])
def test_bicgstab_ir_matches_oracle(ctx, name, make, tf):
    A, b = make()
    f = ctx.factor(dev_colmajor(A), tf=O.DTYPE_NAMES[tf])
    x, rep = f.solve_bicgstab(dev_vec(b))
    x = x.cpu().numpy()
    ref = O.bicgstab_ir_solve(A, b, tf, nb=64)
    n = A.shape[0]
    xr = O.reference_solution(A, b) if n <= 1000 else ref.x
    tol = O.parity_tol(O.cond_inf(A) if n <= 1000 else 1.9e5, O.F64)
    assert rep.status in OK and O.STATUS_NAMES[ref.status] in OK, (rep.status, ref.status)
    assert rep.rhist[0] == ref.rhist[0]
    # as for GMRES-IR: the step that ends at the rounding floor moves with the
    # binary32 noise of the preconditioner, the result does not
    assert abs(rep.iters - ref.iters) <= 3, (rep.iters, ref.iters, rep.rhist, ref.rhist)
    assert len(rep.khist) == rep.iters
    for kg, ko in zip(rep.khist, ref.khist):
        assert abs(kg - ko) <= 2, (rep.khist, ref.khist)
    assert O.rel_err_inf(x, ref.x) <= tol, (O.rel_err_inf(x, ref.x), tol)
    assert O.rel_err_inf(x, xr) <= tol, (O.rel_err_inf(x, xr), tol)


@pytest.mark.parametrize("name,make,tf", [
    ("gauss_N1000_f16", lambda: irgen.case_gaussian(1000, 12), O.F16),
    ("green_a800_N600_f16", lambda: irgen.case_green(600, 800.0), O.F16),
    ("random_N300_f32", lambda: irgen.case_random(300, 3), O.F32),
])
def test_bicgstab_step_matches_oracle_on_the_same_factors(ctx, name, make, tf):
    """One refinement step with one BiCGSTAB iteration (eta = 0), the oracle run on the
    GPU's own factors: d = alpha p + omega s must agree to the binary32 noise of P."""
    A, b = make()
    f = ctx.factor(dev_colmajor(A), tf=O.DTYPE_NAMES[tf])
    LU, piv = f.factors(), f.pivots()
    x, rep = f.solve_bicgstab(dev_vec(b), term=ir.default_term(litmax=1),
                              kopts=ir.krylov_opts(basissize=1, eta=0.0))
    ref = O.bicgstab_ir_solve(A, b, tf, O.Term(litmax=1), O.KrylovOpts(basissize=1, eta=0.0),
                              factors=(LU, piv))
    assert rep.khist == ref.khist == [1]
    d, do = x.cpu().numpy(), ref.x
    tol = max(2e-5, 0.1 * O.cond_inf(A) * 2.0 ** -24)
    err = float(np.max(np.abs(d - do))) / float(np.max(np.abs(do)))
    assert err <= tol, (err, tol)
    assert abs(rep.dhist[0] - ref.dhist[0]) <= tol * ref.dhist[0]


def test_bicgstab_ir_exact_preconditioner(ctx):
    diag = np.array([2.0, -0.5, 4.0, 1.0, 0.25, 8.0, 16.0, -2.0] * 80)
    A = np.asfortranarray(np.diag(diag))
    b = np.round(np.linspace(-512.0, 512.0, 640))
    f = ctx.factor(dev_colmajor(A), tf="f32")
    x, rep = f.solve_bicgstab(dev_vec(b))
    ref = O.bicgstab_ir_solve(A, b, O.F32)
    assert rep.status == O.STATUS_NAMES[ref.status] == "converged"
    assert rep.khist == ref.khist
    assert O.rel_err_inf(x.cpu().numpy(), b / diag) <= 4 * 2.0 ** -52


def test_bicgstab_ir_single_precision_working(ctx):
    """TW = binary32, TR = binary64 wider (eq. wilkterm), as in the BiCGSTAB-IR
    example of Sec. 2.3: the solution of the promoted problem."""
    A64, _ = irgen.case_green(400, 799.0, rule="trapezoid")
    A = np.asfortranarray(A64.astype(np.float32))
    b = (A.astype(np.float64) @ np.ones(400)).astype(np.float32)
    f = ctx.factor(dev_colmajor(A), tf="f16")
    x, rep = f.solve_bicgstab(dev_vec(b), term=ir.default_term(litmax=20))
    ref = O.bicgstab_ir_solve(A, b, O.F16, O.Term(litmax=20), nb=64)
    assert rep.status == O.STATUS_NAMES[ref.status] == "stagnated"
    assert O.rel_err_inf(x.cpu().numpy(), O.reference_solution(A, b)) <= 2.0 ** -23


def test_bicgstab_ir_full_size_closed_form(ctx):
    A, b, xt = irgen.case_green_sine(8192)
    f = ctx.factor(dev_colmajor(A), tf="f16")
    f.bicgstab_reserve()
    x, rep = f.solve_bicgstab(dev_vec(b))
    assert rep.status in OK
    assert all(1 <= k <= 10 for k in rep.khist)
    assert O.rel_err_inf(x.cpu().numpy(), xt) <= O.parity_tol(1.818e5 * 1.01, O.F64)


def test_bicgstab_ir_edge_cases(ctx):
    A, b = irgen.case_gaussian(64, 3)
    f = ctx.factor(dev_colmajor(A), tf="f16")
    x, rep = f.solve_bicgstab(dev_vec(np.zeros(64)))
    assert rep.status == "converged" and rep.iters == 0
    np.testing.assert_array_equal(x.cpu().numpy(), np.zeros(64))
    with pytest.raises(ir.IRError, match="IR_EINVAL"):
        f.solve_bicgstab(dev_vec(b), kopts=ir.krylov_opts(basissize=0))
    # repeated solves are deterministic, and GMRES-IR on the same factors agrees
    x1, r1 = f.solve_bicgstab(dev_vec(b))
    x2, r2 = f.solve_bicgstab(dev_vec(b))
    np.testing.assert_array_equal(x1.cpu().numpy(), x2.cpu().numpy())
    xg, _ = f.solve_gmres(dev_vec(b))
    assert O.rel_err_inf(x1.cpu().numpy(), xg.cpu().numpy()) <= 1e-12
