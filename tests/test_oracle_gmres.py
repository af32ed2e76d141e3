"""Pins of the oracle's GMRES-IR (Sec. 4.2-4.3) against facts that do not come
from the oracle itself: the least-squares characterisation of a GMRES iterate,
finite termination, exact preconditioners, and the paper's printed claims."""
import numpy as np
import pytest

import irgen
import oracle as O


def _krylov_lstsq(M: np.ndarray, z: np.ndarray, k: int) -> np.ndarray:
    """argmin ||z - M d||_2 over d in span{z, M z, ..., M^{k-1} z}, by brute force:
    an orthonormal basis of the explicit power vectors, then a dense least-squares solve."""
    K = np.empty((z.shape[0], k))
    v = z / np.linalg.norm(z)
    for j in range(k):
        K[:, j] = v
        v = M @ v
        v = v / np.linalg.norm(v)
    Q, _ = np.linalg.qr(K)
    c, *_ = np.linalg.lstsq(M @ Q, z, rcond=None)
    return Q @ c


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gmres_iterate_is_the_krylov_least_squares_minimiser(seed):
    rng = np.random.default_rng(700 + seed)
    n = 9
    M = rng.standard_normal((n, n)) + 2.0 * np.eye(n)
    z = rng.standard_normal(n)
    for k in range(1, n):
        d, kk, est = O.gmres(lambda v: M @ v, z, k, 0.0)
        assert kk == k
        dref = _krylov_lstsq(M, z, k)
        res, res_ref = np.linalg.norm(z - M @ d), np.linalg.norm(z - M @ dref)
        assert abs(res - res_ref) <= 1e-10 * np.linalg.norm(z)
        np.testing.assert_allclose(d, dref, rtol=0, atol=1e-8 * np.linalg.norm(dref))
        # the rotations' estimate is the true residual norm of the iterate
        assert abs(est[-1] - res) <= 1e-10 * np.linalg.norm(z)
        # estimates never increase (each Krylov space contains the previous)
        assert all(est[i + 1] <= est[i] * (1 + 1e-12) for i in range(len(est) - 1))


def test_gmres_finite_termination_solves_the_system():
    rng = np.random.default_rng(711)
    n = 7
    M = rng.standard_normal((n, n)) + 3.0 * np.eye(n)
    z = rng.standard_normal(n)
    d, k, _ = O.gmres(lambda v: M @ v, z, n, 0.0)
    assert k == n
    np.testing.assert_allclose(d, np.linalg.solve(M, z), rtol=1e-11, atol=1e-12)


def test_gmres_one_step_closed_form():
    """k = 1: d = alpha z with alpha = <M z, z> / ||M z||^2 (a one-dimensional least squares)."""
    rng = np.random.default_rng(712)
    M = rng.standard_normal((6, 6)) + 2.0 * np.eye(6)
    z = rng.standard_normal(6)
    d, k, _ = O.gmres(lambda v: M @ v, z, 1, 0.0)
    Mz = M @ z
    assert k == 1
    np.testing.assert_allclose(d, (Mz @ z) / (Mz @ Mz) * z, rtol=1e-13)


def test_gmres_breakdown_on_an_eigenvector():
    """z an eigenvector of M: the Krylov space is one-dimensional, h_21 = 0, d = z / lambda."""
    M = np.diag([4.0, 2.0, 3.0, 5.0])
    z = np.array([0.0, 3.0, 0.0, 0.0])
    d, k, _ = O.gmres(lambda v: M @ v, z, 4, 0.0)
    assert k == 1
    np.testing.assert_array_equal(d, z / 2.0)


def test_gmres_stops_at_the_tolerance():
    rng = np.random.default_rng(713)
    n = 30
    M = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / np.sqrt(n)
    z = rng.standard_normal(n)
    _, _, est_all = O.gmres(lambda v: M @ v, z, n, 0.0)
    beta = np.linalg.norm(z)
    for eta in (1e-1, 1e-4, 1e-8):
        d, k, est = O.gmres(lambda v: M @ v, z, n, eta)
        first = next(j for j, e in enumerate(est_all) if e <= eta * beta) + 1
        assert k == first
        assert np.linalg.norm(z - M @ d) <= eta * beta * (1 + 1e-8)


def test_gmres_zero_right_hand_side():
    d, k, est = O.gmres(lambda v: 2.0 * v, np.zeros(5), 5, 1e-8)
    assert k == 0 and not est
    np.testing.assert_array_equal(d, np.zeros(5))


def test_precondition_is_the_scaled_lu_solve():
    """P w for an exactly factorable A: diagonal entries that are powers of two
    (binary32 LU and solve exact), so P w = A^{-1} w to the last bit."""
    diag = np.array([2.0, -0.5, 4.0, 1.0, 0.25, 8.0])
    A = np.asfortranarray(np.diag(diag))
    LU, ipiv, info = O.getrf_tf(O.cast(A, O.F32), O.F32)
    assert info == 0
    w = np.array([3.0, -1.0, 0.5, 8.0, 2.0, -6.0])     # ||w|| = 8: w / ||w|| exact in binary32
    np.testing.assert_array_equal(O.precondition(LU, ipiv, 1.0, w), w / diag)
    np.testing.assert_array_equal(O.precondition(LU, ipiv, 1.0, np.zeros(6)), np.zeros(6))
    # binary16 scale s: A_F = s A, P w = s (A_F)^{-1} w
    np.testing.assert_array_equal(O.precondition(LU, ipiv, 4.0, w), 4.0 * (w / diag))


def test_gmres_ir_exact_preconditioner_one_krylov_step():
    diag = np.array([2.0, -0.5, 4.0, 1.0, 0.25, 8.0, 16.0, -2.0])
    A = np.asfortranarray(np.diag(diag))
    b = np.array([1.0, 2.0, -3.0, 0.5, 1.5, -1.0, 4.0, 0.25])
    res = O.gmres_ir_solve(A, b, O.F32)
    assert res.status == O.CONVERGED
    assert res.khist == [1]
    np.testing.assert_array_equal(res.x, b / diag)


def test_matvec_is_the_binary64_product():
    rng = np.random.default_rng(714)
    A = np.asfortranarray(rng.integers(-8, 8, (12, 12)).astype(np.float64))
    v = rng.integers(-8, 8, 12).astype(np.float64)
    np.testing.assert_array_equal(O.matvec(A, v), A @ v)    # small integers: exact


def test_gmres_ir_rescues_half_precision_where_ir_fails():
    """Sec. 4.3: with a binary16 factorization of the ill-conditioned I - 800 G,
    IR does not converge but GMRES-IR, using the same factors as a
    preconditioner, does (soft pin of the paper's claim, at N = 256)."""
    A, b = irgen.case_green(256, 800.0)
    xref = O.reference_solution(A, b)
    kappa = O.cond_inf(A)
    ir = O.ir_solve(A, b, O.F16)
    gm = O.gmres_ir_solve(A, b, O.F16)
    assert ir.status == O.MAXIT
    assert O.rel_err_inf(ir.x, xref) > O.parity_tol(kappa, O.F64)
    assert O.rel_err_inf(gm.x, xref) <= O.parity_tol(kappa, O.F64)
    assert gm.status in (O.CONVERGED, O.STAGNATED)
    assert all(1 <= k <= 10 for k in gm.khist)
    assert len(gm.khist) == gm.iters


def test_gmres_ir_residual_stagnation_reading():
    """The half-precision GMRES-IR history of Sec. 4.5 continues past a residual
    ratio of 0.69: with the refinement loop's R_max = 0.5 it would have stopped a
    step early; with the Krylov-IR factor R_max_r = 1 it stops where printed."""
    rh = [9.88752e+01, 1.86920e-03, 1.29700e-03, 2.46429e-03]
    eps = 2.0 ** -23
    assert O.term_decide(rh[:3], [1.0, 1.0], rh[0], eps, O.Term(), False) == O.STAGNATED
    assert O.term_decide(rh[:3], [1.0, 1.0], rh[0], eps, O.Term(), False, rmax_r=1.0) is None
    assert O.term_decide(rh, [1.0] * 3, rh[0], eps, O.Term(), False, rmax_r=1.0) == O.STAGNATED


def test_gmres_ir_well_conditioned_matches_ir_accuracy():
    A, b = irgen.case_green(200, 1.0)
    xref = O.reference_solution(A, b)
    gm = O.gmres_ir_solve(A, b, O.F32)
    assert gm.status == O.CONVERGED
    assert O.rel_err_inf(gm.x, xref) <= 1e-14
    # a binary32 preconditioner of a kappa ~ 1 matrix: the 1e-8 tolerance in 2-3 steps
    assert all(k <= 3 for k in gm.khist)


def test_gmres_ir_edge_cases():
    A = np.asfortranarray(np.eye(3))
    res = O.gmres_ir_solve(A, np.zeros(3), O.F32)
    assert res.status == O.CONVERGED and res.iters == 0 and res.khist == []
    A = np.asfortranarray(np.array([[1.0, 2.0], [2.0, 4.0]]))
    res = O.gmres_ir_solve(A, np.ones(2), O.F32)
    assert res.status == O.FAILED and res.info == 2


# ---------------------------------------------------------------------------
# BiCGSTAB (Sec. 2.3, 4.2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1])
def test_bicgstab_finite_termination_and_true_residual(seed):
    """In exact arithmetic BiCGSTAB ends within n iterations; in binary64 on a small,
    well-conditioned nonsymmetric system it reaches the solution, and the residual its
    recurrence carries equals the true residual z - M d."""
    rng = np.random.default_rng(720 + seed)
    n = 8
    M = rng.standard_normal((n, n)) + 4.0 * np.eye(n)
    z = rng.standard_normal(n)
    d, k, est = O.bicgstab(lambda v: M @ v, z, 3 * n, 1e-14)
    assert k <= n + 2
    np.testing.assert_allclose(d, np.linalg.solve(M, z), rtol=1e-11, atol=1e-12)
    for kk in range(1, k + 1):
        dk, _, ek = O.bicgstab(lambda v: M @ v, z, kk, 0.0)
        assert abs(np.linalg.norm(z - M @ dk) - ek[-1]) <= 1e-10 * np.linalg.norm(z)


def test_bicgstab_omega_minimises_the_step_residual():
    """omega = <t, s>/<t, t> is the one-dimensional least-squares choice: the
    first iterate's residual s - omega t is no larger than with a perturbed omega."""
    rng = np.random.default_rng(722)
    n = 12
    M = rng.standard_normal((n, n)) + 3.0 * np.eye(n)
    z = rng.standard_normal(n)
    d, k, est = O.bicgstab(lambda v: M @ v, z, 1, 0.0)
    assert k == 1
    alpha = (z @ z) / (z @ (M @ z))
    s = z - alpha * (M @ z)
    t = M @ s
    for dw in (-1e-3, 1e-3, 0.1):
        om = (t @ s) / (t @ t) + dw
        assert est[-1] <= np.linalg.norm(s - om * t) + 1e-15
    # and the iterate is alpha z + omega s (the two search directions of step one)
    coef, *_ = np.linalg.lstsq(np.stack([z, s], 1), d, rcond=None)
    np.testing.assert_allclose(np.stack([z, s], 1) @ coef, d, rtol=1e-12, atol=1e-14)
    assert abs(coef[0] - alpha) <= 1e-12 * abs(alpha)


def test_bicgstab_identity_one_iteration_and_zero_rhs():
    z = np.array([1.0, -2.0, 3.0, 0.5])
    d, k, est = O.bicgstab(lambda v: v, z, 10, 1e-8)
    assert k == 1 and est[-1] == 0.0
    np.testing.assert_array_equal(d, z)
    d, k, est = O.bicgstab(lambda v: v, np.zeros(4), 10, 1e-8)
    assert k == 0 and not est


def test_bicgstab_ir_rescues_half_precision_and_agrees_with_gmres_ir():
    A, b = irgen.case_green(256, 800.0)
    xref = O.reference_solution(A, b)
    tol = O.parity_tol(O.cond_inf(A), O.F64)
    bi = O.bicgstab_ir_solve(A, b, O.F16)
    gm = O.gmres_ir_solve(A, b, O.F16)
    assert bi.status in (O.CONVERGED, O.STAGNATED)
    assert O.rel_err_inf(bi.x, xref) <= tol
    assert O.rel_err_inf(bi.x, gm.x) <= tol
    assert all(1 <= k <= 10 for k in bi.khist)
