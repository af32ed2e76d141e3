"""Pins of the CPU oracle against facts the paper and mathematics fix.

Nothing here compares the oracle with itself: each test checks it against an
exact rational computation, a library conversion routine, a closed form, a
rounding-error bound, or numbers printed in the paper.
"""
from fractions import Fraction

import itertools
import os

import numpy as np
import pytest

import irgen
import oracle as O


# ---------------------------------------------------------------------------
# rounding to TF (the copy operator I_W^F, Sec. 1)
# ---------------------------------------------------------------------------

def _special_f32():
    vals = [0.0, -0.0, 1.0, -1.0, 1.5, 3.0e-8, 6.0e-5, 6.1e-5, 65504.0, 65519.0, 65520.0, 7e4,
            1e-40, 1e-45, 3.4e38, -2.5e-41, 1 + 2 ** -11, 1 + 3 * 2 ** -11, 1 + 2 ** -8, 1 + 3 * 2 ** -8,
            2 ** -24, 2 ** -25, 3 * 2 ** -26, 2 ** -14 - 2 ** -25]
    rng = np.random.Generator(np.random.PCG64(7))
    rnd = rng.standard_normal(20000) * np.exp(rng.uniform(-30, 30, 20000))
    bits = rng.integers(0, 2 ** 32, 20000, dtype=np.uint64).astype(np.uint32).view(np.float32)
    x = np.concatenate([np.array(vals, dtype=np.float32), rnd.astype(np.float32), bits])
    return x[np.isfinite(x)]


def test_round_fp16_matches_numpy():
    x = _special_f32()
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).astype(np.float32)   # numpy: round-to-nearest-even
    got = O.round_tf(x, O.F16)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    x = _special_f32()
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    got = O.round_tf(x, O.BF16)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_round_tf32_ties_away_and_bits():
    # exact halfway cases round away from zero; others to nearest
    one = np.float32(1.0)
    ulp = 2.0 ** -10
    cases = {1 + ulp / 2: 1 + ulp, -(1 + ulp / 2): -(1 + ulp), 1 + 3 * ulp / 2: 1 + 2 * ulp,
             1 + ulp / 2 - 2 ** -23: 1.0, float(np.finfo(np.float32).max): np.inf}
    for v, want in cases.items():
        assert O.round_tf(np.array([v], np.float32), O.TF32)[0] == np.float32(want), v
    # the result keeps 10 fraction bits: low 13 bits of the binary32 encoding are zero
    x = _special_f32()
    got = O.round_tf(x, O.TF32)
    fin = np.isfinite(got)
    assert not np.any(got[fin].view(np.uint32) & 0x1FFF)
    # and is within half a TF32 ulp of the input (relative 2^-11, normal range)
    nrm = fin & (np.abs(x) > 2.0 ** -120)
    assert np.all(np.abs(got[nrm].astype(np.float64) - x[nrm]) <= np.abs(x[nrm]) * 2.0 ** -11 * (1 + 2 ** -10))
    assert O.round_tf(np.array([one]), O.F32)[0] == one


def test_cast_is_elementwise_rounding_and_fp16_scaling():
    A, _ = irgen.case_gaussian(37, 5)
    for tf in (O.F32, O.TF32, O.BF16):
        AF = O.cast(A, tf)
        ref = O.round_tf(A.astype(np.float32).ravel(order="F"), tf).reshape(A.shape, order="F")
        assert np.array_equal(AF, ref)
    s = O.fp16_scale(A)
    assert s == 1024.0 / np.max(np.abs(A))
    AF = O.cast(A, O.F16, s)
    assert np.max(np.abs(AF)) == 1024.0          # the largest entry lands on 2^10
    ref = (s * A).astype(np.float32).astype(np.float16).astype(np.float32)
    assert np.array_equal(AF, ref)


# ---------------------------------------------------------------------------
# LU with partial pivoting (Algorithm IR, "Factor A = LU")
# ---------------------------------------------------------------------------

def _exact_lu(A):
    """Gaussian elimination with partial pivoting in exact rational arithmetic.

    Pivot = first row with maximal |a_ik|.  Returns (perm, L, U) as Fractions."""
    n = len(A)
    M = [[Fraction(float(A[i][j])) for j in range(n)] for i in range(n)]
    perm = list(range(n))
    ipiv = []
    for k in range(n):
        p = max(range(k, n), key=lambda i: (abs(M[i][k]), -i))
        ipiv.append(p)
        M[k], M[p] = M[p], M[k]
        perm[k], perm[p] = perm[p], perm[k]
        if M[k][k] == 0:
            continue
        for i in range(k + 1, n):
            M[i][k] = M[i][k] / M[k][k]
            for j in range(k + 1, n):
                M[i][j] -= M[i][k] * M[k][j]
    return ipiv, M


def _exact_solve(A, b):
    n = len(A)
    M = [[Fraction(float(A[i][j])) for j in range(n)] + [Fraction(float(b[i]))] for i in range(n)]
    for k in range(n):
        p = max(range(k, n), key=lambda i: abs(M[i][k]))
        M[k], M[p] = M[p], M[k]
        for i in range(n):
            if i != k and M[i][k] != 0:
                f = M[i][k] / M[k][k]
                M[i] = [a - f * c for a, c in zip(M[i], M[k])]
    return [M[i][n] / M[i][i] for i in range(n)]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lu_f64_exact_rational(n, seed):
    A, b = irgen.case_random(n, 100 + seed)
    LU, ipiv, info = O.getrf_f64(A)
    eipiv, M = _exact_lu(A)
    assert info == 0
    assert list(ipiv) == eipiv                              # same pivot order as exact arithmetic
    for i in range(n):
        for j in range(n):
            ex = float(M[i][j])
            assert abs(LU[i, j] - ex) <= 64 * 2 ** -52 * max(1.0, abs(ex)) * n
    # solve + one refinement step reaches the exact solution to a few ulps
    x = O.getrs_f64(LU, ipiv, b)
    x = x + O.getrs_f64(LU, ipiv, O.residual(A, b, x, extended=True))
    xe = [float(v) for v in _exact_solve(A, b)]
    for xi, ei in zip(x, xe):
        assert abs(xi - ei) <= 4 * 2 ** -52 * abs(ei) + 1e-300


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_lu_f32_pivots_and_factors_exact_on_small(n):
    # binary32 factorization of binary32 data: pivots equal exact-arithmetic ones
    A, _ = irgen.case_random(n, 300 + n)
    AF = O.cast(A, O.F32)
    LU, ipiv, info = O.getrf_tf(AF, O.F32)
    eipiv, M = _exact_lu(AF)
    assert list(ipiv) == eipiv
    for i in range(n):
        for j in range(n):
            assert abs(LU[i, j] - float(M[i][j])) <= 64 * 2 ** -23 * max(1.0, abs(float(M[i][j])))


def _rows_with_small_multipliers(A):
    """Brute force over every row order of a tiny matrix: the orders whose LU
    without interchanges, in exact arithmetic, has all |l_ik| <= 1."""
    n = A.shape[0]
    keep = []
    for order in itertools.permutations(range(n)):
        M = [[Fraction(float(A[r][j])) for j in range(n)] for r in order]
        ok = True
        for k in range(n):
            if M[k][k] == 0:
                ok = all(M[i][k] == 0 for i in range(k + 1, n))
                if not ok:
                    break
                continue
            for i in range(k + 1, n):
                l = M[i][k] / M[k][k]
                if abs(l) > 1:
                    ok = False
                    break
                for j in range(k + 1, n):
                    M[i][j] -= l * M[k][j]
            if not ok:
                break
        if ok:
            keep.append(list(order))
    return keep


@pytest.mark.parametrize("n", [2, 3, 4, 5])
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_lu_pivots_are_the_one_row_order_with_small_multipliers(n, seed):
    """Partial pivoting (first row of maximal |a_ik| at every step) is the unique
    row order whose unpivoted LU has every multiplier of magnitude <= 1 when no
    two candidates tie; the oracle's interchanges must produce exactly it."""
    A, _ = irgen.case_random(n, 500 + 10 * n + seed)
    orders = _rows_with_small_multipliers(A)
    assert len(orders) == 1
    _, ipiv, info = O.getrf_f64(A)
    assert info == 0
    assert list(O.perm_from_ipiv(ipiv)) == orders[0]
    AF = O.cast(A, O.F32)
    _, ipiv32, _ = O.getrf_tf(AF, O.F32)
    assert list(O.perm_from_ipiv(ipiv32)) == _rows_with_small_multipliers(AF)[0]


def test_lu_tie_breaks_to_first_row_and_zero_pivot():
    A = np.asfortranarray(np.array([[1.0, 2.0, 0.0], [-3.0, 1.0, 1.0], [3.0, 5.0, 2.0]]))
    _, ipiv, info = O.getrf_f64(A)
    assert ipiv[0] == 1 and info == 0                   # |-3| = |3|: the first row wins
    _, ipiv32, _ = O.getrf_tf(A.astype(np.float32), O.F32)
    assert ipiv32[0] == 1
    S = np.asfortranarray(np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0], [1.0, 0.0, 1.0]]))
    _, _, info = O.getrf_f64(S)
    assert info == 3                                    # LAPACK-style 1-based first zero pivot
    _, _, info32 = O.getrf_tf(S.astype(np.float32), O.TF32, nb=2)
    assert info32 == 3


def _lu_backward(AF, LU, ipiv):
    n = AF.shape[0]
    P = O.perm_from_ipiv(ipiv)
    L = np.tril(LU.astype(np.float64), -1) + np.eye(n)
    U = np.triu(LU.astype(np.float64))
    E = AF.astype(np.float64)[P] - L @ U
    return E, L, U


def _matrices(n):
    yield "green1", irgen.case_green(n, 1.0)[0]
    yield "green800", irgen.case_green(n, 800.0)[0]
    yield "gauss", irgen.case_gaussian(n, 11)[0]
    yield "random", irgen.case_random(n, 12)[0]


@pytest.mark.parametrize("n", [1, 2, 7, 64, 130])
@pytest.mark.parametrize("tf", [O.F32, O.TF32, O.BF16, O.F16])
def test_lu_backward_error_bounds(n, tf):
    """||P A_F - LU|| / ||A_F|| <= 4 N u_F and |P A_F - LU| <= gamma_3N(u_F) |L||U| (eq. comperr)."""
    u = O.UNIT_ROUNDOFF[tf]
    for name, A in _matrices(n):
        s = O.fp16_scale(A) if tf == O.F16 else 1.0
        AF = O.cast(A, tf, s)
        LU, ipiv, info = O.getrf_tf(AF, tf, nb=16)
        assert info == 0
        E, L, U = _lu_backward(AF, LU, ipiv)
        nrm = np.max(np.abs(AF).sum(axis=1))
        assert np.max(np.abs(E).sum(axis=1)) <= 4 * n * u * nrm, name
        if 3 * n * u >= 1:     # eq. (comperr) needs 3 N u_F < 1
            continue
        g = 3 * n * u / (1 - 3 * n * u)
        assert np.all(np.abs(E) <= g * (np.abs(L) @ np.abs(U)) + 1e-30), name
        if tf != O.F32 and n > 16 and name == "random":
            # the TF rounding of the update operands is really applied:
            # the backward error is well above what binary32 alone gives
            assert np.max(np.abs(E)) > 64 * 2 ** -24 * np.max(np.abs(AF)), name


@pytest.mark.parametrize("tf", [O.TF32, O.BF16, O.F16])
def test_lu_tf_update_rounding_points_hand_worked(tf):
    """The trailing update of the TF factorization (reading of Sec. 5.4.1 eq.
    (comperr) with tensor-core operands): A22 <- fl32(A22 - fl32(sum_k
    rTF(l_ik) rTF(u_kj))), both operands rounded to TF, the exact products
    summed in binary64 and rounded to binary32 once per block.  Worked by
    hand on a 4 x 4 matrix with nb = 3 whose leading 3 x 3 block is I, so
    that L11 = U11 = I, l_3k = a_3k, u_k3 = a_k3 and no row moves:

        l_30 = 1/2,              u_03 = 2              -> product 1
        l_31 = 3*2^-13 + 2^-24,  u_13 = 2^-12 + 2^-24  -> rTF: 3*2^-13, 2^-12 -> 3*2^-25
        l_32 = -2^-13,           u_23 = 2^-12          -> -2^-25

    (2^-24 is below half the TF spacing at these values for TF32, bf16 and
    binary16, so rTF drops it.)  The exact sum is 1 + 2^-24, a binary32 tie
    that rounds to even: 1; so a_33 = 2 becomes 2 - 1 = 1.  Each plausible
    slip lands on 1 + 2^-23 instead and gives a_33 = 1 - 2^-23:
      * only L21 rounded: 3*2^-13 (2^-12 + 2^-24) pushes the sum above the tie;
      * only U12 rounded: (3*2^-13 + 2^-24) 2^-12 does the same;
      * no rounding at all: both perturbations, above the tie;
      * products summed in binary32: fl32(1 + 3*2^-25) = 1 + 2^-23, and
        subtracting 2^-25 keeps it there;
    and subtracting each product from a_33 in binary32 in turn ends at
    1 - 2^-23 too (two ties, both to even)."""
    A = np.zeros((4, 4))
    A[:3, :3] = np.eye(3)
    A[3, 0], A[0, 3] = 0.5, 2.0
    A[3, 1], A[1, 3] = 3 * 2.0 ** -13 + 2.0 ** -24, 2.0 ** -12 + 2.0 ** -24
    A[3, 2], A[2, 3] = -(2.0 ** -13), 2.0 ** -12
    A[3, 3] = 2.0
    AF = np.asfortranarray(A.astype(np.float32))
    assert np.array_equal(AF.astype(np.float64), A)       # every entry is binary32
    LU, ipiv, info = O.getrf_tf(AF, tf, nb=3)
    assert info == 0 and list(ipiv) == [0, 1, 2, 3]
    assert LU[3, 3] == np.float32(1.0)
    # the multipliers and U12 are stored unrounded (binary32 storage, reading 8)
    assert LU[3, 1] == AF[3, 1] and LU[1, 3] == AF[1, 3]
    # the same block with binary32 factors (no TF rounding, fmaf chain per entry)
    # takes another path: 2 - 1 - 3*2^-25 (rounded) + 2^-25
    LU32, _, _ = O.getrf_tf(AF, O.F32)
    assert LU32[3, 3] != np.float32(1.0)


def test_lu_tf_with_one_block_is_the_binary32_lu():
    # nb >= N: no trailing update happens, every TF path is the binary32 factorization
    A, _ = irgen.case_random(40, 21)
    AF = O.cast(A, O.TF32)
    a, pa, _ = O.getrf_tf(AF, O.TF32, nb=64)
    b, pb, _ = O.getrf_tf(AF, O.F32)
    assert np.array_equal(a, b) and np.array_equal(pa, pb)


def test_lu_forced_pivots_and_gap_report():
    A, _ = irgen.case_random(30, 22)
    AF = O.cast(A, O.F32)
    LU, ipiv, _, gap = O.getrf_tf(AF, O.F32, want_gap=True)
    assert np.all(gap[:, 0] == gap[:, 2])             # the row taken is the maximal one
    assert np.all(gap[:-1, 1] <= gap[:-1, 0])
    LU2, ipiv2, _ = O.getrf_tf(AF, O.F32, force_piv=ipiv)
    assert np.array_equal(LU, LU2) and np.array_equal(ipiv, ipiv2)
    forced = ipiv.copy()
    forced[0] = 0 if ipiv[0] != 0 else 1
    _, ipiv3, _, gap3 = O.getrf_tf(AF, O.F32, force_piv=np.where(np.arange(30) == 0, forced, -1), want_gap=True)
    assert ipiv3[0] == forced[0] and gap3[0, 2] < gap3[0, 0]


# ---------------------------------------------------------------------------
# triangular solves and residual
# ---------------------------------------------------------------------------

def test_getrs_f32_recovers_exact_integer_solution():
    rng = np.random.Generator(np.random.PCG64(3))
    n = 24
    L = np.tril(rng.integers(-2, 3, (n, n)), -1) + np.eye(n)
    U = np.triu(rng.integers(-2, 3, (n, n))).astype(np.float64)
    U[np.diag_indices(n)] = np.where(rng.random(n) < 0.5, 1.0, 2.0)
    y = rng.integers(-3, 4, n).astype(np.float64) * 2.0 ** -6
    ipiv = np.array([min(n - 1, k + (k % 3)) for k in range(n)], dtype=np.int32)
    v = L @ (U @ y)                                    # small integers times 2^-6: exact in binary32
    assert np.all(np.abs(v) < 2 ** 20)
    # P^T so that getrs's interchanges undo it
    Pv = v.copy()
    for k in reversed(range(n)):
        p = ipiv[k]
        Pv[[k, p]] = Pv[[p, k]]
    LU = np.asfortranarray((np.tril(L, -1) + U).astype(np.float32))
    got = O.getrs_f32(LU, ipiv, Pv.astype(np.float32))
    assert np.array_equal(got.astype(np.float64), y)


@pytest.mark.parametrize("tw", [np.float64, np.float32])
def test_residual_within_gamma_n_of_exact(tw):
    n = 9
    A, b = irgen.case_random(n, 31)
    A = np.asfortranarray(A.astype(tw))
    x = np.random.Generator(np.random.PCG64(32)).standard_normal(n)
    r = O.residual(A, b, x)
    rx = O.residual(A, b, x, extended=True)
    g = n * 2 ** -53 / (1 - n * 2 ** -53)
    for i in range(n):
        ex = Fraction(float(b[i])) - sum(Fraction(float(A[i, j])) * Fraction(float(x[j])) for j in range(n))
        bound = g * (np.abs(A[i]).astype(np.float64) @ np.abs(x)) + 2 ** -53 * abs(float(r[i]))
        assert abs(Fraction(r[i]) - ex) <= Fraction(bound)
        assert abs(Fraction(rx[i]) - ex) <= Fraction(2 ** -52) * abs(ex) + Fraction(bound) * Fraction(2 ** -10)


# ---------------------------------------------------------------------------
# input generators: the Green's operator (Sec. 2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [8, 64, 256])
def test_gmat_midpoint_closed_form_spectrum(n):
    h = 1.0 / n
    k = np.arange(1, n + 1)
    lam = np.sort(h * h / (4 * np.sin(k * np.pi * h / 2) ** 2))
    got = np.sort(np.linalg.eigvalsh(irgen.gmat_midpoint(n)))
    assert np.max(np.abs(got - lam) / lam) < 1e-11
    # largest eigenvalues approach the continuous ones 1/(k^2 pi^2) (Sec. 2)
    cont = 1.0 / (np.arange(1, 4) ** 2 * np.pi ** 2)
    assert np.max(np.abs(lam[::-1][:3] - cont) / cont) < 2.0 / n
    # the first eigenvector is sin(pi x_i)
    x = irgen.midpoint_nodes(n)
    v = np.sin(np.pi * x)
    Gv = irgen.gmat_midpoint(n) @ v
    assert np.max(np.abs(Gv - lam[-1] * v)) < 1e-14


def test_gmat_row_sums():
    n = 100
    x = irgen.midpoint_nodes(n)
    assert np.max(np.abs(irgen.gmat_midpoint(n).sum(axis=1) - (x * (1 - x) / 2 + 1 / (8 * n * n)))) < 1e-14
    xt = np.linspace(0, 1, n)
    assert np.max(np.abs(irgen.gmat_trapezoid(n).sum(axis=1) - xt * (1 - xt) / 2)) < 1e-14


@pytest.mark.slow
def test_trapezoid_condition_number_matches_paper(golden):
    g = golden("paper_values.json")["cond_inf_trapezoid_alpha799_N4096"]
    A, _ = irgen.case_green(4096, 799.0, rule="trapezoid")
    c = np.linalg.cond(A, np.inf)
    assert abs(c - g["value"]) / g["value"] < g["rel_tol"]


# ---------------------------------------------------------------------------
# termination (Sec. 5.1) and the IR loop (Algorithm IR)
# ---------------------------------------------------------------------------

def test_termination_replays_printed_histories(golden):
    for case in golden("termination_histories.json")["cases"]:
        term = O.Term(Rmax=case["Rmax"])
        rh, dh = case["rhist"], case.get("dhist")
        stop = None
        for k in range(1, len(rh)):
            d = dh[:k] if dh is not None else [1.0] * k
            st = O.term_decide(rh[:k + 1], d, case["bnorm"], case["eps_w"], term, case["tr_wider"],
                               rmax_r=case.get("Rmax_r"))
            if st is not None:
                stop = (k, O.STATUS_NAMES[st])
                break
        assert stop == (case["stop_index"], case["status"]), case["name"]


def test_termination_litmax_and_nonfinite():
    term = O.Term(litmax=3)
    rh = [1.0, 0.4, 0.16, 0.064]
    assert O.term_decide(rh[:3], [1, 1], 1.0, 2 ** -52, term, False) is None
    assert O.term_decide(rh, [1, 1, 1], 1.0, 2 ** -52, term, False) == O.MAXIT
    assert O.term_decide([1.0, np.nan], [1.0], 1.0, 2 ** -52, term, False) == O.DIVERGED
    assert O.term_decide([1.0, 1e-14], [1.0], 1.0, 2 ** -52, O.Term(abs_rel_tol=1e-13), False) == O.CONVERGED


def test_ir_reproduces_paper_double_single_history(golden):
    """A = I - Gmat(4096), b = A 1: the history printed in Sec. 2.2.1 (soft pin)."""
    g = golden("paper_values.json")["ir_double_single_alpha1_N4096"]
    A, _ = irgen.case_green(4096, 1.0, rule="trapezoid")
    n = A.shape[0]
    # b = A*x with x = ones, formed by the same matrix-vector product as the residual
    b = -O.residual(A, np.zeros(n), np.ones(n))
    res = O.ir_solve(A, b, O.F32)
    assert res.status == O.CONVERGED
    assert abs(len(res.rhist) - len(g["rhist"])) <= 1
    for got, want in zip(res.rhist, g["rhist"]):
        assert want / 10 <= got <= want * 10
    for got, want in zip(res.dhist, g["dhist"]):
        assert want / 10 <= got <= want * 10
    assert len(res.dhist) == len(res.rhist) - 1
    # Sec. 2.2 prints an error of 8.88178e-16 against x = ones for the IR solution
    assert O.rel_err_inf(res.x, np.ones(n)) < 10 * 8.88178e-16


def test_ir_mps_reproduces_paper_onthefly_history(golden):
    """Mixed precision solves (Sec. 5.3, onthefly = true): the residual history
    printed in Sec. 2.2.1 for A = I - Gmat(4096), b = A 1, digit for digit."""
    g = golden("paper_values.json")["ir_double_single_onthefly_alpha1_N4096"]
    A, _ = irgen.case_green(4096, 1.0, rule="trapezoid")
    n = A.shape[0]
    b = -O.residual(A, np.zeros(n), np.ones(n))
    res = O.ir_solve(A, b, O.F32, solve="mps")
    assert res.status == O.CONVERGED
    assert [float("%.5e" % v) for v in res.rhist] == g["rhist"]
    # the same factors with binary32 solves (eq. vdlow) take another path
    lps = O.ir_solve(A, b, O.F32)
    assert [float("%.5e" % v) for v in lps.rhist] != g["rhist"]


def test_ir_mps_half_precision_factors(golden):
    """TF = binary16 with mixed precision solves (the paper's default for half,
    Sec. 2.2.1): converges, within the printed iteration count."""
    g = golden("paper_values.json")["ir_double_half_alpha1_N4096"]
    A, _ = irgen.case_green(4096, 1.0, rule="trapezoid")
    n = A.shape[0]
    b = -O.residual(A, np.zeros(n), np.ones(n))
    res = O.ir_solve(A, b, O.F16, solve="mps")
    assert res.status == O.CONVERGED
    assert len(res.rhist) <= len(g["rhist"])
    assert res.rhist[1] <= 10 * g["rhist"][1]
    assert O.rel_err_inf(res.x, np.ones(n)) < 10 * 8.88178e-16


def test_ir_mps_solves_in_working_precision():
    """With factors that are exact (a diagonal of powers of two) a solve in TW =
    binary64 gives A^{-1} b exactly, so MPS stops after one step with r = 0;
    the binary32 solve of eq. (vdlow) rounds P r / ||r|| to binary32 first and
    needs further steps.  TW = binary32: the solve is binary32 on fl32(r)."""
    diag = np.array([2.0, -0.5, 4.0, 1.0, 0.25, 8.0, 16.0, -2.0] * 4)
    A = np.asfortranarray(np.diag(diag))
    b = np.random.default_rng(3).standard_normal(32)
    res = O.ir_solve(A, b, O.F32, solve="mps")
    assert res.status == O.CONVERGED and res.rhist[-1] == 0.0 and res.iters == 1
    np.testing.assert_array_equal(res.x, b / diag)
    lps = O.ir_solve(A, b, O.F32)
    assert lps.iters >= 2
    A32 = np.asfortranarray(A.astype(np.float32))
    b32 = b.astype(np.float32)
    r32 = O.ir_solve(A32, b32, O.F32, solve="mps")
    np.testing.assert_array_equal(r32.sol, b32 / diag.astype(np.float32))
    with pytest.raises(ValueError):
        O.ir_solve(A, b, O.F32, solve="hps")


def test_ir_tf_storage_hand_worked():
    """Factors kept in TF (store_tf).  A = [[3, 0], [1, 1]] (every entry exact in
    TF): the panel's binary32 scaling gives l21 = 1 * fl32(1/3), which is not a
    TF number, u11 = 3, u12 = 0, u22 = 1.  Stored in binary16, l21 becomes
    rTF(fl32(1/3)) = 1365 * 2^-12 = 0.333251953125 (bfloat16: 171 * 2^-9).  For
    b = (3, 0) the first step (eq. vdlow: rho = 3, v = (1, 0)) solves L y = v,
    U z = y: z2 = -l21, and d = rho z, so d2 = -3 l21: -0.999755859375 with
    binary16 storage, -1.001953125 with bfloat16, and -3 fl32(1/3) =
    -1.0000000298023224 (exact in binary64) when the binary32 multiplier is
    used."""
    A = np.asfortranarray(np.array([[3.0, 0.0], [1.0, 1.0]]))
    b = np.array([3.0, 0.0])
    third = float(np.float32(1.0) / np.float32(3.0))
    for tf, l21 in ((O.F16, 1365 * 2.0 ** -12), (O.BF16, 171 * 2.0 ** -9)):
        res = O.ir_solve(A, b, tf, fp16_scaling=False, store_tf=True, term=O.Term(litmax=1))
        assert res.LU[1, 0] == np.float32(l21)
        assert res.x[1] == -3 * l21
        plain = O.ir_solve(A, b, tf, fp16_scaling=False, term=O.Term(litmax=1))
        assert plain.LU[1, 0] == np.float32(third) and plain.x[1] == -3 * third == -1.0000000298023224
    with pytest.raises(ValueError):
        O.ir_solve(A, b, O.F32, store_tf=True)


@pytest.mark.parametrize("tf", [O.F16, O.BF16])
def test_ir_tf_storage_rounds_every_factor_once(tf):
    """The stored factors are exactly the TF roundings of the binary32 ones (every
    entry, diagonal included); exact factors are unchanged (a diagonal of powers
    of two solves in one step either way); IR with stored factors still converges
    on a well-conditioned system, with its contraction bounded by the storage
    error u_TF (|L||U|) of eq. (comperr)."""
    A, b = irgen.case_gaussian(150, 77)
    plain = O.ir_solve(A, b, tf, nb=64)
    st = O.ir_solve(A, b, tf, nb=64, store_tf=True)
    np.testing.assert_array_equal(st.LU, O.round_tf(plain.LU, tf).reshape(plain.LU.shape))
    assert np.array_equal(st.ipiv, plain.ipiv)
    assert st.status in (O.CONVERGED, O.STAGNATED)
    xr = O.reference_solution(A, b)
    assert O.rel_err_inf(st.x, xr) <= 1e-12
    h = st.rhist
    u = O.UNIT_ROUNDOFF[tf]
    kappa = O.cond_inf(A)
    assert h[1] / h[0] <= 4 * 150 * u * kappa      # first step's contraction, storage error included
    d = np.asfortranarray(np.diag(2.0 ** np.arange(-3, 5, dtype=float)))
    e = O.ir_solve(d, np.ones(8), tf, fp16_scaling=False, store_tf=True)
    assert e.iters == 1 and e.rhist[-1] == 0.0


@pytest.mark.parametrize("case,tf", [("I-G", O.F32), ("I-G", O.TF32), ("I-G", O.F16), ("gauss", O.F32)])
def test_ir_mps_contraction_within_rate_bound(case, tf):
    """Eq. (rate2) (Sec. 5.4.2): with mixed precision solves the residual
    contracts per step by at most alpha = u_F (||A|| + 13 sqrt(N) kappa(L)
    kappa(U)), infinity norms, while it is far above its rounding floor.  The
    bound is checked on cases where it is informative (alpha < 1), on the
    first two steps; then every step against the bound that adds the
    residual's rounding, and the final residual against the stagnation level
    of eq. (stagterm)."""
    n = 128
    A, b = (irgen.case_green(n, 1.0, rule="trapezoid") if case == "I-G" else irgen.case_gaussian(n, 7))
    s = O.fp16_scale(A) if tf == O.F16 else 1.0
    LU, _, _ = O.getrf_tf(O.cast(A, tf, s), tf, 64)
    L = np.tril(LU.astype(np.float64), -1) + np.eye(n)
    U = np.triu(LU.astype(np.float64))
    kappa = lambda M: np.linalg.norm(M, np.inf) * np.linalg.norm(np.linalg.inv(M), np.inf)
    u_f = {O.F32: 2.0 ** -23, O.TF32: 2.0 ** -10, O.BF16: 2.0 ** -7, O.F16: 2.0 ** -10}[tf]
    alpha = u_f * (np.linalg.norm(A, np.inf) + 13 * np.sqrt(n) * kappa(L) * kappa(U))
    res = O.ir_solve(A, b, tf, solve="mps", nb=64)
    assert alpha < 1
    for k in range(2):
        assert res.rhist[k + 1] <= alpha * res.rhist[k], (k, res.rhist, alpha)
    # Sec. 5.4.2 with the residual's own rounding (eqs. residerr, stagterm):
    # ||r_{k+1}|| <= alpha ||r_k|| + (1 + alpha)/(1 - alpha) xi at every step,
    # xi = gamma_N(u_W) (C ||A|| ||x*|| + ||b||), C the iterates' bound
    xs = O.reference_solution(A, b)
    gam = n * 2.0 ** -53 / (1 - n * 2.0 ** -53)
    c_bound = max(1.0, np.max(np.abs(res.x)) / np.max(np.abs(xs)))
    xi = gam * (c_bound * np.linalg.norm(A, np.inf) * np.max(np.abs(xs)) + np.max(np.abs(b)))
    floor = (1 + alpha) / (1 - alpha) * xi
    for k in range(len(res.rhist) - 1):
        assert res.rhist[k + 1] <= alpha * res.rhist[k] + floor, (k, res.rhist, alpha, floor)
    assert res.rhist[-1] <= floor


def test_ir_accuracy_alpha800_matches_table(golden):
    """alpha = 800, x = 1: converged error near Table ip3's ELP (soft)."""
    g = golden("paper_values.json")["accuracy_alpha800"]
    A, b = irgen.case_green(512, 800.0, rule="trapezoid", rhs="A1")
    res = O.ir_solve(A, b, O.F32)
    err = O.rel_err_inf(res.x, np.ones(512))
    assert err < 10 * g["ELP"][0]
    resid = np.max(np.abs(O.residual(A, b, res.x))) / np.max(np.abs(b))
    assert resid < 10 * g["RLP"][0]


def test_ir_green_sine_closed_form():
    """x_true = sin(pi x) is an eigenvector of G_mid, so A x_true = (1 - alpha lambda_1) x_true."""
    n, alpha = 384, 800.0
    A, b, xt = irgen.case_green_sine(n, alpha)
    h = 1.0 / n
    lam = np.sort(h * h / (4 * np.sin(np.arange(1, n + 1) * np.pi * h / 2) ** 2))
    mu = 1 - alpha * lam
    kappa2 = np.max(np.abs(mu)) / np.min(np.abs(mu))
    res = O.ir_solve(A, b, O.F32)
    assert res.status in (O.CONVERGED, O.STAGNATED)
    assert O.rel_err_inf(res.x, xt) <= 10 * kappa2 * 2 ** -52 * np.sqrt(n)


@pytest.mark.parametrize("tf", [O.TF32, O.BF16, O.F16])
def test_ir_low_precision_converges_on_well_conditioned(tf):
    A, b = irgen.case_gaussian(200, 41)
    res = O.ir_solve(A, b, tf, nb=32)
    xr = O.reference_solution(A, b)
    assert res.status in (O.CONVERGED, O.STAGNATED)
    kappa = O.cond_inf(A)
    assert O.rel_err_inf(res.x, xr) <= O.parity_tol(kappa, O.F64)


def test_ir_fp16_fails_on_ill_conditioned():
    """Half-precision factors of I - 800 G are not accurate enough (Sec. 3)."""
    A, b = irgen.case_green(512, 800.0, rule="trapezoid", rhs="A1")
    res = O.ir_solve(A, b, O.F16)
    assert res.status != O.CONVERGED


def test_ir_promoted_problem_single_single_double():
    """TW = TF = binary32 with TR = binary64 (Sec. 2.2.2): converges to the promoted solution."""
    n = 256
    A, b = irgen.case_svd(n, 44, kappa=1e4)
    res = O.ir_solve(A, b, O.F32)
    xp = O.reference_solution(A, b)
    kappa = O.cond_inf(A)
    # Thm. carsonh1 / eq. irterm: error <= 4 (N+1) kappa u_r + u_w, with the TW rounding of the result
    bound = 4 * (n + 1) * kappa * 2 ** -53 + 2 ** -24
    assert res.status == O.STAGNATED
    assert O.rel_err_inf(res.sol, xp) <= bound
    assert O.rel_err_inf(res.x, xp) <= 4 * (n + 1) * kappa * 2 ** -53 + 1e-12


def test_ir_edge_cases():
    # empty, 1x1, zero right-hand side, singular
    r = O.ir_solve(np.zeros((0, 0), order="F"), np.zeros(0), O.F32)
    assert r.status == O.CONVERGED and r.x.shape == (0,)
    r = O.ir_solve(np.array([[4.0]], order="F"), np.array([2.0]), O.F32)
    assert r.status == O.CONVERGED and r.x[0] == 0.5
    A, _ = irgen.case_gaussian(10, 1)
    r = O.ir_solve(A, np.zeros(10), O.F32)
    assert r.status == O.CONVERGED and not np.any(r.x)
    S = np.asfortranarray(np.ones((4, 4)))
    r = O.ir_solve(S, np.ones(4), O.F32)
    assert r.status == O.FAILED and r.info == 2


def test_reference_solution_exact_small():
    A, b = irgen.case_random(6, 77)
    xr = O.reference_solution(A, b)
    xe = [float(v) for v in _exact_solve(A, b)]
    assert max(abs(a - e) / abs(e) for a, e in zip(xr, xe)) <= 2 ** -52


def test_lu_column_scaling_is_lapack_reciprocal():
    """getf2 scales the pivot column by fl(1/a_kk) (binary32: fl32(a * fl32(1/a_kk))),
    and divides only when |a_kk| is below the smallest normal number."""
    # pivot 7, entry 3: 3 * fl(1/7) = 0.42857146 while 3 / 7 = 0.42857143 in binary32
    LUd, _, _ = O.getrf_tf(np.asfortranarray(np.array([[7.0, 0.0], [3.0, 1.0]], dtype=np.float32)), O.F32)
    assert LUd[1, 0] == np.float32(0.42857146)          # 3 * fl(1/7); 3 / 7 would give 0.42857143
    assert LUd[1, 0] != np.float32(np.float32(3.0) / np.float32(7.0))
    LU64, _, _ = O.getrf_f64(np.asfortranarray(np.array([[7.0, 0.0], [3.0, 1.0]])))
    assert LU64[1, 0] == 3.0 * (1.0 / 7.0)
    tiny = np.float32(1e-39)     # subnormal pivot: plain division
    B = np.asfortranarray(np.array([[tiny, 0.0], [np.float32(5e-40), 1.0]], dtype=np.float32))
    LUb, _, _ = O.getrf_tf(B, O.F32)
    assert LUb[1, 0] == np.float32(np.float32(5e-40) / tiny)


@pytest.mark.parametrize("a,b", [(3.0, 1.0), (-177.78664, 1.0), (7.0, 2.0), (0.1, 0.3)])
def test_scalar_promoted_problem_stops_at_exact_solution(a, b):
    """n = 1, TW = TF = binary32, TR = binary64 (the promoted problem, Sec. 2.2.2).

    The iterate approaches b/a geometrically, so the residual eventually
    vanishes exactly (fl(a x) = b) before eq. (wilkterm) ever fires; IR must
    stop there as converged, with the binary32 solution fl32(b/a), instead of
    dividing by ||r|| = 0 in the next scaled solve (eq. vdlow)."""
    A = np.array([[a]], dtype=np.float32, order="F")
    bb = np.array([b], dtype=np.float32)
    res = O.ir_solve(A, bb, O.F32, term=O.Term(litmax=30))
    assert res.status == O.CONVERGED
    assert res.rhist[-1] == 0.0
    assert np.all(np.isfinite(res.x))
    exact = np.float64(bb[0]) / np.float64(A[0, 0])
    assert res.sol[0] == np.float32(exact)
    assert abs(res.x[0] - exact) <= 2 * np.spacing(abs(exact))


# ---------------------------------------------------------------------------
# backward-error termination (Sec. 5.1.1, eq. term) and ||A||_1
# ---------------------------------------------------------------------------

def test_norm1_is_the_column_sum_norm():
    # nonsymmetric: ||A||_1 (columns) = 9 differs from ||A||_inf (rows) = 7, so a
    # transposed operand fails
    A = np.asfortranarray(np.array([[1.0, -4.0, 0.0], [2.0, 0.0, 3.0], [0.0, 5.0, -1.0]]))
    assert O.norm1(A) == 9.0
    assert O.norm1(A.astype(np.float32)) == 9.0
    assert O.norm1(np.zeros((0, 0))) == 0.0


def test_backward_error_test_replaces_the_residual_test():
    t = O.Term(mode=1)
    eps = 2.0 ** -52
    # ||r|| = 1e-14: far above eps ||b|| (residterm fails) but below eps (||b|| + ||A|| ||x||)
    rh = [1.0, 1e-3, 1e-14]
    assert O.term_decide(rh, [1, 1], 1.0, eps, O.Term(), False) is None
    assert O.term_decide(rh, [1, 1], 1.0, eps, t, False, anorm=100.0, xnorm=1000.0) == O.CONVERGED
    assert O.term_decide(rh, [1, 1], 1.0, eps, t, False, anorm=1.0, xnorm=1.0) is None
    # C_e scales the bound
    assert O.term_decide(rh, [1, 1], 1.0, eps, O.Term(mode=1, Ce=100.0), False, anorm=1.0, xnorm=1.0) \
        == O.CONVERGED
    # TR wider than TW: only the correction test stops the loop, whatever the mode
    assert O.term_decide(rh, [1.0, 0.9], 1.0, 2.0 ** -23, t, True, anorm=1e9, xnorm=1e9) == O.STAGNATED


def test_ir_backward_error_termination_on_ill_conditioned_system():
    """I - 799 G at N = 512 (the system of Sec. 5.1.3): the residual floor is far
    above eps ||b||, so eq. (residterm) never holds and the loop ends on
    stagnation; ||A|| ||x|| ~ 5e4 makes eq. (term) hold at that floor, one
    step earlier and with the same iterate."""
    A = np.asfortranarray(np.eye(512) - 799.0 * irgen.gmat_trapezoid(512))
    b = np.ones(512)
    r0 = O.ir_solve(A, b, O.F32)
    r1 = O.ir_solve(A, b, O.F32, O.Term(mode=1))
    assert r0.status == O.STAGNATED and r1.status == O.CONVERGED
    assert r1.iters == r0.iters - 1
    assert r1.rhist == r0.rhist[:-1]
    assert r1.rhist[-1] <= 2.0 ** -52 * (1.0 + O.norm1(A) * np.max(np.abs(r1.x)))


def test_oracle_is_bitwise_independent_of_the_thread_count():
    """The oracle's parallel loops split only independent work (rows of a
    rank-1 update, rows of a residual), so its results do not depend on the
    number of OpenMP threads: one thread reproduces them bit for bit."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import sys; sys.path.insert(0, %r); import numpy as np, irgen, oracle as O\n"
        "A, b = irgen.case_random(300, 77)\n"
        "LU, ipiv, _ = O.getrf_tf(O.cast(A, O.TF32), O.TF32, 64)\n"
        "LU64, ipiv64, _ = O.getrf_f64(A)\n"
        "r = O.residual(A, b, np.linspace(-1, 1, 300))\n"
        "sys.stdout.buffer.write(LU.tobytes() + ipiv.tobytes() + LU64.tobytes() + ipiv64.tobytes() + r.tobytes())\n"
    ) % root
    outs = []
    for threads in ("1", "4"):
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, timeout=300)
        assert p.returncode == 0, p.stderr.decode()[-2000:]
        outs.append(p.stdout)
    assert len(outs[0]) > 0 and outs[0] == outs[1]
