"""Factors kept in TF (store_tf): binary16 / bfloat16 factors in 2 bytes.

After the factorization every entry of L and U is rounded to TF once (the
paper keeps its factorization copy in TF, Sec. 1 and 2.5) and the correction
solves read the 2-byte copy, promoting each entry exactly.  Checked against the
oracle's ir_solve(store_tf=True), which rounds its factors the same way: where
the oracle's result meets the parity bar, the same status and x within the bar
of the oracle's and x_ref; the stored factors are TF numbers and satisfy the
TF backward-error bound; a raw correction solve on them agrees with the
oracle's substitution on the same (stored) factors; an entry that overflows TF
is reported.
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
    yield "gauss_N700_f16", lambda: irgen.case_gaussian(700, 29), O.F16
    yield "gauss_N700_bf16", lambda: irgen.case_gaussian(700, 29), O.BF16
    yield "green_a100_N700_f16", lambda: irgen.case_green(700, 100.0), O.F16
    yield "green_a1_N129_bf16", lambda: irgen.case_green(129, 1.0), O.BF16
    yield "gauss_N1_f16", lambda: irgen.case_gaussian(1, 4), O.F16
    yield "gauss_N5000_f16", lambda: irgen.case_gaussian(5000, 31), O.F16


@pytest.mark.parametrize("name,make,tf", list(_cases()), ids=[c[0] for c in _cases()])
def test_store_tf_matches_oracle(ctx, name, make, tf):
    A, b = make()
    n = A.shape[0]
    f = ctx.factor(dev_colmajor(A), tf=O.DTYPE_NAMES[tf], store_tf=True)
    x, rep = f.solve(dev_vec(b), term=ir.default_term(litmax=20))
    x = x.cpu().numpy()
    ref = O.ir_solve(A, b, tf, O.Term(litmax=20), nb=64, store_tf=True)
    xr = O.reference_solution(A, b)
    tol = P.bar(O.cond_inf(A) if n <= 2000 else float(np.linalg.cond(A, np.inf)))
    assert O.rel_err_inf(ref.x, xr) <= tol          # the oracle meets the bar: compare
    assert rep.status == O.STATUS_NAMES[ref.status], (rep.rhist, ref.rhist)
    assert abs(rep.iters - ref.iters) <= 2
    assert O.rel_err_inf(x, ref.x) <= tol
    assert O.rel_err_inf(x, xr) <= tol
    # the stored factors are TF numbers and a TF factorization of the rounded copy
    LU = f.factors()
    assert np.array_equal(O.round_tf(LU, tf).reshape(LU.shape), LU)
    s = O.fp16_scale(A) if tf == O.F16 else 1.0
    AF = O.cast(A, tf, s)
    u = O.UNIT_ROUNDOFF[tf]
    L = np.tril(LU.astype(np.float64), -1) + np.eye(n)
    U = np.triu(LU.astype(np.float64))
    E = AF.astype(np.float64)[O.perm_from_ipiv(f.pivots())] - L @ U
    assert np.max(np.abs(E).sum(axis=1)) <= 4 * n * u * np.max(np.abs(AF).sum(axis=1))


@pytest.mark.parametrize("n", [300, 4500])
def test_store_tf_raw_solve_on_stored_factors(ctx, n):
    """d = U^{-1} L^{-1} P v read from the 2-byte copy, against the oracle's binary32
    substitution on the same stored factors (both within the conditioning bound)."""
    A, _ = irgen.case_random(n, 70 + n)
    f = ctx.factor(dev_colmajor(A), tf="bf16", store_tf=True)
    LU, piv = f.factors(), f.pivots()
    v = np.random.Generator(np.random.PCG64(n)).standard_normal(n).astype(np.float32)
    d = f.lu_solve(dev_vec(v)).cpu().numpy()
    do = O.getrs_f32(LU, piv, v)
    L = np.tril(LU.astype(np.float64), -1) + np.eye(n)
    U = np.triu(LU.astype(np.float64))
    dx = np.linalg.solve(U, np.linalg.solve(L, O.apply_pivots(piv, v.astype(np.float64))))
    cond = np.linalg.cond(L, np.inf) * np.linalg.cond(U, np.inf)
    tol = 4 * n * 2.0 ** -24 * cond * np.max(np.abs(dx))
    assert np.max(np.abs(d - dx)) <= tol
    assert np.max(np.abs(do - dx)) <= tol


def test_store_tf_overflow_is_reported(ctx):
    """Wilkinson's growth matrix (1 on the diagonal and in the last column, -1
    below the diagonal): partial pivoting takes no interchange and the last
    column doubles at every step, u_nn = 2^(n-1).  Scaled for binary16 (the
    largest entry on 2^10) and n = 8, u_nn = 2^17 exceeds the binary16 range:
    stored in TF the factorization is non-finite; kept in binary32 it is not."""
    n = 8
    A = np.eye(n) - np.tril(np.ones((n, n)), -1)
    A[:, -1] = 1.0
    A = np.asfortranarray(A)
    f = ctx.factor(dev_colmajor(A), tf="f16", store_tf=True)
    assert f.info() == (0, True)
    with pytest.raises(ir.IRError) as e:
        f.solve(dev_vec(np.ones(n)))
    assert e.value.code == 5                     # IR_ENONFINITE
    g = ctx.factor(dev_colmajor(A), tf="f16")
    assert g.info() == (0, False)
    assert g.factors()[n - 1, n - 1] == 2.0 ** 17


def test_store_tf_rejects_other_factorization_types(ctx):
    A = dev_colmajor(np.eye(4))
    for tf in ("f32", "tf32"):
        with pytest.raises(ir.IRError, match="IR_EINVAL"):
            ctx.factor(A, tf=tf, store_tf=True)
