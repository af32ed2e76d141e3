"""Parity of the CUDA factorization (cast + blocked LU) with the oracle."""
import numpy as np
import pytest

import irgen
import oracle as O
from gpu_util import dev_colmajor

pytestmark = pytest.mark.gpu

NB = 64   # outer block of the CUDA factorization (the oracle's nb for TF != binary32)


def _matrix(kind, n, seed):
    if kind == "random":
        return irgen.case_random(n, seed)[0]          # genuine row interchanges
    if kind == "gauss":
        return irgen.case_gaussian(n, seed)[0]
    if kind == "green800":
        return irgen.case_green(n, 800.0)[0]
    raise ValueError(kind)


@pytest.mark.parametrize("n", [1, 2, 3, 17, 63, 64, 65, 127, 128, 129, 200, 257, 300, 513])
@pytest.mark.parametrize("kind", ["random", "green800"])
def test_lu_f32_bitexact(ctx, n, kind):
    """TF = binary32: pivots and factors are bitwise those of the unblocked oracle LU."""
    A = _matrix(kind, n, 1000 + n)
    f = ctx.factor(dev_colmajor(A), tf="f32")
    LU, piv = f.factors(), f.pivots()
    LUo, pivo, info = O.getrf_tf(O.cast(A, O.F32), O.F32)
    assert info == 0 and f.info() == (0, False)
    assert np.array_equal(piv, pivo)
    assert np.array_equal(LU.view(np.uint32), LUo.view(np.uint32))


@pytest.mark.parametrize("n", [5, 40, 64])
@pytest.mark.parametrize("tf", [O.TF32, O.BF16, O.F16])
def test_cast_and_panel_bitexact_single_block(ctx, n, tf):
    """n <= 64: one panel, no tensor-core update -- the rounded copy (incl. the binary16
    scaling) and the binary32 panel are bitwise the oracle's."""
    A = _matrix("random", n, 2000 + n)
    f = ctx.factor(dev_colmajor(A), tf=O.DTYPE_NAMES[tf])
    s = O.fp16_scale(A) if tf == O.F16 else 1.0
    LUo, pivo, _ = O.getrf_tf(O.cast(A, tf, s), tf, nb=NB)
    assert np.array_equal(f.pivots(), pivo)
    assert np.array_equal(f.factors().view(np.uint32), LUo.view(np.uint32))


def _column_magnitudes(LU, k):
    """|a_ik| of the candidates of step k (rows >= k, final row order), rebuilt from
    the factors: a_kk = u_kk and a_ik = l_ik u_kk below the diagonal."""
    col = LU[k:, k].astype(np.float64) * LU[k, k]
    col[0] = LU[k, k]
    return np.abs(col)


@pytest.mark.parametrize("n", [65, 130, 257, 520])
@pytest.mark.parametrize("tf", [O.TF32, O.BF16, O.F16])
@pytest.mark.parametrize("kind", ["random", "gauss"])
def test_lu_tensor_core_parity(ctx, n, tf, kind):
    """Tensor-core trailing update.  The GPU's pivots are valid partial pivots
    (|l_ik| <= 1); with them replayed in the oracle, every step where the GPU took
    another row than the oracle's maximum is a near tie: the oracle's top-two gap is
    within the measured GPU/oracle discrepancy of that column.  The factors agree to
    the TF rounding level and satisfy the TF backward-error bound."""
    A = _matrix(kind, n, 3000 + n)
    f = ctx.factor(dev_colmajor(A), tf=O.DTYPE_NAMES[tf])
    LU, piv = f.factors(), f.pivots()
    assert f.info() == (0, False)
    assert np.all(np.abs(np.tril(LU, -1)) <= 1.0)
    s = O.fp16_scale(A) if tf == O.F16 else 1.0
    AF = O.cast(A, tf, s)
    LUo, pivo, info, gap = O.getrf_tf(AF, tf, nb=NB, force_piv=piv, want_gap=True)
    ks = np.nonzero(gap[:, 2] < gap[:, 0])[0]
    for k in ks:
        delta = np.max(np.abs(_column_magnitudes(LU, k) - _column_magnitudes(LUo, k)))
        assert gap[k, 0] - gap[k, 2] <= 2 * delta + 4 * 2.0 ** -24 * gap[k, 0], (k, gap[k], delta)
    # first block column: bitwise (no tensor-core update has touched it)
    assert np.array_equal(LU[:, :NB].view(np.uint32), LUo[:, :NB].view(np.uint32))
    u = O.UNIT_ROUNDOFF[tf]
    if kind == "gauss":
        # well-conditioned Schur complements: disagreements are rare and the whole
        # factorization is normwise close at the TF rounding level.  (For the
        # unshifted random matrices the late Schur complements are ill-conditioned
        # and amplify the accumulation-order differences; there the backward-error
        # bound below is the check.)
        assert len(ks) <= max(2, n // 50)
        rel = np.max(np.abs(LU.astype(np.float64) - LUo)) / np.max(np.abs(LUo))
        assert rel <= 64 * u, rel
    # and the GPU factors satisfy the backward-error bound of the TF factorization
    P = O.perm_from_ipiv(piv)
    L = np.tril(LU.astype(np.float64), -1) + np.eye(n)
    U = np.triu(LU.astype(np.float64))
    E = AF.astype(np.float64)[P] - L @ U
    assert np.max(np.abs(E).sum(axis=1)) <= 4 * n * u * np.max(np.abs(AF).sum(axis=1))


def test_lu_zero_pivot_reports_info(ctx):
    S = np.asfortranarray(np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0], [1.0, 0.0, 1.0]]))
    f = ctx.factor(dev_colmajor(S), tf="f32")
    assert f.info() == (3, False)


def test_lu_nonfinite_input_is_flagged(ctx):
    A = irgen.case_gaussian(70, 5)[0]
    A[3, 9] = np.nan
    f = ctx.factor(dev_colmajor(A), tf="tf32")
    assert f.info()[1] is True
