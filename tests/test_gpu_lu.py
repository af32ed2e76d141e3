"""Parity of the CUDA factorization (cast + blocked LU) with the oracle."""
import numpy as np
import pytest

import irgen
import oracle as O
import parity as P
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


@pytest.mark.parametrize("n", [65, 130, 257, 520, 1100])
@pytest.mark.parametrize("tf", [O.TF32, O.BF16, O.F16])
@pytest.mark.parametrize("kind", ["random", "gauss"])
def test_lu_tensor_core_parity(ctx, n, tf, kind):
    """Tensor-core trailing update.  The GPU's pivots are valid partial pivots
    (|l_ik| <= 1).  The oracle replays them (pivot-replay mode); wherever the GPU
    took another row than the oracle's maximum, the oracle's top candidate and the
    GPU's row must lie within the a-priori envelope of the step (binary32
    accumulation and TF rounding flips, sized by the sums column k received,
    from the oracle's factors; see parity.pivot_envelope) -- a near tie.  Away
    from near ties every pivot is the oracle's.  On the shifted Gaussian
    matrices no step is a near tie, so every pivot must be the oracle's; on the
    unshifted random matrices the Schur complements cancel heavily (sums of
    |l||u| far above the candidates), most steps fall inside the envelope and
    the backward-error bound is the real check.  The factors agree to the TF
    rounding level (shifted Gaussian) and satisfy the TF backward-error bound."""
    A = _matrix(kind, n, 3000 + n)
    f = ctx.factor(dev_colmajor(A), tf=O.DTYPE_NAMES[tf])
    LU, piv = f.factors(), f.pivots()
    assert f.info() == (0, False)
    assert np.all(np.abs(np.tril(LU, -1)) <= 1.0)
    s = O.fp16_scale(A) if tf == O.F16 else 1.0
    AF = O.cast(A, tf, s)
    LUo, pivo, info, gap = O.getrf_tf(AF, tf, nb=NB, force_piv=piv, want_gap=True)
    env = P.pivot_envelope(AF, LUo, pivo, NB, tf)
    deviated = np.nonzero(gap[:, 2] < gap[:, 0])[0]
    for k in deviated:
        assert gap[k, 0] - gap[k, 2] <= 2 * env[k], (k, gap[k], env[k])
    # first block column: bitwise (no tensor-core update has touched it)
    assert np.array_equal(LU[:, :NB].view(np.uint32), LUo[:, :NB].view(np.uint32))
    u = O.UNIT_ROUNDOFF[tf]
    if kind == "gauss":
        # well-conditioned Schur complements: near ties are rare and the whole
        # factorization is normwise close at the TF rounding level.  (For the
        # unshifted random matrices the late Schur complements are ill-conditioned
        # and amplify the accumulation-order differences; there the backward-error
        # bound below is the check.)
        assert len(deviated) == 0
        rel = np.max(np.abs(LU.astype(np.float64) - LUo)) / np.max(np.abs(LUo))
        assert rel <= 64 * u, rel
    # and the GPU factors satisfy the backward-error bound of the TF factorization
    Pm = O.perm_from_ipiv(piv)
    L = np.tril(LU.astype(np.float64), -1) + np.eye(n)
    U = np.triu(LU.astype(np.float64))
    E = AF.astype(np.float64)[Pm] - L @ U
    assert np.max(np.abs(E).sum(axis=1)) <= 4 * n * u * np.max(np.abs(AF).sum(axis=1))


@pytest.mark.parametrize("group", [1, 2, 4, 16])
@pytest.mark.parametrize("tf", [O.F16, O.TF32])
def test_lu_tensor_core_group_sizes(ctx, group, tf):
    """The far trailing columns receive a group of block steps' products at once
    (K = 64 group on the tensor cores); the rows inside the group still get them
    block by block.  For every group size the pivots are the oracle's away from
    near ties (a-priori envelope), the factors are normwise within the TF
    rounding level of the oracle's and satisfy the backward-error bound."""
    n = 1500
    A = _matrix("gauss", n, 3100 + group)
    f = ctx.factor(dev_colmajor(A), tf=O.DTYPE_NAMES[tf], group=group)
    assert f.schedule()[2] == group
    LU, piv = f.factors(), f.pivots()
    assert f.info() == (0, False)
    s = O.fp16_scale(A) if tf == O.F16 else 1.0
    AF = O.cast(A, tf, s)
    LUo, pivo, info, gap = O.getrf_tf(AF, tf, nb=NB, force_piv=piv, want_gap=True)
    env = P.pivot_envelope(AF, LUo, pivo, NB, tf)
    deviated = np.nonzero(gap[:, 2] < gap[:, 0])[0]
    for k in deviated:
        assert gap[k, 0] - gap[k, 2] <= 2 * env[k], (k, gap[k], env[k])
    assert len(deviated) <= n // 50
    u = O.UNIT_ROUNDOFF[tf]
    rel = np.max(np.abs(LU.astype(np.float64) - LUo)) / np.max(np.abs(LUo))
    assert rel <= 64 * u, rel
    Pm = O.perm_from_ipiv(piv)
    L = np.tril(LU.astype(np.float64), -1) + np.eye(n)
    U = np.triu(LU.astype(np.float64))
    E = AF.astype(np.float64)[Pm] - L @ U
    assert np.max(np.abs(E).sum(axis=1)) <= 4 * n * u * np.max(np.abs(AF).sum(axis=1))


def test_lu_f16_pivots_full_size_c3(ctx):
    """The N = 8192 shifted Gaussian system with scaled binary16 factors (the
    benchmark's workload): pivots in replay against the oracle's emulated-TF
    factorization with the a-priori near-tie envelope, and factors normwise
    within the TF rounding level of the oracle's."""
    n = 8192
    A, _ = irgen.case_gaussian(n, 1002)
    f = ctx.factor(dev_colmajor(A), tf="f16")
    LU, piv = f.factors(), f.pivots()
    s = O.fp16_scale(A)
    AF = O.cast(A, O.F16, s)
    LUo, pivo, info, gap = O.getrf_tf(AF, O.F16, nb=NB, force_piv=piv, want_gap=True)
    assert info == 0
    env = P.pivot_envelope(AF, LUo, pivo, NB, O.F16)
    deviated = np.nonzero(gap[:, 2] < gap[:, 0])[0]
    for k in deviated:
        assert gap[k, 0] - gap[k, 2] <= 2 * env[k], (k, gap[k], env[k])
    assert len(deviated) <= n // 50
    rel = np.max(np.abs(LU.astype(np.float64) - LUo)) / np.max(np.abs(LUo))
    assert rel <= 64 * O.UNIT_ROUNDOFF[O.F16], rel


def test_lu_f32_bitexact_full_size_16_cta_panel(ctx):
    """N = 8192: the panel runs as a 16-CTA cluster (512 rows per CTA); the binary32
    factors and pivots are still bitwise the unblocked oracle LU's."""
    n = 8192
    A, _ = irgen.case_gaussian(n, 1002)
    f = ctx.factor(dev_colmajor(A), tf="f32")
    LUo, pivo, info = O.getrf_tf(O.cast(A, O.F32), O.F32)
    assert info == 0
    assert np.array_equal(f.pivots(), pivo)
    assert np.array_equal(f.factors().view(np.uint32), LUo.view(np.uint32))


def test_lu_zero_pivot_reports_info(ctx):
    S = np.asfortranarray(np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0], [1.0, 0.0, 1.0]]))
    f = ctx.factor(dev_colmajor(S), tf="f32")
    assert f.info() == (3, False)


def test_lu_nonfinite_input_is_flagged(ctx):
    A = irgen.case_gaussian(70, 5)[0]
    A[3, 9] = np.nan
    f = ctx.factor(dev_colmajor(A), tf="tf32")
    assert f.info()[1] is True
