"""Systems taller than one panel cluster holds (n > 8192): the first panels
run as one cooperative launch whose CTAs exchange each column's pivot
candidates through global memory.  The binary32 factors stay bitwise the
unblocked oracle LU's; refinement with binary16 factors meets the oracle's IR;
at n = 20000 (40-CTA panels) the refined solution has a backward error at the
binary64 level (a property that holds at any size; the oracle's LU would take
minutes there)."""
import numpy as np
import pytest

import irgen
import oracle as O
import parity as P
from gpu_util import dev_colmajor, dev_vec

pytestmark = pytest.mark.gpu


def test_lu_f32_bitexact_tall_panels(ctx):
    """n = 8704: panels 0..7 have more than 8192 rows (17 CTAs, grid exchange),
    the rest run as clusters; pivots and binary32 factors bitwise the oracle's."""
    n = 8704
    A, _ = irgen.case_gaussian(n, 1101)
    f = ctx.factor(dev_colmajor(A), tf="f32")
    LUo, pivo, info = O.getrf_tf(O.cast(A, O.F32), O.F32)
    assert info == 0
    assert np.array_equal(f.pivots(), pivo)
    assert np.array_equal(f.factors().view(np.uint32), LUo.view(np.uint32))


def test_tall_f16_ir_matches_oracle(ctx):
    """n = 8704, binary16 factors: the oracle's IR meets the parity bar, and the
    GPU's status, step count (within two) and x agree with it."""
    n = 8704
    A, b = irgen.case_gaussian(n, 1102)
    xr = O.reference_solution(A, b)
    kappa = float(np.linalg.cond(A, np.inf))
    f = ctx.factor(dev_colmajor(A), tf="f16")
    x, rep = f.solve(dev_vec(b))
    x = x.cpu().numpy()
    ref = O.ir_solve(A, b, O.F16, nb=64)
    tol = P.bar(kappa)
    assert O.rel_err_inf(ref.x, xr) <= tol
    assert rep.status == O.STATUS_NAMES[ref.status]
    assert abs(rep.iters - ref.iters) <= 2
    assert O.rel_err_inf(x, ref.x) <= tol
    assert O.rel_err_inf(x, xr) <= tol


def test_n20000_f16_backward_error(ctx):
    """n = 20000 (40-CTA cooperative panels): IR with binary16 factors converges
    to a normwise backward error within 3 gamma_n u_64, measured with a binary64
    residual (which adds at most gamma_n u_64 of its own: bound 4 gamma_n)."""
    n = 20000
    A, b = irgen.case_gaussian(n, 1103)
    f = ctx.factor(dev_colmajor(A), tf="f16")
    x, rep = f.solve(dev_vec(b))
    assert rep.status in ("converged", "stagnated")
    x = x.cpu().numpy()
    r = O.residual(A, b, x)
    normA = np.max(np.abs(A).sum(axis=1))
    eta = np.max(np.abs(r)) / (normA * np.max(np.abs(x)) + np.max(np.abs(b)))
    u = 2.0 ** -53
    assert eta <= 4 * n * u / (1 - n * u), eta
