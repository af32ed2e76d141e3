"""A borrowed A with a leading dimension larger than n (a column-major view
into a wider buffer): the cast, the binary16 scale's maximum (its column-wise
path), the factorization and the refinement's residuals read it through lda
and give bitwise what the contiguous copy gives."""
import numpy as np
import pytest
import torch

import irgen
from gpu_util import dev_colmajor, dev_vec

pytestmark = pytest.mark.gpu


def _padded(A: np.ndarray, extra: int) -> torch.Tensor:
    n = A.shape[0]
    lda = n + extra
    buf = torch.full((lda * n,), float("nan"), dtype=torch.float64, device="cuda")   # padding never read
    V = buf.as_strided((n, n), (1, lda))
    V.copy_(torch.from_numpy(np.ascontiguousarray(A)).cuda())
    return V


@pytest.mark.parametrize("tf", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("n,extra", [(300, 7), (1000, 24)])
def test_padded_lda_is_bitwise_the_contiguous_copy(ctx, tf, n, extra):
    A, b = irgen.case_gaussian(n, 1200 + n)
    Ap = _padded(A, extra)
    assert Ap.stride() == (1, n + extra)
    fp = ctx.factor(Ap, tf=tf)
    fc = ctx.factor(dev_colmajor(A), tf=tf)
    assert np.array_equal(fp.pivots(), fc.pivots())
    assert np.array_equal(fp.factors().view(np.uint32), fc.factors().view(np.uint32))
    xp, rp = fp.solve(dev_vec(b))
    xc, rc = fc.solve(dev_vec(b))
    assert rp.status == rc.status and rp.iters == rc.iters and rp.rhist == rc.rhist
    assert rp.scale == rc.scale
    assert torch.equal(xp, xc)
