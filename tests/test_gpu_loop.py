"""The refinement loop of ir_solve runs on the device: all litmax corrections
are enqueued at once and a one-thread kernel applies the termination test of
Sec. 5.1 after every residual, after which the remaining kernels return at
once.  These tests check that the device loop stops where the test says, that
the skipped iterations change nothing, and that its decisions are those of the
oracle's loop on the same histories."""
import numpy as np
import pytest
import torch

import irgen
import oracle as O
from gpu_util import dev_colmajor, dev_vec
from paper_2311_14616_gb300 import ir

pytestmark = pytest.mark.gpu

STATUS = {"converged": O.CONVERGED, "stagnated": O.STAGNATED, "maxit": O.MAXIT, "diverged": O.DIVERGED}


@pytest.fixture(scope="module")
def system(ctx):
    A, b = irgen.case_gaussian(700, 11)
    f = ctx.factor(dev_colmajor(A), tf="f16")
    return A, b, f


def test_litmax_cuts_the_loop(system):
    """litmax = 2 stops after two corrections; the histories up to there are the
    full run's, bit for bit (the same kernels ran on the same data)."""
    A, b, f = system
    xf, rf = f.solve(dev_vec(b))
    assert rf.iters > 2
    x2, r2 = f.solve(dev_vec(b), term=ir.default_term(litmax=2))
    assert r2.iters == 2 and r2.status == "maxit"
    assert r2.rhist == rf.rhist[:3] and r2.dhist == rf.dhist[:2]
    assert not torch.equal(x2, xf)


def test_enqueued_iterations_past_the_decision_change_nothing(system):
    """With litmax = 31 (the most the report holds) the loop still stops at the
    same step with the same iterate: the kernels after the decision do no work."""
    A, b, f = system
    xf, rf = f.solve(dev_vec(b))
    xl, rl = f.solve(dev_vec(b), term=ir.default_term(litmax=ir.MAX_HIST - 1))
    assert rl.iters == rf.iters and rl.status == rf.status and rl.rhist == rf.rhist
    assert torch.equal(xl, xf)


def test_decisions_are_the_oracles_on_the_same_histories(system):
    """The device test, replayed by the oracle's termination rule on the
    device's own histories, decides the same status at the same step."""
    A, b, f = system
    _, r = f.solve(dev_vec(b))
    t = O.Term()
    eps = 2.0 ** -53
    for k in range(1, r.iters + 1):
        st = O.term_decide(r.rhist[: k + 1], r.dhist[:k], r.rhist[0], eps, t, tr_wider=False)
        if k < r.iters:
            assert st is None, k
        else:
            assert st == STATUS[r.status]


def test_nonfinite_rhs_then_normal_solve(system):
    """A non-finite b ends the solve before any correction and leaves x
    untouched; the next solve on the same factorization is unaffected."""
    A, b, f = system
    xf, rf = f.solve(dev_vec(b))
    bad = b.copy()
    bad[3] = np.nan
    x = torch.full((700,), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(ir.IRError) as e:
        f.solve(dev_vec(bad), x)
    assert e.value.code == 5
    assert torch.all(x == 7.0)
    x2, r2 = f.solve(dev_vec(b))
    assert torch.equal(x2, xf) and r2.iters == rf.iters
