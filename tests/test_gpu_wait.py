"""The bounded device waits give up, report IR_ETIMEOUT and leave the context usable.

Every spin-wait of the CUDA library is bounded (2 s): after the limit the
kernel raises a flag in device memory, the host reads it and the call returns
IR_ETIMEOUT.  ir_check_wait_timeout runs the correction solves' wait on a value
of the factorization's workspace that no solve writes, with a short limit, so
the wait must run out; nothing hangs and no GPU fault is involved (the wait
ends by itself).  The next solve on the same factorization and context must be
as correct as before.
"""
import time

import numpy as np
import pytest
import torch

import irgen
import oracle as O
from gpu_util import dev_colmajor, dev_vec
from paper_2311_14616_gb300 import ir

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,tf", [(300, "f32"), (5000, "f16")])
def test_bounded_wait_gives_up_then_solve_is_correct(ctx, n, tf):
    A, b = irgen.case_gaussian(n, 6100 + n)
    f = ctx.factor(dev_colmajor(A), tf=tf)
    x0, rep0 = f.solve(dev_vec(b))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    code = f.check_wait_timeout(0.02)
    dt = time.perf_counter() - t0
    assert code == 6, ir.ERRORS.get(code, code)          # IR_ETIMEOUT
    assert dt < 1.5, dt                                  # it gave up at its own limit, not at 2 s
    assert "gave up" in ir.lib().ir_last_error().decode()
    # the same factorization solves again, bit for bit as before the probe
    x1, rep1 = f.solve(dev_vec(b))
    assert rep1.status == rep0.status and rep1.rhist == rep0.rhist
    assert torch.equal(x0, x1)
    xr = O.reference_solution(A, b)
    assert O.rel_err_inf(x1.cpu().numpy(), xr) <= 1e-12
    # and a new factorization on the same context works
    g = ctx.factor(dev_colmajor(A), tf=tf)
    x2, rep2 = g.solve(dev_vec(b))
    assert torch.equal(x2, x1)


def test_bounded_wait_limit_is_checked(ctx):
    A, _ = irgen.case_gaussian(64, 1)
    f = ctx.factor(dev_colmajor(A), tf="f32")
    assert f.check_wait_timeout(0.0) == 1                # IR_EINVAL
    assert f.check_wait_timeout(2.5) == 1                # above the library's own limit
