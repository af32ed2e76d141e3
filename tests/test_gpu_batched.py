"""Batched driver (one persistent launch over many uneven systems) against the oracle.

* TF = binary32: every step of the batch kernel takes the oracle's rounding
  decisions (fmaf chains in the unblocked LU's order, LAPACK getf2 reciprocal
  scaling, the reference trsv order of the solves, the residual's fma chain),
  so iterates, statuses, iteration counts and residual norms are bitwise the
  oracle's ir_solve results, for TW = binary64 and for TW = binary32 (where
  TR is wider and eq. (wilkterm) decides).
* TF = binary16 / bfloat16 / TF32: the trailing update sums in binary32 where
  the oracle sums exactly, so the factors differ by rounding.  Each member is
  placed by the oracle's own run (parity.classify): away from the convergence
  boundary of its TF the status must be the oracle's, and where the oracle's
  x meets the parity bar against x_ref the GPU's x must meet it against both
  x_ref and the oracle's x; the tests assert how many members were compared.
  Every reported residual norm must equal, bitwise, the oracle's binary64
  residual of the returned iterate.
* The full-size workload (2000 systems, N uniform in [32, 512]) is checked on
  a sample of systems against the oracle and on all systems by the residual
  property; runs replayed from a CUDA graph equal direct runs.
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

STATUS = {O.CONVERGED: "converged", O.STAGNATED: "stagnated", O.MAXIT: "maxit",
          O.DIVERGED: "diverged", O.FAILED: "failed"}
TF = {"f32": O.F32, "tf32": O.TF32, "bf16": O.BF16, "f16": O.F16}
EDGE_SIZES = [0, 1, 2, 3, 31, 63, 64, 65, 100, 127, 128, 129, 255, 300, 447, 511, 512]


def _upload(As, bs, dtype=np.float64):
    return ([dev_colmajor(np.asfortranarray(A.astype(dtype))) for A in As],
            [dev_vec(b.astype(dtype)) for b in bs])


def _run(ctx, As, bs, tf, dtype=np.float64, term=None):
    Ad, bd = _upload(As, bs, dtype)
    plan = ctx.batch(Ad, bd, tf=tf, term=term)
    plan.run()
    torch.cuda.synchronize()
    res = plan.results()
    xs = [x.cpu().numpy() for x in plan.xs]
    plan.destroy()
    return xs, res


# litmax of the low-precision comparisons: bfloat16 factors reach the rounding floor
# after 8 - 12 steps, so with the default 10 the stop between eq. (stag) and
# litmax would be decided by floor noise; 20 leaves every converging run room to
# end by eq. (stag) (parity.status_must_match)
LITMAX_LP = 20


def _classify_member(A, b, x, r, tf, litmax=LITMAX_LP):
    """Compare one batch member with the oracle's IR on the same system; returns
    the oracle's class and whether x and the status were compared."""
    o = O.ir_solve(A, b, TF[tf], O.Term(litmax=litmax), nb=64)
    xr = O.reference_solution(A, b)
    kappa = O.cond_inf(A)
    tol = P.bar(kappa)
    cls = P.classify(o, O.rel_err_inf(o.x, xr) <= tol)
    st = P.status_must_match(o, cls, litmax)
    if st:
        assert r["status"] == STATUS[o.status], (A.shape[0], cls, r, o.rhist)
    if cls == "conv":
        assert O.rel_err_inf(x, o.x) <= tol, (A.shape[0], O.rel_err_inf(x, o.x), tol)
        assert O.rel_err_inf(x, xr) <= tol, (A.shape[0], O.rel_err_inf(x, xr), tol)
    return cls, st


def _rnorm_of(A, b, x):
    r = O.residual(A, b.astype(np.float64), x.astype(np.float64))
    if not r.size:
        return 0.0
    return float("nan") if np.isnan(r).any() else float(np.max(np.abs(r)))


def _same(a, b):
    return a == b or (np.isnan(a) and np.isnan(b))


@pytest.mark.parametrize("tw", [np.float64, np.float32])
def test_batch_f32_bitwise_equals_oracle(ctx, tw):
    _, As, bs = irgen.case_batch_sizes(EDGE_SIZES, 4100)
    As = [np.asfortranarray(A.astype(tw)) for A in As]
    bs = [b.astype(tw) for b in bs]
    xs, res = _run(ctx, As, bs, "f32", tw)
    for A, b, x, r in zip(As, bs, xs, res):
        n = A.shape[0]
        if n == 0:
            assert r["status"] == "converged" and r["iters"] == 0
            continue
        o = O.ir_solve(A, b, O.F32, nb=64)
        assert r["info"] == o.info == 0
        assert r["status"] == STATUS[o.status], (n, r, o.status)
        assert r["iters"] == len(o.rhist) - 1, n
        assert np.array_equal(x.view(np.uint8), o.sol.view(np.uint8)), n
        assert r["rnorm"] == o.rhist[-1], n


@pytest.mark.parametrize("tf", ["f16", "bf16", "tf32"])
def test_batch_low_precision_vs_oracle(ctx, tf):
    ns = [32, 47, 64, 65, 96, 130, 192, 257, 320, 384, 449, 512]
    alphas, As, bs = irgen.case_batch_sizes(ns, 4200 + len(tf))
    xs, res = _run(ctx, As, bs, tf, term=ir.default_term(litmax=LITMAX_LP))
    compared = status_cmp = 0
    for A, b, x, r, alpha in zip(As, bs, xs, res, alphas):
        n = A.shape[0]
        if tf == "f16":
            assert r["scale"] == 1024.0 / np.max(np.abs(A))
        assert r["status"] != "failed" and not r["nonfinite"]
        # the reported norm is the binary64 residual of the returned iterate, bit for bit
        assert _same(r["rnorm"], _rnorm_of(A, b, x)), n
        if r["status"] == "converged":
            # the residual test itself must hold
            assert r["rnorm"] <= 2.0 ** -52 * np.max(np.abs(b))
        cls, st = _classify_member(A, b, x, r, tf)
        compared += cls == "conv"
        status_cmp += st
    # most members are away from the boundary of their TF: most compare
    assert compared >= 0.8 * len(ns) and status_cmp >= 0.8 * len(ns), (compared, status_cmp)


def test_batch_edge_sizes_low_precision(ctx):
    _, As, bs = irgen.case_batch_sizes(EDGE_SIZES, 4300)
    xs, res = _run(ctx, As, bs, "bf16")
    for A, b, x, r in zip(As, bs, xs, res):
        if A.shape[0] == 0:
            assert r["status"] == "converged" and r["iters"] == 0
            continue
        assert r["status"] != "failed"
        assert _same(r["rnorm"], _rnorm_of(A, b, x))


def test_batch_failures_are_per_system(ctx):
    _, As, bs = irgen.case_batch_sizes([40, 70, 90, 33], 4400)
    As[1] = np.zeros((70, 70), order="F")                 # zero pivot at step 1
    As[2] = As[2].copy(order="F")
    As[2][5, 7] = np.nan                                  # non-finite input
    bs[3] = bs[3].copy()
    bs[3][0] = np.inf
    xs, res = _run(ctx, As, bs, "f16", term=ir.default_term(litmax=LITMAX_LP))
    # the healthy systems are solved as if alone
    for i in (0,):
        assert res[i]["status"] != "failed"
        assert _same(res[i]["rnorm"], _rnorm_of(As[i], bs[i], xs[i]))
        assert _classify_member(As[i], bs[i], xs[i], res[i], "f16") == ("conv", True)
    assert res[1]["status"] == "failed" and res[1]["info"] == 1 and not res[1]["nonfinite"]
    assert res[2]["status"] == "failed" and res[2]["nonfinite"]
    assert res[3]["status"] == "failed" and res[3]["nonfinite"]


def test_batch_rejects_bad_arguments(ctx):
    A = dev_colmajor(np.eye(513))
    b = dev_vec(np.ones(513))
    with pytest.raises(ir.IRError) as e:
        ctx.batch([A], [b], tf="f16")
    assert e.value.code == 7                                # IR_EUNSUPPORTED
    with pytest.raises(ir.IRError) as e:
        ctx.batch([dev_colmajor(np.eye(4))], [dev_vec(np.ones(4))], tf="f64")
    assert e.value.code == 1                                # IR_EINVAL: TF = binary64


def test_empty_batch(ctx):
    plan = ctx.batch([], [], tf="f16")
    plan.run()
    assert plan.results() == []


@pytest.fixture(scope="module")
def full_batch():
    ns, alphas, As, bs = irgen.case_batch(2000, 1005)
    return ns, alphas, As, bs


@pytest.mark.parametrize("tf", ["f16", "bf16"])
def test_full_batch_2000_systems(ctx, full_batch, tf):
    ns, alphas, As, bs = full_batch
    Ad, bd = _upload(As, bs)
    plan = ctx.batch(Ad, bd, tf=tf, term=ir.default_term(litmax=LITMAX_LP))
    plan.run()
    torch.cuda.synchronize()
    res = plan.results()
    xs = [x.cpu().numpy() for x in plan.xs]
    # every system: the reported norm is the binary64 residual of the returned iterate
    for A, b, x, r in zip(As, bs, xs, res):
        assert r["status"] != "failed"
        assert _same(r["rnorm"], _rnorm_of(A, b, x))
        if r["status"] == "converged":
            assert r["rnorm"] <= 2.0 ** -52 * np.max(np.abs(b))
    # the largest errors against a binary64 solve are failures of the method itself:
    # the oracle's IR on the same systems does not converge either
    def _err(A, b, x):
        xr = np.linalg.solve(A, b)
        return np.max(np.abs(x - xr)) / np.max(np.abs(xr))
    err = np.array([_err(A, b, x) if r["status"] != "converged" else 0.0
                    for A, b, x, r in zip(As, bs, xs, res)])
    for i in np.argsort(err)[-3:]:
        if err[i] > 1e-8:
            o = O.ir_solve(As[i], bs[i], TF[tf], O.Term(litmax=LITMAX_LP), nb=64)
            xo = o.sol.astype(np.float64)
            xr = O.reference_solution(As[i], bs[i])
            assert P.classify(o, O.rel_err_inf(xo, xr) <= P.bar(O.cond_inf(As[i]))) != "conv", (i, err[i])
            assert O.rel_err_inf(xo, xr) > 1e-10, (i, err[i])
    # a sample against the oracle's own IR: status wherever the member is away from
    # the convergence boundary, x wherever the oracle's x meets the bar
    g = np.random.Generator(np.random.PCG64(77))
    sample = g.choice(len(ns), size=40, replace=False)
    compared = status_cmp = 0
    for i in sample:
        cls, st = _classify_member(As[i], bs[i], xs[i], res[i], tf)
        compared += cls == "conv"
        status_cmp += st
    # a quarter of these systems have alpha close to a singular mode (kappa up to
    # ~1e5); bfloat16's convergence boundary (kappa u_F ~ 1) cuts into them
    frac = 0.8 if tf == "f16" else 0.7
    assert compared >= frac * len(sample) and status_cmp >= 0.8 * len(sample), (compared, status_cmp)
    # a replay from a CUDA graph gives the same bits
    first = [x.clone() for x in plan.xs]
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            plan.run()
    for x in plan.xs:
        x.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for a, b in zip(first, plan.xs):
        assert torch.equal(a, b)
    assert plan.results() == res
    plan.destroy()


def test_one_shot_entry_point_matches_plan(ctx):
    _, As, bs = irgen.case_batch_sizes([77, 300, 129], 4500)
    Ad, bd = _upload(As, bs)
    xs, res = ctx.solve_batched(Ad, bd, tf="f16")
    xs2, res2 = _run(ctx, As, bs, "f16")
    assert res == res2
    for a, b in zip(xs, xs2):
        assert np.array_equal(a.cpu().numpy(), b)


def test_batch_autotune_picks_a_candidate_and_keeps_parity(ctx):
    """opts.autotune: the plan times the tensor-core crossover on the batch itself;
    the tuned plan's results still meet the oracle bar (the SIMT and tensor-core
    updates round the same operands to TF)."""
    _, As, bs = irgen.case_batch_sizes([48, 130, 200, 257, 384, 512, 96, 300], seed=31)
    plan = ctx.batch([dev_colmajor(A) for A in As], [dev_vec(b) for b in bs], tf="f16", autotune=True,
                     term=ir.default_term(litmax=LITMAX_LP))
    grid, tcm = plan.schedule()
    assert grid >= 1 and tcm in (64, 128, 192, 256, 1 << 20)
    plan.run()
    res = plan.results()
    compared = 0
    for A, b, x, r in zip(As, bs, plan.xs, res):
        cls, _ = _classify_member(A, b, x.cpu().numpy(), r, "f16")
        compared += cls == "conv"
    assert compared >= 0.8 * len(As), compared
    untuned = ctx.batch([dev_colmajor(A) for A in As], [dev_vec(b) for b in bs], tf="f16")
    assert untuned.schedule()[1] == 64


def test_factor_autotune_schedule(ctx):
    A, b, xt = irgen.case_green_sine(2048)
    f = ctx.factor(dev_colmajor(A), tf="f32", autotune=True)
    nb, r, grp = f.schedule()
    assert nb == 64 and r in (8, 12, 16, 24, 32) and grp == 1
    x, rep = f.solve(dev_vec(b))
    assert rep.status in ("converged", "stagnated")
    assert O.rel_err_inf(x.cpu().numpy(), xt) <= O.parity_tol(1.8e5, O.F64)
    # the binary32 factors do not depend on the schedule (bitwise)
    g = ctx.factor(dev_colmajor(A), tf="f32")
    assert g.schedule() == (64, 16, 1)
    np.testing.assert_array_equal(f.factors(), g.factors())
    # a second tuned factorization of the same size reuses the context's choice
    h = ctx.factor(dev_colmajor(A), tf="f32", autotune=True)
    assert h.schedule() == f.schedule()


def test_batch_precision_escalation(ctx):
    """ir_batch_run_escalate: the members whose binary16 IR did not converge are
    solved again with binary32 factors on the device; those results are bitwise
    the oracle's binary32 IR (the batch's binary32 path is the oracle's
    arithmetic), the others are the binary16 run's.  Capturable in a graph."""
    ns = [96, 200, 320, 448, 512, 160, 384, 256, 64, 500, 128, 300]
    alphas, As, bs = irgen.case_batch_sizes(ns, seed=1234)
    # two members near a singular mode (1 - alpha lambda_k ~ 0): binary16 IR fails there
    for i, a in ((2, 88.9), (5, 157.8)):
        n = ns[i]
        As[i] = np.asfortranarray(np.eye(n) - a * irgen.gmat_midpoint(n))
    rtol = 1e-10
    Ad = [dev_colmajor(A) for A in As]
    bd = [dev_vec(b) for b in bs]
    plain = ctx.batch(Ad, bd, tf="f16")
    plain.run()
    first = plain.results()
    plan = ctx.batch(Ad, bd, tf="f16")
    plan.run_escalate("f32", rtol)
    res = plan.results()
    xs = [x.cpu().numpy() for x in plan.xs]
    escalated = [i for i, r in enumerate(first)
                 if not (r["status"] == "converged"
                         or (r["status"] in ("stagnated", "maxit") and r["rnorm"] <= rtol * r["bnorm"]))]
    assert escalated, "the near-singular members should not reach 1e-10 with binary16 factors"
    assert len(escalated) < len(ns)
    for i, r in enumerate(res):
        if i in escalated:
            o = O.ir_solve(As[i], bs[i], O.F32)
            assert r["tf"] == ir.F32
            assert r["status"] == O.STATUS_NAMES[o.status] and r["iters"] == o.iters
            np.testing.assert_array_equal(xs[i], o.x)
        else:
            assert r["tf"] == ir.F16 and r == first[i]
    # graph capture of the escalating run gives the same bits
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            plan.run_escalate("f32", rtol)
    for x in plan.xs:
        x.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for a, x in zip(xs, plan.xs):
        np.testing.assert_array_equal(a, x.cpu().numpy())
    assert plan.results() == res
    with pytest.raises(ir.IRError, match="IR_EINVAL"):
        plan.run_escalate("f16")
