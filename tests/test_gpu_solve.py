"""Parity of the CUDA correction solve, residual and refinement loop with the oracle."""
import numpy as np
import pytest
import torch

import irgen
import oracle as O
import parity as P
from gpu_util import dev_colmajor, dev_vec
from paper_2311_14616_gb300 import ir

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 7, 64, 65, 130, 333, 1000])
def test_lu_solve_matches_oracle_substitution(ctx, n):
    """d = U^{-1} L^{-1} P v on the GPU's own factors vs the oracle's substitution."""
    A, _ = irgen.case_random(n, 50 + n)
    f = ctx.factor(dev_colmajor(A), tf="f32")
    LU, piv = f.factors(), f.pivots()
    v = np.random.Generator(np.random.PCG64(n)).standard_normal(n).astype(np.float32)
    d = f.lu_solve(dev_vec(v)).cpu().numpy()
    do = O.getrs_f32(LU, piv, v)
    # both are binary32 solves of the same triangular systems; their difference is
    # bounded by the conditioning of the factors times the binary32 unit roundoff
    L = np.tril(LU.astype(np.float64), -1) + np.eye(n)
    U = np.triu(LU.astype(np.float64))
    dx = np.linalg.solve(U, np.linalg.solve(L, O.apply_pivots(piv, v.astype(np.float64))))
    cond = np.linalg.cond(L, np.inf) * np.linalg.cond(U, np.inf)
    tol = 4 * n * 2.0 ** -24 * cond * np.max(np.abs(dx))
    assert np.max(np.abs(d - dx)) <= tol
    assert np.max(np.abs(do - dx)) <= tol


@pytest.mark.parametrize("n", [1, 5, 255, 256, 257, 1023, 3000])
@pytest.mark.parametrize("tw", [np.float64, np.float32])
def test_residual_matches_oracle(ctx, n, tw):
    A, b = irgen.case_gaussian(n, 70 + n)
    A = np.asfortranarray(A.astype(tw))
    b = b.astype(tw)
    x = np.random.Generator(np.random.PCG64(n + 1)).standard_normal(n)
    r, rn = ctx.residual(dev_colmajor(A), dev_vec(b), dev_vec(x))
    r = r.cpu().numpy()
    ro = O.residual(A, b, x)
    g = 2 * n * 2.0 ** -53
    bound = g * (np.abs(A).astype(np.float64) @ np.abs(x) + np.abs(b.astype(np.float64)))
    assert np.all(np.abs(r - ro) <= bound + 1e-300)
    assert float(rn.cpu()[0]) == np.max(np.abs(r))


def _cfg_cases():
    yield "green_a1_N256_f32", lambda: irgen.case_green(256, 1.0), O.F32, dict(abs_rel_tol=1e-13)
    yield "green_sine_a800_N512_f32", lambda: irgen.case_green_sine(512)[:2], O.F32, {}
    # TF32 factors of this kappa ~ 1e5 system contract slowly: allow 30 iterations
    yield "green_sine_a800_N520_tf32", lambda: irgen.case_green_sine(520)[:2], O.TF32, dict(litmax=30)
    yield "gauss_N700_f16", lambda: irgen.case_gaussian(700, 9), O.F16, {}
    yield "gauss_N700_bf16", lambda: irgen.case_gaussian(700, 9), O.BF16, {}
    yield "gauss_N300_tf32", lambda: irgen.case_gaussian(300, 4), O.TF32, {}
    yield "random_N300_f32", lambda: irgen.case_random(300, 3), O.F32, {}


@pytest.mark.parametrize("name,make,tf,term", list(_cfg_cases()), ids=[c[0] for c in _cfg_cases()])
def test_ir_matches_oracle(ctx, name, make, tf, term):
    A, b = make()
    n = A.shape[0]
    f = ctx.factor(dev_colmajor(A), tf=O.DTYPE_NAMES[tf])
    x, rep = f.solve(dev_vec(b), term=ir.default_term(**term))
    x = x.cpu().numpy()
    ref = O.ir_solve(A, b, tf, O.Term(**term), nb=64)
    xr = O.reference_solution(A, b)
    kappa = O.cond_inf(A)
    tol = O.parity_tol(kappa, O.F64)
    # status away from the convergence boundary of the TF (parity.classify).  Binary32
    # factors are bitwise the oracle's (one iteration of slack for the solves' order);
    # with TF32 / 16-bit factors the contraction factor kappa u_F c (Sec. 5.4.2) carries
    # the factorization's own error, which the tensor core's binary32 accumulation and
    # the oracle's exact sums make differently -- near the boundary (TF32 on the
    # kappa ~ 1e5 Green's system: kappa u_TF32 ~ 65) by a factor of two or so -- so the
    # step count is held to within a factor of two
    cls = P.classify(ref, O.rel_err_inf(ref.x, xr) <= tol)
    if P.status_must_match(ref, cls, ir.default_term(**term).litmax):
        assert rep.status == O.STATUS_NAMES[ref.status]
    else:
        assert rep.status in ("converged", "stagnated")
    if tf == O.F32:
        assert abs(rep.iters - ref.iters) <= 1
    else:
        assert ref.iters // 2 <= rep.iters <= 2 * ref.iters + 1, (rep.iters, ref.iters)
    assert rep.rhist[0] == ref.rhist[0]
    # every case here is one where the oracle's own IR meets the bar against x_ref
    # (whatever its stopping rule: these runs end by eq. (stag) at the rounding
    # floor), so the GPU's x is always compared, with both
    assert O.rel_err_inf(ref.x, xr) <= tol, (name, O.rel_err_inf(ref.x, xr), tol)
    assert O.rel_err_inf(x, ref.x) <= tol, (O.rel_err_inf(x, ref.x), tol)
    assert O.rel_err_inf(x, xr) <= tol, (O.rel_err_inf(x, xr), tol)


def test_ir_promoted_single_single_double(ctx):
    """TW = TF = binary32, TR = binary64 (Sec. 2.2.2): correction-stagnation rule and
    the bound of Thm. carsonh1 against the promoted problem's solution."""
    n = 384
    A, b = irgen.case_svd(n, 1004, kappa=1e4)
    f = ctx.factor(dev_colmajor(A), tf="f32")
    x, rep = f.solve(dev_vec(b))
    ref = O.ir_solve(A, b, O.F32)
    xp = O.reference_solution(A, b)
    kappa = O.cond_inf(A)
    assert x.dtype == torch.float32
    assert rep.status == "stagnated" and ref.status == O.STAGNATED
    bound = 4 * (n + 1) * kappa * 2.0 ** -53 + 2.0 ** -24
    assert O.rel_err_inf(x.cpu().numpy(), xp) <= bound


def test_ir_singular_and_nonfinite(ctx):
    S = np.asfortranarray(np.ones((4, 4)))
    f = ctx.factor(dev_colmajor(S), tf="f32")
    with pytest.raises(ir.IRError) as e:
        f.solve(dev_vec(np.ones(4)))
    assert e.value.code == 4 and e.value.report.info == 2 and e.value.report.status == "failed"
    A, b = irgen.case_gaussian(50, 2)
    f = ctx.factor(dev_colmajor(A), tf="f32")
    b[7] = np.inf
    with pytest.raises(ir.IRError) as e:
        f.solve(dev_vec(b))
    assert e.value.code == 5


def test_ir_edge_sizes_and_zero_rhs(ctx):
    A = np.array([[4.0]], order="F")
    f = ctx.factor(dev_colmajor(A), tf="f32")
    x, rep = f.solve(dev_vec(np.array([2.0])))
    assert x.cpu().item() == 0.5 and rep.status == "converged"
    A0 = np.zeros((0, 0), order="F")
    f0 = ctx.factor(torch.zeros((0, 0), dtype=torch.float64, device="cuda"), tf="f32")
    x0, rep0 = f0.solve(torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert x0.numel() == 0 and rep0.status == "converged"
    A, _ = irgen.case_gaussian(90, 3)
    f = ctx.factor(dev_colmajor(A), tf="tf32")
    x, rep = f.solve(dev_vec(np.zeros(90)))
    assert rep.status == "converged" and rep.iters == 0 and not torch.any(x)


def test_invalid_arguments_and_limits(ctx):
    from paper_2311_14616_gb300.ir import IRError
    n = 77825                   # one row more than the tallest panel (152 CTAs x 512 rows)
    big = torch.empty((n, n), dtype=torch.float32, device="cuda")    # 24 GB, never read
    with pytest.raises(IRError) as e:
        ctx.factor(big.t(), tf="f32")
    assert e.value.code == 7
    del big
    with pytest.raises(IRError) as e:
        ctx.factor(dev_colmajor(np.eye(4)), tf=9)
    assert e.value.code == 1


def test_refactor_reuses_storage(ctx):
    A, b = irgen.case_gaussian(200, 11)
    B, _ = irgen.case_gaussian(200, 12)
    f = ctx.factor(dev_colmajor(A), tf="f32")
    Bt = dev_colmajor(B)
    f.refactor(Bt)
    x, rep = f.solve(dev_vec(b))
    xr = O.reference_solution(B, b)
    ref = O.ir_solve(B, b, O.F32)
    assert rep.status in ("converged", "stagnated") and ref.status in (O.CONVERGED, O.STAGNATED)
    assert O.rel_err_inf(x.cpu().numpy(), xr) <= 1e-12
    assert np.array_equal(f.factors(), O.getrf_tf(O.cast(B, O.F32), O.F32)[0])


def test_solve_host_end_to_end(ctx):
    A, b = irgen.case_green(300, 800.0)
    xh, rep = ctx.solve_host(torch.from_numpy(A), torch.from_numpy(b), tf="f32")
    xr = O.reference_solution(A, b)
    assert not xh.is_cuda
    assert O.rel_err_inf(xh.numpy(), xr) <= O.parity_tol(O.cond_inf(A), O.F64)
    # the context keeps the buffers and the factorization for the same shape: a
    # second call with another matrix of that shape refactors into them, and a
    # call of another shape replaces them -- each result is its own system's
    A2, b2 = irgen.case_gaussian(300, 8)
    xh2, _ = ctx.solve_host(torch.from_numpy(A2), torch.from_numpy(b2), tf="f32")
    assert O.rel_err_inf(xh2.numpy(), O.reference_solution(A2, b2)) <= 1e-12
    xh1, _ = ctx.solve_host(torch.from_numpy(A), torch.from_numpy(b), tf="f32")
    np.testing.assert_array_equal(xh1.numpy(), xh.numpy())
    A3, b3 = irgen.case_gaussian(77, 9)
    xh3, _ = ctx.solve_host(torch.from_numpy(A3), torch.from_numpy(b3), tf="f16")
    assert O.rel_err_inf(xh3.numpy(), O.reference_solution(A3, b3)) <= 1e-12


def test_lu_solve_backward_stable_with_ill_conditioned_diagonal_blocks(ctx):
    """U = D W with D graded from 1 to 1e-12 and W unit upper triangular close
    to I: no interchanges, U = A, and two of its three 128-row diagonal blocks
    have condition numbers above 1e5 (3e5), far too high for an explicit
    inverse, so the solve takes them by substitution; the correction solve
    must stay backward stable (componentwise, gamma_n |U| |d|), as the LU
    solve of Algorithm IR assumes (Sec. 5.4.1)."""
    n = 300
    g = np.random.default_rng(5)
    dg = np.logspace(0, -12, n) * np.where(g.random(n) < 0.5, -1.0, 1.0)
    W = np.eye(n) + np.triu(g.standard_normal((n, n)), 1) * (0.3 / np.sqrt(n))
    A = np.asfortranarray((dg[:, None] * W).astype(np.float32))
    f = ctx.factor(dev_colmajor(A), tf="f32")
    assert np.array_equal(f.pivots(), np.arange(n, dtype=np.int32))
    v = g.standard_normal(n).astype(np.float32)
    d = f.lu_solve(dev_vec(v)).cpu().numpy().astype(np.float64)
    U = A.astype(np.float64)
    r = U @ d - v.astype(np.float64)
    bound = 2 * n * 2.0 ** -24 * (np.abs(U) @ np.abs(d) + np.abs(v))
    assert np.all(np.abs(r) <= bound), float(np.max(np.abs(r) / bound))


@pytest.mark.parametrize("tw", [np.float64, np.float32])
def test_backward_error_termination_matches_oracle(ctx, tw):
    """eq. (term) with ||A||_1: on I - 799 G (Sec. 5.1.3's system) the residual floor
    is far above eps ||b||; the backward-error test stops there as converged, where
    the residual test stops on stagnation one step later."""
    A64 = np.asfortranarray(np.eye(512) - 799.0 * irgen.gmat_trapezoid(512))
    A = np.asfortranarray(A64.astype(tw))
    b = np.ones(512, dtype=tw)
    f = ctx.factor(dev_colmajor(A), tf="f32")
    for mode in (0, 1):
        x, rep = f.solve(dev_vec(b), term=ir.default_term(mode=mode))
        ref = O.ir_solve(A, b, O.F32, O.Term(mode=mode))
        assert rep.status == O.STATUS_NAMES[ref.status], (mode, rep.rhist, ref.rhist)
        # TW = binary32: the correction test (eq. wilkterm) decides, one step of slack
        assert abs(rep.iters - ref.iters) <= (0 if tw == np.float64 else 1)
        xr = O.reference_solution(A, b)
        tol = O.parity_tol(O.cond_inf(A), O.F64) if tw == np.float64 else 2.0 ** -23
        assert O.rel_err_inf(x.cpu().numpy(), xr) <= tol
    if tw == np.float64:
        assert ref.status == O.CONVERGED
    # the norm is cached per factorization and recomputed after a refactor
    B = np.asfortranarray(2.0 * A)
    f.refactor(dev_colmajor(B))
    x, rep = f.solve(dev_vec(b), term=ir.default_term(mode=1))
    ref = O.ir_solve(B, b, O.F32, O.Term(mode=1))
    assert rep.status == O.STATUS_NAMES[ref.status]
    assert abs(rep.iters - ref.iters) <= (0 if tw == np.float64 else 1)


def test_gmres_ir_backward_error_termination(ctx):
    A = np.asfortranarray(np.eye(512) - 799.0 * irgen.gmat_trapezoid(512))
    b = np.ones(512)
    f = ctx.factor(dev_colmajor(A), tf="f16")
    x, rep = f.solve_gmres(dev_vec(b), term=ir.default_term(mode=1))
    ref = O.gmres_ir_solve(A, b, O.F16, O.Term(mode=1), nb=64)
    assert rep.status == O.STATUS_NAMES[ref.status] == "converged"
    assert abs(rep.iters - ref.iters) <= 1
    assert O.rel_err_inf(x.cpu().numpy(), O.reference_solution(A, b)) <= O.parity_tol(O.cond_inf(A), O.F64)


def test_term_mode_validation(ctx):
    A, b = irgen.case_gaussian(40, 1)
    f = ctx.factor(dev_colmajor(A), tf="f32")
    with pytest.raises(ir.IRError, match="IR_EINVAL"):
        f.solve(dev_vec(b), term=ir.default_term(mode=2))
    As = [dev_colmajor(A)]
    with pytest.raises(ir.IRError, match="IR_EUNSUPPORTED"):
        ctx.solve_batched(As, [dev_vec(b)], tf="f32", term=ir.default_term(mode=1))


def test_solve_many_columns_equal_single_solves(ctx):
    """ir_solve_many: one factorization, nrhs independent IR loops; each column is
    bitwise the single-right-hand-side solve, with its own termination."""
    A, _ = irgen.case_green(777, 800.0)
    g = np.random.Generator(np.random.PCG64(4242))
    B = g.standard_normal((777, 5))
    B[:, 3] = 0.0                                      # a zero column converges at once
    f = ctx.factor(dev_colmajor(A), tf="f32")
    X, reps = f.solve_many(torch.from_numpy(B).cuda())
    X = X.cpu().numpy()
    for j in range(5):
        x, rep = f.solve(dev_vec(np.ascontiguousarray(B[:, j])))
        np.testing.assert_array_equal(X[:, j], x.cpu().numpy())
        assert reps[j].status == rep.status and reps[j].rhist == rep.rhist
    assert reps[3].status == "converged" and reps[3].iters == 0
    xr = O.reference_solution(A, B[:, 0])
    assert O.rel_err_inf(X[:, 0], xr) <= O.parity_tol(O.cond_inf(A), O.F64)


@pytest.mark.parametrize("n,tf,store,tw", [(700, "f32", False, np.float64), (5000, "f32", False, np.float64),
                                            (1500, "f16", True, np.float64), (300, "bf16", False, np.float64),
                                            (600, "f16", False, np.float32)])
def test_solve_many_blocked_equals_single_solves(ctx, n, tf, store, tw):
    """ir_solve_many refines up to 4 columns together: each factor tile of the
    correction solve is applied to all of them and each residual reads A once,
    with every column's own scaling, history and termination.  Per column the
    arithmetic is that of the single-column path, in the same order, so x and
    the histories are bitwise the single solves' -- for blocks of 4, a ragged
    last block, a zero column, a non-finite column, the sync-free solve pair
    (n > 4096), 2-byte factors, the backward-error test, and TW = binary32."""
    A, _ = irgen.case_gaussian(n, 5000 + n)
    A = np.asfortranarray(A.astype(tw))
    g = np.random.Generator(np.random.PCG64(n))
    B = g.standard_normal((n, 9)).astype(tw)
    B[:, 5] = 0.0
    B[:, 2] *= 1e-3
    f = ctx.factor(dev_colmajor(A), tf=tf, store_tf=store)
    for mode in (0, 1):
        term = ir.default_term(mode=mode)
        X, reps = f.solve_many(torch.from_numpy(B).cuda(), term=term)
        X = X.cpu().numpy()
        for j in range(9):
            x, rep = f.solve(dev_vec(np.ascontiguousarray(B[:, j])), term=term)
            np.testing.assert_array_equal(X[:, j], x.cpu().numpy())
            assert reps[j].status == rep.status and reps[j].rhist == rep.rhist and reps[j].dhist == rep.dhist
        assert reps[5].status == "converged" and reps[5].iters == 0
    # a non-finite column fails alone; the others are solved
    B[7, 3] = np.inf
    with pytest.raises(ir.IRError) as e:
        f.solve_many(torch.from_numpy(B).cuda())
    assert e.value.code == 5
    x0, rep0 = f.solve(dev_vec(np.ascontiguousarray(B[:, 0])))
    assert rep0.status in ("converged", "stagnated")     # the factorization is still usable


def test_cluster_solve_pair_is_bitwise_the_two_kernel_pair():
    """For N <= 4096 the correction solve runs as one thread-block cluster (y and z
    pushed between CTAs through distributed shared memory, tiles streamed by TMA);
    it applies the same tiles in the same order with the same arithmetic as the
    two-kernel pair (selected with IR_NO_CLUSTER_SOLVE=1), so every result is the
    same bits: raw solves, refinement histories and GMRES-IR corrections."""
    import os
    import subprocess
    import sys
    code = r'''
import json, sys, numpy as np
sys.path.insert(0, ".")
import irgen
from paper_2311_14616_gb300 import ir
from tests.gpu_util import dev_colmajor, dev_vec
ctx = ir.Context(0)
out = []
for n, tf, mk in [(4096, "f32", lambda: irgen.case_green_sine(4096)[:2]), (1, "f32", lambda: irgen.case_gaussian(1, 1)),
                  (130, "bf16", lambda: irgen.case_green(130, 800.0)), (2049, "f16", lambda: irgen.case_green(2049, 799.0)),
                  (3000, "tf32", lambda: irgen.case_random(3000, 5))]:
    A, b = mk()
    f = ctx.factor(dev_colmajor(A), tf=tf)
    v = np.random.Generator(np.random.PCG64(n)).standard_normal(n).astype(np.float32)
    d = f.lu_solve(dev_vec(v)).cpu().numpy()
    x, rep = f.solve(dev_vec(b))
    xg, repg = f.solve_gmres(dev_vec(b))
    out.append([d.tobytes().hex(), x.cpu().numpy().tobytes().hex(), xg.cpu().numpy().tobytes().hex(),
                rep.rhist, repg.khist])
print(json.dumps(out))
'''
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = []
    for flag in ("0", "1"):
        r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=600,
                           env=dict(os.environ, IR_NO_CLUSTER_SOLVE=flag))
        assert r.returncode == 0, r.stderr[-2000:]
        res.append(r.stdout.strip().splitlines()[-1])
    assert res[0] == res[1]
