"""The seeded input generators (irgen) against the recipes they claim: the
spectrum of the kappa = 1e6 SVD workload, the sizes and coefficients of the
uneven batch, and the eigenvector right-hand side of the Green's workload."""
import numpy as np
import pytest

import irgen


@pytest.mark.parametrize("n", [8, 64, 200])
def test_svd_case_has_the_geometric_spectrum(n):
    A, b = irgen.case_svd(n, 44, kappa=1e6)
    assert A.dtype == np.float32 and b.dtype == np.float32 and A.flags.f_contiguous
    s_want = 1e6 ** (-np.arange(n) / (n - 1))
    s_got = np.linalg.svd(A.astype(np.float64), compute_uv=False)
    # A is the binary32 rounding of U diag(s) V^T: each singular value moves by
    # at most ||A64 - fl32(A64)||_2 <= ||.||_F <= n 2^-24 max|a_ij|
    tol = n * 2.0 ** -24 * np.max(np.abs(A))
    assert np.max(np.abs(s_got - s_want)) <= tol
    assert s_got[0] == pytest.approx(1.0, abs=tol)
    # b = fl32(A64 1): within binary32 rounding of the rounded matrix's product
    b_re = A.astype(np.float64) @ np.ones(n)
    assert np.max(np.abs(b.astype(np.float64) - b_re)) <= 2 * n * 2.0 ** -24 * np.max(np.abs(b_re)) + 1e-7


def test_batch_case_recipe():
    count = 400
    ns, alphas, As, bs = irgen.case_batch(count, 1005)
    assert len(ns) == len(alphas) == len(As) == len(bs) == count
    assert ns.min() >= 32 and ns.max() <= 512
    assert np.all((alphas >= 1.0) & (alphas <= 800.0))
    # N ~ U{32..512}: mean 272, standard deviation of the mean ~ 139 / sqrt(count)
    assert abs(ns.mean() - 272.0) < 5 * 139.0 / np.sqrt(count)
    for n, a, A, b in list(zip(ns, alphas, As, bs))[:12]:
        n = int(n)
        assert A.shape == (n, n) and A.flags.f_contiguous and np.all(b == 1.0)
        # symmetric part I - alpha G_mid (G is symmetric), the rest 1e-3 (E - E^T)/2
        G = irgen.gmat_midpoint(n)
        S = (A + A.T) / 2
        E_sym = (S - (np.eye(n) - a * G)) / 1e-3
        E_skew = (A - A.T) / 2 / 1e-3
        # the symmetric and skew parts of a Gaussian matrix have entry variance 1/2
        assert 0.3 < np.var(E_sym) < 0.7 and 0.3 < np.var(E_skew[np.triu_indices(n, 1)]) < 0.7
    # the same seed gives the same systems; sizes given explicitly reuse the recipe
    ns2, alphas2, As2, _ = irgen.case_batch(count, 1005)
    assert np.array_equal(ns, ns2) and np.array_equal(alphas, alphas2) and np.array_equal(As[0], As2[0])
    al3, As3, bs3 = irgen.case_batch_sizes([0, 40], 7)
    assert As3[0].shape == (0, 0) and As3[1].shape == (40, 40) and 1.0 <= al3[1] <= 800.0


@pytest.mark.parametrize("n", [64, 384])
def test_green_sine_rhs_is_the_first_eigenvector(n):
    """x_true_i = sin(pi x_i) is the k = 1 eigenvector of G_mid with eigenvalue
    h^2 / (4 sin^2(pi h / 2)), so b = A x_true = (1 - alpha lambda_1) x_true."""
    alpha = 800.0
    A, b, xt = irgen.case_green_sine(n, alpha)
    h = 1.0 / n
    lam1 = h * h / (4.0 * np.sin(np.pi * h / 2) ** 2)
    assert np.max(np.abs(b - (1.0 - alpha * lam1) * xt)) <= 64 * n * 2.0 ** -52 * alpha * np.max(np.abs(xt))
    assert np.array_equal(xt, np.sin(np.pi * irgen.midpoint_nodes(n)))


def test_gaussian_case_is_diagonally_shifted():
    n = 300
    A, b = irgen.case_gaussian(n, 12)
    off = A - np.diag(np.diag(A))
    assert abs(np.mean(np.diag(A)) - 2.0 * np.sqrt(n)) < 0.5
    assert abs(np.std(off[~np.eye(n, dtype=bool)]) - 1.0) < 0.02 and b.shape == (n,)
