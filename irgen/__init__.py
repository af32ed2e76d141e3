"""Seeded synthetic inputs for the iterative-refinement solver and its oracle.

This module is shared by the CPU oracle (``oracle/``), the CUDA path's tests and
``bench.py``.  It builds matrices and right-hand sides only; it holds none of
the solver's arithmetic (no factorization, no triangular solve, no residual,
no termination logic).

Matrices are returned as numpy arrays in **column-major** (Fortran) order,
which is the layout the C-ABI expects (LAPACK convention, leading dimension =
number of rows).

Workloads (the paper's integral-equation example of Sec. 2 and the dense
random systems of the build's measurement plan):

* ``gmat_midpoint(N)``  -- midpoint-rule discretisation of the Green's
  operator of -d^2/dx^2 on [0, 1] (Sec. 2): h = 1/N, x_i = (i - 1/2) h,
  G_ij = h g(x_i, x_j), g(x, y) = x (1 - y) for x <= y, y (1 - x) otherwise.
* ``gmat_trapezoid(N)`` -- the paper's own N-point trapezoid rule (Sec. 2 and
  the example of Sec. 2.2.2): h = 1/(N - 1), x_j = j h.  The end weights h/2
  multiply g(x, 0) = g(x, 1) = 0, so G_ij = h g(x_i, x_j) for all i, j.
* dense Gaussian systems with a diagonal shift, an SVD-built ill-conditioned
  matrix, and a batch of uneven Green's-function systems.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "green_g", "gmat_midpoint", "gmat_trapezoid", "midpoint_nodes",
    "case_green", "case_green_sine", "case_gaussian", "case_svd", "case_batch",
    "case_random", "case_batch_sizes", "row_dot", "SEED_BASE",
]

SEED_BASE = 1000


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def green_g(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Green's function of -d^2/dx^2 on [0,1] with zero boundary values (Sec. 2)."""
    X, Y = np.meshgrid(x, y, indexing="ij")
    return np.where(X <= Y, X * (1.0 - Y), Y * (1.0 - X))


def midpoint_nodes(n: int) -> np.ndarray:
    h = 1.0 / n
    return (np.arange(n, dtype=np.float64) + 0.5) * h


def gmat_midpoint(n: int) -> np.ndarray:
    """Midpoint-rule Green's matrix, column-major float64 (n x n)."""
    if n == 0:
        return np.zeros((0, 0), order="F")
    h = 1.0 / n
    x = midpoint_nodes(n)
    return np.asfortranarray(h * green_g(x, x))


def gmat_trapezoid(n: int) -> np.ndarray:
    """The paper's N-point trapezoid-rule Green's matrix (Sec. 2), column-major."""
    if n < 2:
        return np.zeros((n, n), order="F")
    h = 1.0 / (n - 1)
    x = np.arange(n, dtype=np.float64) * h
    return np.asfortranarray(h * green_g(x, x))


def row_dot(A: np.ndarray, x: np.ndarray) -> np.ndarray:
    """A x in binary64 as a sequential sum per row in column order (multiply, then
    add, each rounded): the same bits on every machine, unlike a BLAS product,
    whose blocking and fused operations depend on the library."""
    A = np.asarray(A, dtype=np.float64)
    out = np.zeros(A.shape[0])
    for j in range(A.shape[1]):
        out = out + A[:, j] * x[j]
    return out


def case_green(n: int, alpha: float, rule: str = "midpoint", rhs: str = "ones"):
    """A = I - alpha G (Sec. 2).  rhs = 'ones' gives b = 1; 'A1' gives b = A 1."""
    G = gmat_midpoint(n) if rule == "midpoint" else gmat_trapezoid(n)
    A = np.asfortranarray(np.eye(n) - alpha * G)
    if rhs == "ones":
        b = np.ones(n)
    elif rhs == "A1":
        b = row_dot(A, np.ones(n))
    else:
        raise ValueError(rhs)
    return A, b


def case_green_sine(n: int, alpha: float = 800.0):
    """A = I - alpha G_mid, x_true_i = sin(pi x_i), b = A x_true."""
    A, _ = case_green(n, alpha)
    xt = np.sin(np.pi * midpoint_nodes(n))
    return A, row_dot(A, xt), xt


def case_gaussian(n: int, seed: int):
    """A = N(0,1) entries + 2 sqrt(N) I, b ~ N(0,1)."""
    g = _rng(seed)
    A = g.standard_normal((n, n))
    A[np.diag_indices(n)] += 2.0 * np.sqrt(n)
    b = g.standard_normal(n)
    return np.asfortranarray(A), b


def case_random(n: int, seed: int):
    """Unshifted Gaussian matrix: genuine row interchanges under partial pivoting."""
    g = _rng(seed)
    return np.asfortranarray(g.standard_normal((n, n))), g.standard_normal(n)


def case_svd(n: int, seed: int, kappa: float = 1e6):
    """A = U diag(s) V^T, s geometric from 1 to 1/kappa; returned as float32 A, b.

    b = fl32(A64 @ 1), where A64 is the float64 product before rounding.
    """
    g = _rng(seed)
    U, _ = np.linalg.qr(g.standard_normal((n, n)))
    V, _ = np.linalg.qr(g.standard_normal((n, n)))
    if n > 1:
        s = kappa ** (-np.arange(n, dtype=np.float64) / (n - 1))
    else:
        s = np.ones(n)
    A64 = (U * s) @ V.T
    b = row_dot(A64, np.ones(n)).astype(np.float32)
    return np.asfortranarray(A64.astype(np.float32)), b


def case_batch(count: int, seed: int, nmin: int = 32, nmax: int = 512):
    """Uneven batch: N_i ~ U{nmin..nmax}, A_i = I - alpha_i G_mid + 1e-3 E_i, b_i = 1.

    alpha_i ~ U[1, 800], E_i has N(0,1) entries.  Returns (ns, alphas, As, bs).
    """
    g = _rng(seed)
    ns = g.integers(nmin, nmax + 1, size=count)
    alphas = g.uniform(1.0, 800.0, size=count)
    As, bs = [], []
    for n, a in zip(ns, alphas):
        n = int(n)
        E = g.standard_normal((n, n))
        A = np.eye(n) - a * gmat_midpoint(n) + 1e-3 * E
        As.append(np.asfortranarray(A))
        bs.append(np.ones(n))
    return ns.astype(np.int64), alphas, As, bs


def case_batch_sizes(ns, seed: int):
    """The recipe of case_batch with the sizes given: A_i = I - alpha_i G_mid + 1e-3 E_i
    (alpha_i ~ U[1, 800], E_i N(0,1)), b_i = 1.  Returns (alphas, As, bs)."""
    g = _rng(seed)
    alphas = g.uniform(1.0, 800.0, size=len(ns))
    As, bs = [], []
    for n, a in zip(ns, alphas):
        n = int(n)
        E = g.standard_normal((n, n))
        A = np.eye(n) - a * gmat_midpoint(n) + 1e-3 * E if n else np.zeros((0, 0))
        As.append(np.asfortranarray(A))
        bs.append(np.ones(n))
    return alphas, As, bs
