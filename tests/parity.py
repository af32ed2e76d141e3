"""Parity rules shared by the GPU tests (test infrastructure; uses the oracle).

* ``bar(kappa)``: the forward-error bar for a solution of Algorithm IR with
  TW = binary64, max(1e-12, 10 kappa_inf eps64) against the binary64 oracle
  solution x_ref (the literal 1e-12 for kappa <= 1e8 where the rounding floor
  allows it; the paper's own converged solutions at kappa ~ 1e5 are ~2e-12 off,
  Table ip3).
* ``classify(o, ok)``: where the oracle's own refinement run ``o`` sits with
  respect to the convergence boundary of its factorization precision.  The
  termination rule of Sec. 5.1 decides with the ratio ||r_{k+1}|| / ||r_k||
  against R_max (eq. stag), and the ratio measures the contraction factor of
  the iteration, which is proportional to kappa u_F (Sec. 5.4.2, eq. rate2).
  "Within 2x of the boundary" is therefore read on the ratios: a run is near
  the boundary when any ratio of its contraction phase lies in [R_max/2,
  2 R_max).  The contraction phase is the part of the history still 100x above
  the final residual; below that the ratios measure rounding noise at the
  floor, not the contraction.  Classes:
    conv  contraction ratios < R_max/2 and x meets the bar
    slow  contraction ratios < R_max/2, litmax reached before the bar
    fail  the first ratio >= 2 R_max (the iteration diverges at once)
    near  everything else (excluded from status comparisons)
* ``pivot_envelope(AF, LU, ipiv, nb, tf)``: the a-priori envelope of the
  candidates of each pivot step of a tensor-core factorization (see the
  function).
"""
from __future__ import annotations

import numpy as np

import oracle as O

EPS64 = 2.0 ** -52


def bar(kappa: float) -> float:
    return max(1e-12, 10.0 * kappa * EPS64)


def meets_bar(x, xr, kappa: float) -> bool:
    return O.rel_err_inf(x, xr) <= bar(kappa)


def classify(o, ok: bool, rmax: float = 0.5) -> str:
    h = o.rhist
    if len(h) < 2:
        return "conv" if ok else "near"
    rat = [h[k + 1] / h[k] if h[k] > 0 else 0.0 for k in range(len(h) - 1)]
    floor = h[-1]
    contraction = [r for k, r in enumerate(rat) if h[k + 1] > 100.0 * floor]
    if rat[0] >= 2 * rmax:
        return "fail"
    if any(r >= rmax / 2 for r in contraction):
        return "near"
    if ok:
        return "conv"
    if o.status == O.MAXIT:
        return "slow"
    return "near"


def status_must_match(o, cls: str, litmax: int = 10) -> bool:
    """Whether the GPU's status must equal the oracle's.  A converging run stops at
    the rounding floor, where the step at which eq. (stag) fires is noise; when the
    oracle's run ends within two steps of litmax the other run may reach litmax
    first, so only runs that end earlier are held to the same status."""
    if cls == "near":
        return False
    if cls == "conv":
        return o.iters <= litmax - 2
    return True


def pivot_envelope(AF: np.ndarray, LU: np.ndarray, ipiv: np.ndarray, nb: int, tf: int,
                   c: float = 4.0) -> np.ndarray:
    """E[k]: how far the GPU's candidate magnitudes at pivot step k may lie from the
    oracle's, fixed from the oracle's own factors before looking at the GPU's.

    Column k reaches step k after ceil(k / nb) blocked trailing updates, sums of
    products rTF(l_im) rTF(u_mk), m < k.  Two sources of difference:
      * accumulation: the tensor core sums nb products in binary32 where the
        oracle sums them exactly and rounds once, and the sum is added to the
        binary32 entry: about nb u32 sum_m |l_im||u_mk| + u32 |a_ik| per update,
        the reading's tau_k = 4 nb 2^-23 ceil(k/nb) times (T_ik + |a_ik|);
      * rounding flips: once an operand's binary32 value differs in its last bits
        (from an earlier accumulation difference), its rounding to TF can land on
        the neighbouring TF number, a change of up to 2 u_TF of the operand, so
        a product can move by up to 4 u_TF |l_im||u_mk|: 4 u_TF T_ik.
    T_ik = sum_{m<k} |l_im||u_mk| is eq. (comperr)'s |L||U| restricted to the
    updates column k received; the envelope takes its largest value among the
    step's candidates i >= k (rows in the final order, |P A_F| added).
    """
    n = LU.shape[0]
    if n == 0:
        return np.zeros(0)
    L = np.tril(LU.astype(np.float64), -1) + np.eye(n)
    U = np.triu(LU.astype(np.float64))
    T = np.abs(L) @ np.abs(U)                       # (|L||U|)_ik = sum_{m <= min(i,k)}
    T -= np.abs(L) * np.abs(np.diag(U))[None, :]    # drop m = k: what column k received before step k
    T = np.where(np.arange(n)[:, None] >= np.arange(n)[None, :], T, 0.0)   # candidates i >= k
    Aabs = np.abs(AF.astype(np.float64)[O.perm_from_ipiv(ipiv)])
    Aabs = np.where(np.arange(n)[:, None] >= np.arange(n)[None, :], Aabs, 0.0)
    tau = c * nb * 2.0 ** -23 * np.ceil(np.arange(n) / nb)
    return tau * (T + Aabs).max(axis=0) + 4.0 * O.UNIT_ROUNDOFF[tf] * T.max(axis=0)


def candidates(LU: np.ndarray, k: int) -> np.ndarray:
    """|a_ik| of the candidates of step k (rows >= k, final row order), rebuilt
    from the factors: a_kk = u_kk, a_ik = l_ik u_kk below the diagonal."""
    col = LU[k:, k].astype(np.float64) * LU[k, k]
    col[0] = LU[k, k]
    return np.abs(col)
