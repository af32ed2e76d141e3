"""CPU oracle for the iterative-refinement solver -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously-correct implementation of the paper's method
(Kelley, "Using MultiPrecisionArrays.jl: Iterative Refinement in Julia"):

* ``ir_solve``      -- Algorithm IR (Sec. 1) with low-precision solves and the
                       residual scaling of eqs. (vdlow)/(promotevd) (Sec. 5.3),
                       the termination rules of Sec. 5.1 and the residual in
                       TR = binary64 (Sec. 2.2.2, eq. xferrule).
* ``cast``/``getrf_tf``/``getrs_f32``/``residual`` -- the steps, in C
                       (``ir_oracle.c``), unblocked and in the paper's order.
* ``reference_solution`` -- the binary64 solution x_ref every result is
                       compared with: binary64 LU solve refined with
                       extended-precision residuals until the corrections stop
                       shrinking.
* ``term_decide``   -- the termination test of Sec. 5.1, a pure function that
                       the tests replay the paper's printed histories through.
* ``gmres_ir_solve`` -- GMRES-IR (Sec. 4.3): the correction equation solved by
                       left-preconditioned GMRES with P = U^{-1} L^{-1}
                       (eq. pdef), ``gmres_correction``.
* ``bicgstab_ir_solve`` -- BiCGSTAB-IR (Sec. 2.3, 4.2): the same with BiCGSTAB.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library and never imports it.

Readings of the paper taken here (each also listed in the design notes):
* u_W in the termination tests is Julia's ``eps(TW)`` (2^-52, 2^-23), the value
  the paper's printed histories agree with.
* The small-residual test (eq. residterm) is applied as ``||r|| <= C_r u_W ||b||``:
  the toy IR listing of Sec. 2.1.1 loops while ``rnorm > tol*norm(b)``, and the
  Float16 history of Sec. 2.2.1 stops at a residual equal to eps.
* The stagnation test (eq. stag) is ``||r_new|| >= R_max ||r_old||``; when
  TR is wider than TW only the correction test (eq. wilkterm)
  ``||d_new|| >= R_max ||d_old||`` is applied (Sec. 5.1; the histories of
  Sec. 2.2.2 and 2.3 continue past residual ratios >= R_max).
* Norms are infinity norms; the solve scales r by ||r||_inf (eq. vdlow).
* An iteration is one residual computation (Sec. 5.1.2); litmax bounds them.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import sys
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "ir_oracle.c")

F64, F32, TF32, BF16, F16 = 0, 1, 2, 3, 4
DTYPE_NAMES = {F64: "f64", F32: "f32", TF32: "tf32", BF16: "bf16", F16: "f16"}
# Julia eps(T): the spacing of T at 1.0 (Sec. 5.4.1 uses it as u)
EPS = {F64: 2.0 ** -52, F32: 2.0 ** -23, TF32: 2.0 ** -10, BF16: 2.0 ** -7, F16: 2.0 ** -10}
# unit roundoff (half the spacing), for the rounding-error bounds of Sec. 5.4
UNIT_ROUNDOFF = {k: v / 2 for k, v in EPS.items()}

CONVERGED, STAGNATED, MAXIT, DIVERGED, FAILED = 0, 1, 2, 3, 4
STATUS_NAMES = {CONVERGED: "converged", STAGNATED: "stagnated", MAXIT: "maxit",
                DIVERGED: "diverged", FAILED: "failed"}


def build(force: bool = False) -> str:
    """Compile ir_oracle.c into a shared library (gcc, OpenMP, no contraction)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    flags = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared"]
    if platform.machine() in ("x86_64", "AMD64"):
        flags.append("-mfma")  # hardware fma; results equal the libm fma exactly
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *flags, _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        sig = {
            "orc_round_tf": (ctypes.c_float, [ctypes.c_float, i32]),
            "orc_round_tf_array": (None, [i64, vp, vp, i32]),
            "orc_cast": (None, [i64, i32, vp, i64, dbl, i32, vp, i64]),
            "orc_maxabs": (dbl, [i64, i32, vp, i64]),
            "orc_getrf_f64": (i64, [i64, vp, i64, vp]),
            "orc_getrf_tf": (i64, [i64, vp, i64, vp, i32, i64, vp, vp]),
            "orc_getrs_f32": (None, [i64, vp, i64, vp, vp]),
            "orc_getrs_f64": (None, [i64, vp, i64, vp, vp]),
            "orc_residual": (None, [i64, i32, vp, i64, vp, vp, vp]),
            "orc_residual_ext": (None, [i64, i32, vp, i64, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _tw_of(A: np.ndarray) -> int:
    if A.dtype == np.float64:
        return F64
    if A.dtype == np.float32:
        return F32
    raise TypeError(f"working precision must be float64 or float32, got {A.dtype}")


# --------------------------------------------------------------------------
# steps
# --------------------------------------------------------------------------

def round_tf(x: np.ndarray, tf: int) -> np.ndarray:
    """Round binary32 values to TF (TF32: ties away; bf16/fp16: ties to even)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    lib().orc_round_tf_array(x.size, _p(x), _p(y), tf)
    return y


def maxabs(A: np.ndarray) -> float:
    A = np.asfortranarray(A)
    n = A.shape[0]
    return float(lib().orc_maxabs(n, _tw_of(A), _p(A), max(n, 1)))


def fp16_scale(A: np.ndarray) -> float:
    """s = 2^10 / max|a_ij|, the scaling that moves A into the binary16 range."""
    m = maxabs(A)
    return 1.0 if m == 0.0 or not np.isfinite(m) else 1024.0 / m


def cast(A: np.ndarray, tf: int, s: float = 1.0) -> np.ndarray:
    """A_F = round_TF(fl32(s A)) as a column-major binary32 array (Sec. 1)."""
    A = np.asfortranarray(A)
    n = A.shape[0]
    AF = np.empty((n, n), dtype=np.float32, order="F")
    lib().orc_cast(n, _tw_of(A), _p(A), max(n, 1), s, tf, _p(AF), max(n, 1))
    return AF


def getrf_f64(A: np.ndarray):
    """Unblocked binary64 LU with partial pivoting -> (LU, ipiv, info)."""
    LU = np.array(A, dtype=np.float64, order="F", copy=True)
    n = LU.shape[0]
    ipiv = np.zeros(n, dtype=np.int32)
    info = lib().orc_getrf_f64(n, _p(LU), max(n, 1), _p(ipiv))
    return LU, ipiv, int(info)


def getrf_tf(AF: np.ndarray, tf: int, nb: int = 0, force_piv: Optional[np.ndarray] = None,
             want_gap: bool = False):
    """LU of the binary32 factorization copy (see ir_oracle.c) -> (LU, ipiv, info[, gap])."""
    LU = np.array(AF, dtype=np.float32, order="F", copy=True)
    n = LU.shape[0]
    ipiv = np.zeros(n, dtype=np.int32)
    fp = None
    if force_piv is not None:
        fp = np.ascontiguousarray(force_piv, dtype=np.int32)
    gap = np.zeros(3 * n, dtype=np.float32) if want_gap else None
    info = lib().orc_getrf_tf(n, _p(LU), max(n, 1), _p(ipiv), tf, nb,
                              _p(fp) if fp is not None else None,
                              _p(gap) if gap is not None else None)
    if want_gap:
        return LU, ipiv, int(info), gap.reshape(n, 3)
    return LU, ipiv, int(info)


def getrs_f32(LU: np.ndarray, ipiv: np.ndarray, v: np.ndarray) -> np.ndarray:
    v = np.array(v, dtype=np.float32, copy=True)
    n = v.shape[0]
    LU = np.asfortranarray(LU, dtype=np.float32)
    lib().orc_getrs_f32(n, _p(LU), max(n, 1), _p(np.ascontiguousarray(ipiv, dtype=np.int32)), _p(v))
    return v


def getrs_f64(LU: np.ndarray, ipiv: np.ndarray, v: np.ndarray) -> np.ndarray:
    v = np.array(v, dtype=np.float64, copy=True)
    n = v.shape[0]
    LU = np.asfortranarray(LU, dtype=np.float64)
    lib().orc_getrs_f64(n, _p(LU), max(n, 1), _p(np.ascontiguousarray(ipiv, dtype=np.int32)), _p(v))
    return v


def residual(A: np.ndarray, b: np.ndarray, x: np.ndarray, extended: bool = False) -> np.ndarray:
    """r = b - A x in binary64 (or the host's long double when extended)."""
    A = np.asfortranarray(A)
    n = A.shape[0]
    b64 = np.ascontiguousarray(b, dtype=np.float64)
    x64 = np.ascontiguousarray(x, dtype=np.float64)
    r = np.empty(n, dtype=np.float64)
    f = lib().orc_residual_ext if extended else lib().orc_residual
    f(n, _tw_of(A), _p(A), max(n, 1), _p(b64), _p(x64), _p(r))
    return r


def apply_pivots(ipiv: np.ndarray, v: np.ndarray) -> np.ndarray:
    """P v: the interchanges ipiv applied in order (LAPACK laswp semantics)."""
    v = np.array(v, copy=True)
    for k, p in enumerate(ipiv):
        if p != k:
            v[[k, p]] = v[[p, k]]
    return v


def perm_from_ipiv(ipiv: np.ndarray) -> np.ndarray:
    """perm with (P A)[i] = A[perm[i]]."""
    return apply_pivots(ipiv, np.arange(len(ipiv)))


# --------------------------------------------------------------------------
# Algorithm IR
# --------------------------------------------------------------------------

@dataclass
class Term:
    """Termination parameters (the TERM structure of Sec. 5.1.3)."""
    Cr: float = 1.0
    Ce: float = 1.0
    Rmax: float = 0.5
    litmax: int = 10
    abs_rel_tol: float = 0.0  # > 0: converged iff ||r|| <= abs_rel_tol ||b||
    mode: int = 0             # 0: small residual (eq. residterm); 1: small backward error (eq. term)


@dataclass
class IRResult:
    x: np.ndarray                   # the binary64 accumulator (TR)
    sol: np.ndarray                 # x rounded to TW
    rhist: list = field(default_factory=list)
    dhist: list = field(default_factory=list)
    status: int = CONVERGED
    info: int = 0
    ipiv: Optional[np.ndarray] = None
    LU: Optional[np.ndarray] = None
    scale: float = 1.0

    @property
    def iters(self) -> int:
        return len(self.rhist) - 1


def term_decide(rhist, dhist, bnorm: float, eps_w: float, term: Term, tr_wider: bool,
                rmax_r: Optional[float] = None, anorm: float = 0.0, xnorm: float = 0.0):
    """Termination test of Sec. 5.1, applied after each residual computation.

    rhist = [||r_0||, ..., ||r_k||] (r_0 = b), dhist = [||d_0||, ..., ||d_{k-1}||].
    rmax_r replaces R_max in the residual-stagnation test (eq. stag) when
    given (GMRES-IR); the correction test (eq. wilkterm) keeps term.Rmax.
    term.mode = 1 replaces eq. (residterm) by the backward-error test eq. (term),
    ||r|| <= C_e u_W (||b|| + ||A|| ||x||), with anorm = ||A||_1 and xnorm =
    ||x||_inf of the current iterate.
    Returns a status code, or None to continue.
    """
    k = len(rhist) - 1
    rn = rhist[-1]
    if not np.isfinite(rn):
        return DIVERGED
    if rn == 0.0:
        # x solves the (promoted) system exactly; the scaling r / ||r|| of
        # eq. (vdlow) is undefined for the next step, so stop here
        return CONVERGED
    if tr_wider:
        # eq. (wilkterm): corrections stagnate
        if len(dhist) >= 2 and dhist[-1] >= term.Rmax * dhist[-2]:
            return STAGNATED
    else:
        if term.mode == 1:
            if rn <= term.Ce * eps_w * (bnorm + anorm * xnorm):    # eq. (term)
                return CONVERGED
        else:
            tol = term.abs_rel_tol if term.abs_rel_tol > 0 else term.Cr * eps_w
            if rn <= tol * bnorm:             # eq. (residterm)
                return CONVERGED
        rm = term.Rmax if rmax_r is None else rmax_r
        if k >= 1 and rn >= rm * rhist[-2]:   # eq. (stag)
            return STAGNATED
    if k >= term.litmax:
        return MAXIT
    return None


def ir_solve(A: np.ndarray, b: np.ndarray, tf: int, term: Optional[Term] = None,
             nb: int = 0, fp16_scaling: bool = True, tr_wider: Optional[bool] = None,
             solve: str = "lps", store_tf: bool = False) -> IRResult:
    """Algorithm IR (Sec. 1) with TR = binary64 and solves in binary32.

    1. A_F = round_TF(s A) (s = 2^10/max|a| for TF = binary16, else 1);
       factor A_F = P^T L U (getrf_tf).
    2. x = 0, r = b, rhist = [||b||].
    3. repeat: rho = ||r||; v = fl32(P r / rho); v = U^{-1} L^{-1} v in binary32
       (eq. vdlow); d = (rho s) fl64(v) (eq. promotevd); x += d;
       r = b - A x in binary64; test termination.
    The solution is returned both as the binary64 accumulator and rounded to TW.

    solve = "mps": the mixed precision solves of Sec. 5.3 (interprecision
    transfers on the fly): r is rounded to TW, not below it, and the triangular
    solves run in TW on the factors promoted to TW (exactly), so there is no
    scaling by ||r||: d = s fl64(U^{-1} L^{-1} P fl_W(r)) evaluated in TW.

    store_tf = True (TF = binary16 or bfloat16): the factors are kept in TF,
    as the paper's factorization copy is (Sec. 1, the MPArray of Sec. 2.5):
    after the factorization every entry of L and U is rounded to TF once, and
    the solves use those values (promoted exactly, as in Sec. 5.3).
    """
    if solve not in ("lps", "mps"):
        raise ValueError(solve)
    term = term or Term()
    A = np.asfortranarray(A)
    tw = _tw_of(A)
    n = A.shape[0]
    if tr_wider is None:
        tr_wider = tw == F32   # TR = binary64 is wider than TW = binary32
    b64 = np.ascontiguousarray(b, dtype=np.float64)
    eps_w = EPS[tw]
    s = fp16_scale(A) if (tf == F16 and fp16_scaling) else 1.0
    AF = cast(A, tf, s)
    LU, ipiv, info = getrf_tf(AF, tf, nb)
    if store_tf:
        if tf not in (BF16, F16):
            raise ValueError("2-byte factor storage is for TF = binary16 or bfloat16")
        LU = np.asfortranarray(round_tf(LU, tf).reshape(LU.shape))
    x = np.zeros(n)
    res = IRResult(x=x, sol=x.astype(A.dtype), ipiv=ipiv, LU=LU, scale=s, info=info)
    bnorm = float(np.max(np.abs(b64))) if n else 0.0
    res.rhist.append(bnorm)
    if info != 0:
        res.status = FAILED
        return res
    if bnorm == 0.0:
        res.status = CONVERGED
        return res
    anorm = norm1(A) if term.mode == 1 else 0.0
    r = b64.copy()
    LU64 = LU.astype(np.float64) if (solve == "mps" and tw == F64) else None
    while True:
        if solve == "mps":
            if tw == F64:
                d = s * getrs_f64(LU64, ipiv, r)
            else:
                d = s * getrs_f32(LU, ipiv, r.astype(np.float32)).astype(np.float64)
        else:
            rho = float(np.max(np.abs(r)))
            v = getrs_f32(LU, ipiv, (r / rho).astype(np.float32))
            d = (rho * s) * v.astype(np.float64)
        x += d
        res.dhist.append(float(np.max(np.abs(d))))
        r = residual(A, b64, x)
        res.rhist.append(float(np.max(np.abs(r))))
        st = term_decide(res.rhist, res.dhist, bnorm, eps_w, term, tr_wider,
                         anorm=anorm, xnorm=float(np.max(np.abs(x))))
        if st is not None:
            res.status = st
            break
    res.x = x
    res.sol = x.astype(A.dtype)
    return res


# --------------------------------------------------------------------------
# GMRES-IR (Sec. 4.2-4.3; Sec. 2.3 IR-Krylov)
# --------------------------------------------------------------------------

@dataclass
class KrylovOpts:
    """Options of the Krylov correction solve.

    basissize: the Krylov basis size, i.e. the most GMRES iterations per
               refinement step (default 10, Sec. 4.3).
    eta:       GMRES stops early when its residual estimate falls to
               eta ||P r||_2 (the paper leaves this tolerance unstated).
    Rmax_r:    residual-stagnation factor of the outer loop (eq. stag) when TR
               is not wider than TW; 1 stops when the residual no longer
               decreases (the N = 8102 half-precision GMRES-IR history of
               Sec. 4.5 continues past a ratio of 0.69).
    """
    basissize: int = 10
    eta: float = 1e-8
    Rmax_r: float = 1.0


def precondition(LU: np.ndarray, ipiv: np.ndarray, s: float, w: np.ndarray) -> np.ndarray:
    """P w with P = U^{-1} L^{-1} (eq. pdef) applied as the refinement solve is.

    rho = ||w||_inf; v = fl32(Pi w / rho); v = U^{-1} L^{-1} v in binary32;
    P w = (rho s) fl64(v) (eqs. vdlow, promotevd; s is the binary16 scale of
    A_F = s A, since (s A)^{-1} = A^{-1} / s).  P 0 = 0.
    """
    rho = float(np.max(np.abs(w))) if w.size else 0.0
    if rho == 0.0:
        return np.zeros_like(w, dtype=np.float64)
    v = getrs_f32(LU, ipiv, (w / rho).astype(np.float32))
    return (rho * s) * v.astype(np.float64)


def matvec(A: np.ndarray, v: np.ndarray) -> np.ndarray:
    """A v in TR = binary64 with A promoted exactly: the residual of b = 0, negated."""
    return -residual(A, np.zeros(A.shape[0]), v)


def gmres(op, z: np.ndarray, m: int, eta: float):
    """GMRES (Saad and Schultz) for op(d) = z from d_0 = 0, in binary64.

    Minimises ||z - op(d)||_2 over d in the Krylov space K_k(op, z):
      beta = ||z||_2, v_0 = z / beta, g = beta e_1;
      for j = 0..m-1: w = op(v_j); classical Gram-Schmidt against v_0..v_j,
        done twice (h = h' + h''); h_{j+1,j} = ||w||_2; v_{j+1} = w / h_{j+1,j};
        the Givens rotations of the earlier columns are applied to column j of
        H, a new rotation (c, s) = (h_jj, h_{j+1,j}) / hypot(h_jj, h_{j+1,j})
        zeroes h_{j+1,j}, and g_{j+1} = -s g_j, g_j = c g_j;
        stop when |g_{j+1}| <= eta beta, on breakdown (h_{j+1,j} = 0) or at m;
      y = R^{-1} g (back substitution, R the rotated H), d = V_k y.
    Returns (d, k, est): k iterations, est[j] = |g_{j+1}| (the residual norm
    after iteration j as the rotations give it).
    """
    n = z.shape[0]
    beta = float(np.sqrt(np.dot(z, z)))
    if beta == 0.0 or m < 1:
        return np.zeros(n), 0, []
    V = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    cs = np.zeros(m)
    sn = np.zeros(m)
    g = np.zeros(m + 1)
    V[:, 0] = z / beta
    g[0] = beta
    k = 0
    est = []
    for j in range(m):
        w = op(V[:, j])
        Vj = V[:, :j + 1]
        h1 = Vj.T @ w
        w = w - Vj @ h1
        h2 = Vj.T @ w
        w = w - Vj @ h2
        H[:j + 1, j] = h1 + h2
        hn = float(np.sqrt(np.dot(w, w)))
        H[j + 1, j] = hn
        if hn > 0.0:
            V[:, j + 1] = w / hn
        for i in range(j):
            a, b_ = H[i, j], H[i + 1, j]
            H[i, j] = cs[i] * a + sn[i] * b_
            H[i + 1, j] = -sn[i] * a + cs[i] * b_
        nu = float(np.hypot(H[j, j], H[j + 1, j]))
        if nu == 0.0:
            cs[j], sn[j] = 1.0, 0.0
        else:
            cs[j], sn[j] = H[j, j] / nu, H[j + 1, j] / nu
        H[j, j] = nu
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        k = j + 1
        est.append(abs(g[j + 1]))
        if abs(g[j + 1]) <= eta * beta or hn == 0.0:
            break
    y = np.zeros(k)
    for i in range(k - 1, -1, -1):
        acc = g[i]
        for l in range(i + 1, k):
            acc -= H[i, l] * y[l]
        y[i] = acc / H[i, i] if H[i, i] != 0.0 else 0.0
    return V[:, :k] @ y, k, est


def gmres_correction(A: np.ndarray, LU: np.ndarray, ipiv: np.ndarray, s: float, r: np.ndarray,
                     m: int, eta: float):
    """Left-preconditioned GMRES for the correction equation A d = r (Sec. 4.3):
    ``gmres`` on P A d = P r, with P (eq. pdef) applied by ``precondition``
    and A v in binary64 (the high-precision matrix-vector product).
    Returns (d, k)."""
    d, k, _ = gmres(lambda v: precondition(LU, ipiv, s, matvec(A, v)),
                    precondition(LU, ipiv, s, r), m, eta)
    return d, k


def bicgstab(op, z: np.ndarray, kmax: int, eta: float):
    """BiCGSTAB (van der Vorst) for op(d) = z from d_0 = 0, in binary64.

    r = z, r^ = r, rho_old = alpha = omega = 1, v = p = 0; for i = 1..kmax:
      rho = <r^, r>;  beta = (rho / rho_old)(alpha / omega);
      p = r + beta (p - omega v);  v = op(p);  alpha = rho / <r^, v>;
      s = r - alpha v;  if ||s||_2 <= eta ||z||_2: d += alpha p, stop;
      t = op(s);  omega = <t, s> / <t, t>;  d += alpha p + omega s;
      r = s - omega t;  stop if ||r||_2 <= eta ||z||_2;  rho_old = rho.
    A zero rho, <r^, v> or <t, t> (breakdown) stops the iteration with the
    current d.  Returns (d, k, est): k iterations (two op applications each,
    one for a stop at s), est[i] = the recurrence's ||r||_2 after iteration i.
    """
    n = z.shape[0]
    d = np.zeros(n)
    r = z.astype(np.float64).copy()
    z0 = float(np.sqrt(np.dot(r, r)))
    if z0 == 0.0 or kmax < 1:
        return d, 0, []
    rh = r.copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros(n)
    p = np.zeros(n)
    est = []
    k = 0
    for _ in range(kmax):
        rho = float(np.dot(rh, r))
        if rho == 0.0:
            break
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = op(p)
        sig = float(np.dot(rh, v))
        if sig == 0.0:
            break
        alpha = rho / sig
        s = r - alpha * v
        k += 1
        sn = float(np.sqrt(np.dot(s, s)))
        if sn <= eta * z0:
            d = d + alpha * p
            est.append(sn)
            break
        t = op(s)
        tt = float(np.dot(t, t))
        if tt == 0.0:
            d = d + alpha * p
            est.append(sn)
            break
        omega = float(np.dot(t, s)) / tt
        d = d + alpha * p + omega * s
        r = s - omega * t
        rn = float(np.sqrt(np.dot(r, r)))
        est.append(rn)
        if rn <= eta * z0 or omega == 0.0:
            break
        rho_old = rho
    return d, k, est


@dataclass
class GMRESIRResult(IRResult):
    khist: list = field(default_factory=list)


def bicgstab_ir_solve(A: np.ndarray, b: np.ndarray, tf: int, term: Optional[Term] = None,
                      kopts: Optional[KrylovOpts] = None, nb: int = 0, fp16_scaling: bool = True,
                      tr_wider: Optional[bool] = None, factors=None) -> GMRESIRResult:
    """BiCGSTAB-IR (Sec. 2.3, 4.2): ``gmres_ir_solve`` with the correction equation
    P A d = P r solved by ``bicgstab`` (at most kopts.basissize iterations);
    khist[i] counts BiCGSTAB iterations of refinement step i."""
    return gmres_ir_solve(A, b, tf, term, kopts, nb, fp16_scaling, tr_wider, factors, method="bicgstab")


def gmres_ir_solve(A: np.ndarray, b: np.ndarray, tf: int, term: Optional[Term] = None,
                   kopts: Optional[KrylovOpts] = None, nb: int = 0, fp16_scaling: bool = True,
                   tr_wider: Optional[bool] = None, factors=None, method: str = "gmres") -> GMRESIRResult:
    """GMRES-IR (Sec. 4.3): Algorithm IR with the correction d from
    ``gmres_correction`` instead of one low-precision solve.  Factorization,
    residual (TR = binary64) and the termination tests of Sec. 5.1 are those of
    ``ir_solve``, except that the residual-stagnation factor is kopts.Rmax_r;
    khist[i] is the number of GMRES iterations of refinement step i.
    factors = (LU, ipiv): use these factors of A_F = s A instead of computing
    them (to compare the refinement alone with another implementation's).
    """
    term = term or Term()
    kopts = kopts or KrylovOpts()
    A = np.asfortranarray(A)
    tw = _tw_of(A)
    n = A.shape[0]
    if tr_wider is None:
        tr_wider = tw == F32
    b64 = np.ascontiguousarray(b, dtype=np.float64)
    eps_w = EPS[tw]
    s = fp16_scale(A) if (tf == F16 and fp16_scaling) else 1.0
    if factors is None:
        LU, ipiv, info = getrf_tf(cast(A, tf, s), tf, nb)
    else:
        LU, ipiv = np.asfortranarray(factors[0], dtype=np.float32), np.asarray(factors[1], dtype=np.int32)
        info = 0
    x = np.zeros(n)
    res = GMRESIRResult(x=x, sol=x.astype(A.dtype), ipiv=ipiv, LU=LU, scale=s, info=info)
    bnorm = float(np.max(np.abs(b64))) if n else 0.0
    res.rhist.append(bnorm)
    if info != 0:
        res.status = FAILED
        return res
    if bnorm == 0.0:
        res.status = CONVERGED
        return res
    anorm = norm1(A) if term.mode == 1 else 0.0
    r = b64.copy()
    while True:
        if method == "gmres":
            d, k = gmres_correction(A, LU, ipiv, s, r, kopts.basissize, kopts.eta)
        else:
            d, k, _ = bicgstab(lambda v: precondition(LU, ipiv, s, matvec(A, v)),
                               precondition(LU, ipiv, s, r), kopts.basissize, kopts.eta)
        res.khist.append(k)
        x += d
        res.dhist.append(float(np.max(np.abs(d))))
        r = residual(A, b64, x)
        res.rhist.append(float(np.max(np.abs(r))))
        st = term_decide(res.rhist, res.dhist, bnorm, eps_w, term, tr_wider, rmax_r=kopts.Rmax_r,
                         anorm=anorm, xnorm=float(np.max(np.abs(x))))
        if st is not None:
            res.status = st
            break
    res.x = x
    res.sol = x.astype(A.dtype)
    return res


# --------------------------------------------------------------------------
# reference solution and conditioning
# --------------------------------------------------------------------------

def reference_solution(A: np.ndarray, b: np.ndarray, maxit: int = 10) -> np.ndarray:
    """x_ref ~ fl64(A^{-1} b): binary64 LU solve refined with extended residuals.

    For binary32 A the problem solved is the promoted one (A and b promoted
    exactly to binary64), as in Sec. 2.2.2.
    """
    A = np.asfortranarray(A)
    b64 = np.ascontiguousarray(b, dtype=np.float64)
    LU, ipiv, info = getrf_f64(A.astype(np.float64))
    if info:
        raise np.linalg.LinAlgError(f"singular matrix (zero pivot at {info})")
    x = getrs_f64(LU, ipiv, b64)
    dold = np.inf
    for _ in range(maxit):
        r = residual(A, b64, x, extended=True)
        d = getrs_f64(LU, ipiv, r)
        x = x + d
        dn = float(np.max(np.abs(d)))
        if dn == 0.0 or dn >= 0.5 * dold:
            break
        dold = dn
    return x


def norm1(A: np.ndarray) -> float:
    """||A||_1 = max_j sum_i |a_ij| in binary64 (the operator norm of the
    backward-error test eq. (term); Sec. 5.1.1 and the OPNORM column of Sec. 5.2)."""
    A64 = np.asarray(A, dtype=np.float64)
    if A64.size == 0:
        return 0.0
    return float(np.max(np.sum(np.abs(A64), axis=0)))


def inverse_f64(A: np.ndarray) -> np.ndarray:
    A64 = np.asfortranarray(A, dtype=np.float64)
    n = A64.shape[0]
    LU, ipiv, info = getrf_f64(A64)
    if info:
        raise np.linalg.LinAlgError("singular")
    inv = np.empty((n, n), order="F")
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        inv[:, j] = getrs_f64(LU, ipiv, e)
    return inv


def cond_inf(A: np.ndarray) -> float:
    """kappa_inf(A) = ||A||_inf ||A^{-1}||_inf with the oracle's explicit inverse."""
    A64 = np.asarray(A, dtype=np.float64)
    return float(np.max(np.abs(A64).sum(axis=1)) * np.max(np.abs(inverse_f64(A64)).sum(axis=1)))


def rel_err_inf(x: np.ndarray, xref: np.ndarray) -> float:
    den = float(np.max(np.abs(xref)))
    return float(np.max(np.abs(np.asarray(x, dtype=np.float64) - xref))) / (den if den else 1.0)


def parity_tol(kappa: float, tw: int) -> float:
    """max(1e-12, 10 kappa eps(TW)): the forward-error bar for converged IR."""
    return max(1e-12, 10.0 * kappa * EPS[tw])
