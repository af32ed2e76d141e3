"""Thin ctypes binding of the C ABI in include/ir.h (argument marshalling only).

Every numerical step runs in the CUDA library; this module converts torch
tensors to device pointers, fills the option structs and raises on errors.
It fails loudly when the compiled library is missing: there is no fallback.

Layout: matrices are column-major (LAPACK / Julia).  A torch tensor ``A`` of
shape (n, n) is passed as is when it is already column-major
(``A.stride() == (1, lda)``); otherwise a column-major copy is made and kept
alive by the returned factorization (the factorization borrows A).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field
from typing import List, Optional

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgb300ir.so")

F64, F32, TF32, BF16, F16 = 0, 1, 2, 3, 4
DTYPES = {"f64": F64, "f32": F32, "tf32": TF32, "bf16": BF16, "f16": F16}
STATUS = {0: "converged", 1: "stagnated", 2: "maxit", 3: "diverged", 4: "failed"}
ERRORS = {0: "IR_OK", 1: "IR_EINVAL", 2: "IR_ENOMEM", 3: "IR_ECUDA", 4: "IR_ESINGULAR",
          5: "IR_ENONFINITE", 6: "IR_ETIMEOUT", 7: "IR_EUNSUPPORTED"}
MAX_HIST = 32


class IRError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("TW", ctypes.c_int), ("TF", ctypes.c_int), ("TR", ctypes.c_int),
                ("fp16_scale", ctypes.c_int), ("nb", ctypes.c_int), ("autotune", ctypes.c_int),
                ("group", ctypes.c_int), ("onthefly", ctypes.c_int), ("store_tf", ctypes.c_int)]


class Term(ctypes.Structure):
    _fields_ = [("Cr", ctypes.c_double), ("Ce", ctypes.c_double), ("Rmax", ctypes.c_double),
                ("litmax", ctypes.c_int), ("mode", ctypes.c_int), ("abs_rel_tol", ctypes.c_double)]


class _Report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int),
                ("rhist", ctypes.c_double * MAX_HIST), ("dhist", ctypes.c_double * MAX_HIST),
                ("info", ctypes.c_int64), ("scale", ctypes.c_double)]


class BatchResult(ctypes.Structure):
    """ir_batch_result (one per system of a batch)."""
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("info", ctypes.c_int64),
                ("nonfinite", ctypes.c_int32), ("timeout", ctypes.c_int32), ("rnorm", ctypes.c_double),
                ("scale", ctypes.c_double), ("tf", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("bnorm", ctypes.c_double)]


BATCH_MAX_N = 512
MAX_BASIS = 64


class KrylovOpts(ctypes.Structure):
    """ir_krylov_opts: GMRES basis size, its stopping tolerance, the residual-stagnation factor."""
    _fields_ = [("basissize", ctypes.c_int), ("eta", ctypes.c_double), ("Rmax_r", ctypes.c_double)]


@dataclass
class Report:
    iters: int
    status: str
    rhist: List[float] = field(default_factory=list)
    dhist: List[float] = field(default_factory=list)
    info: int = 0
    scale: float = 1.0
    khist: List[int] = field(default_factory=list)   # GMRES iterations per step (GMRES-IR)


_lib = None


def lib():
    """The loaded C library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        P = ctypes.POINTER
        sigs = {
            "ir_default_opts": (None, [P(Opts)]),
            "ir_default_term": (None, [P(Term)]),
            "ir_init": (i32, [i32, P(vp)]),
            "ir_finalize": (None, [vp]),
            "ir_factor": (i32, [vp, i64, vp, i64, P(Opts), vp, P(vp)]),
            "ir_refactor": (i32, [vp, vp, i64, vp]),
            "ir_solve": (i32, [vp, vp, vp, P(Term), vp, P(_Report)]),
            "ir_solve_host": (i32, [vp, i64, vp, i64, vp, vp, P(Opts), P(Term), vp, P(_Report)]),
            "ir_lu_solve": (i32, [vp, vp, vp, vp]),
            "ir_check_wait_timeout": (i32, [vp, ctypes.c_double, vp]),
            "ir_solve_many": (i32, [vp, i64, vp, i64, vp, i64, P(Term), vp, vp]),
            "ir_default_krylov_opts": (None, [P(KrylovOpts)]),
            "ir_gmres_reserve": (i32, [vp, i32]),
            "ir_solve_gmres": (i32, [vp, vp, vp, P(Term), P(KrylovOpts), vp, P(_Report), vp]),
            "ir_bicgstab_reserve": (i32, [vp]),
            "ir_solve_bicgstab": (i32, [vp, vp, vp, P(Term), P(KrylovOpts), vp, P(_Report), vp]),
            "ir_residual": (i32, [vp, i64, i32, vp, i64, vp, vp, vp, vp, vp]),
            "ir_batch_create": (i32, [vp, i64, vp, vp, vp, vp, vp, P(Opts), P(Term), P(vp)]),
            "ir_batch_run": (i32, [vp, vp, vp]),
            "ir_batch_run_escalate": (i32, [vp, i32, ctypes.c_double, vp, vp]),
            "ir_batch_destroy": (None, [vp]),
            "ir_factor_solve_batched": (i32, [vp, i64, vp, vp, vp, vp, vp, P(Opts), P(Term), vp, vp]),
            "ir_fact_pivots": (i32, [vp, vp]),
            "ir_fact_schedule": (i32, [vp, P(i32), P(i32), P(i32)]),
            "ir_batch_schedule": (i32, [vp, P(i32), P(i32)]),
            "ir_fact_factors": (i32, [vp, vp, i64]),
            "ir_fact_info": (i32, [vp, P(i64), P(i32)]),
            "ir_fact_destroy": (None, [vp]),
            "ir_strerror": (ctypes.c_char_p, [i32]),
            "ir_last_error": (ctypes.c_char_p, []),
            "ir_kernel_launches": (ctypes.c_ulonglong, []),
            "ir_profile_start": (None, []),
            "ir_profile_stop": (i32, [vp, vp, i32]),
            "ir_profile_kind": (ctypes.c_char_p, [i32]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code: int):
    if code != 0:
        L = lib()
        raise IRError(code, f"{L.ir_strerror(code).decode()} ({L.ir_last_error().decode()})")


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _tw_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"working precision must be float64 or float32, got {t.dtype}")


def as_colmajor(A: torch.Tensor):
    """(tensor, lda) with column-major storage; copies only when needed."""
    if A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be square")
    n = A.shape[0]
    if n <= 1 or (A.stride(0) == 1 and A.stride(1) >= n):
        return A, max(A.stride(1) if n > 1 else 1, 1)
    F = A.t().contiguous().t()
    return F, max(n, 1)


def default_term(**kw) -> Term:
    t = Term()
    lib().ir_default_term(ctypes.byref(t))
    for k, v in kw.items():
        setattr(t, k, v)
    return t


def krylov_opts(**kw) -> KrylovOpts:
    """ir_krylov_opts with the defaults (basissize 10, eta 1e-8, Rmax_r 1) and overrides."""
    k = KrylovOpts()
    lib().ir_default_krylov_opts(ctypes.byref(k))
    for name, v in kw.items():
        setattr(k, name, v)
    return k


def make_opts(TW: int, TF: int, fp16_scale: bool = True, nb: int = 0, autotune: bool = False,
              group: int = 0, onthefly: bool = False, store_tf: bool = False) -> Opts:
    o = Opts()
    lib().ir_default_opts(ctypes.byref(o))
    o.TW, o.TF, o.TR, o.fp16_scale, o.nb, o.autotune = TW, TF, F64, int(fp16_scale), nb, int(autotune)
    o.group = int(group)
    o.onthefly = int(onthefly)
    o.store_tf = int(store_tf)
    return o


def _report(r: _Report) -> Report:
    k = r.iters
    return Report(iters=k, status=STATUS.get(r.status, str(r.status)),
                  rhist=list(r.rhist[: k + 1]), dhist=list(r.dhist[:k]), info=r.info, scale=r.scale)


class Context:
    """ir_ctx: one per device."""

    def __init__(self, device: int = 0):
        self._h = ctypes.c_void_p()
        _check(lib().ir_init(device, ctypes.byref(self._h)))
        self.device = device

    def close(self):
        if self._h:
            lib().ir_finalize(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def factor(self, A: torch.Tensor, tf="f32", fp16_scale: bool = True, nb: int = 0,
               stream=None, autotune: bool = False, group: int = 0, onthefly: bool = False,
               store_tf: bool = False) -> "Factorization":
        """mplu (Sec. 2.4): onthefly = True selects the mixed precision solves of Sec. 5.3;
        store_tf = True keeps binary16 / bfloat16 factors in 2 bytes (Sec. 1, 2.5)."""
        Ac, lda = as_colmajor(A)
        tfc = DTYPES[tf] if isinstance(tf, str) else int(tf)
        opts = make_opts(_tw_code(Ac), tfc, fp16_scale, nb, autotune, group, onthefly, store_tf)
        h = ctypes.c_void_p()
        _check(lib().ir_factor(self._h, Ac.shape[0], ctypes.c_void_p(Ac.data_ptr()), lda,
                               ctypes.byref(opts), _stream_ptr(stream), ctypes.byref(h)))
        return Factorization(self, h, Ac, lda, tfc)

    def residual(self, A: torch.Tensor, b: torch.Tensor, x: torch.Tensor, stream=None):
        """(r, ||r||_inf) with r = b - A x in binary64, computed on the device."""
        Ac, lda = as_colmajor(A)
        n = Ac.shape[0]
        x64 = x.to(torch.float64).contiguous()
        r = torch.empty(n, dtype=torch.float64, device=Ac.device)
        rn = torch.empty(1, dtype=torch.float64, device=Ac.device)
        bb = b.to(Ac.dtype).contiguous()
        _check(lib().ir_residual(self._h, n, _tw_code(Ac), ctypes.c_void_p(Ac.data_ptr()), lda,
                                 ctypes.c_void_p(bb.data_ptr()), ctypes.c_void_p(x64.data_ptr()),
                                 ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(rn.data_ptr()),
                                 _stream_ptr(stream)))
        return r, rn

    def solve_host(self, A_host: torch.Tensor, b_host: torch.Tensor, tf="f32", term=None,
                   fp16_scale: bool = True, stream=None, onthefly: bool = False):
        """End-to-end solve from host (CPU) tensors; returns (x_host, Report)."""
        if A_host.is_cuda or b_host.is_cuda:
            raise ValueError("solve_host takes CPU tensors")
        Ac, lda = as_colmajor(A_host)
        n = Ac.shape[0]
        bb = b_host.to(Ac.dtype).contiguous()
        x = torch.empty(n, dtype=Ac.dtype, pin_memory=Ac.is_pinned())
        tfc = DTYPES[tf] if isinstance(tf, str) else int(tf)
        opts = make_opts(_tw_code(Ac), tfc, fp16_scale, onthefly=onthefly)
        t = term if term is not None else default_term()
        rep = _Report()
        _check(lib().ir_solve_host(self._h, n, ctypes.c_void_p(Ac.data_ptr()), lda,
                                   ctypes.c_void_p(bb.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                   ctypes.byref(opts), ctypes.byref(t), _stream_ptr(stream),
                                   ctypes.byref(rep)))
        return x, _report(rep)


    def batch(self, As, bs, xs=None, tf="f16", term: Optional[Term] = None, fp16_scale: bool = True,
              autotune: bool = False):
        """Plan a batch of independent systems (ir_batch_create); see Batch."""
        return Batch(self, As, bs, xs, tf, term, fp16_scale, autotune=autotune)

    def solve_batched(self, As, bs, tf="f16", term: Optional[Term] = None, fp16_scale: bool = True,
                      stream=None):
        """One-shot batch (ir_factor_solve_batched): returns (xs, results)."""
        b = Batch(self, As, bs, None, tf, term, fp16_scale, plan=False)
        code = lib().ir_factor_solve_batched(self._h, b.count, b._n_arr, b._A_arr, b._lda_arr, b._b_arr,
                                             b._x_arr, ctypes.byref(b.opts), ctypes.byref(b.term),
                                             _stream_ptr(stream), ctypes.c_void_p(b.results_dev.data_ptr()))
        _check(code)
        return b.xs, b.results()


def _ptr_array(ts):
    arr = (ctypes.c_void_p * max(len(ts), 1))()
    for i, t in enumerate(ts):
        arr[i] = t.data_ptr() if t.numel() else None
    return arr


class Batch:
    """ir_batch: many independent systems solved by one persistent launch.

    As: list of square device tensors (TW = float64 or float32, all the same
    dtype, n_i <= 512); bs: right-hand sides; xs: solution buffers (allocated
    when None).  The plan borrows all of them.  run() enqueues the batch on a
    stream (no host synchronisation, capturable in a CUDA graph);
    results() reads the per-system outcomes after the stream has finished.
    """

    def __init__(self, ctx: Context, As, bs, xs=None, tf="f16", term: Optional[Term] = None,
                 fp16_scale: bool = True, plan: bool = True, autotune: bool = False):
        if len(As) != len(bs) or (xs is not None and len(xs) != len(As)):
            raise ValueError("As, bs and xs must have the same length")
        self.ctx, self.count = ctx, len(As)
        cols = [as_colmajor(A) for A in As]
        self.As = [c[0] for c in cols]
        tws = {_tw_code(A) for A in self.As}
        if len(tws) > 1:
            raise TypeError("all matrices of a batch need the same working precision")
        tw = tws.pop() if tws else F64
        dt = torch.float64 if tw == F64 else torch.float32
        dev = self.As[0].device if self.As else torch.device("cuda", ctx.device)
        self.bs = [b.to(device=dev, dtype=dt).contiguous() for b in bs]
        self.xs = list(xs) if xs is not None else [torch.empty_like(b) for b in self.bs]
        self.ns = [A.shape[0] for A in self.As]
        tfc = DTYPES[tf] if isinstance(tf, str) else int(tf)
        self.opts = make_opts(tw, tfc, fp16_scale, autotune=autotune)
        self.term = term if term is not None else default_term()
        self._n_arr = (ctypes.c_int64 * max(self.count, 1))(*self.ns)
        self._lda_arr = (ctypes.c_int64 * max(self.count, 1))(*[c[1] for c in cols])
        self._A_arr = _ptr_array(self.As)
        self._b_arr = _ptr_array(self.bs)
        self._x_arr = _ptr_array(self.xs)
        nbytes = ctypes.sizeof(BatchResult) * max(self.count, 1)
        self.results_dev = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
        self._h = ctypes.c_void_p()
        if plan:
            _check(lib().ir_batch_create(ctx._h, self.count, self._n_arr, self._A_arr, self._lda_arr,
                                         self._b_arr, self._x_arr, ctypes.byref(self.opts),
                                         ctypes.byref(self.term), ctypes.byref(self._h)))

    def schedule(self):
        """(grid, tc_min_trail) of the plan (ir_batch_schedule)."""
        g, t = ctypes.c_int(), ctypes.c_int()
        _check(lib().ir_batch_schedule(self._h, ctypes.byref(g), ctypes.byref(t)))
        return g.value, t.value

    def run(self, stream=None):
        _check(lib().ir_batch_run(self._h, ctypes.c_void_p(self.results_dev.data_ptr()), _stream_ptr(stream)))

    def run_escalate(self, tf2="f32", rtol: float = 1e-10, stream=None):
        """run(), then the members that neither converged nor stopped with ||r|| <= rtol ||b||
        again with TF = tf2 (ir_batch_run_escalate)."""
        t2 = DTYPES[tf2] if isinstance(tf2, str) else int(tf2)
        _check(lib().ir_batch_run_escalate(self._h, t2, ctypes.c_double(rtol),
                                           ctypes.c_void_p(self.results_dev.data_ptr()), _stream_ptr(stream)))

    def results(self):
        """Per-system outcomes as a list of dicts (synchronises the device)."""
        raw = bytes(self.results_dev.cpu().numpy().tobytes())
        arr = (BatchResult * max(self.count, 1)).from_buffer_copy(raw)
        out = []
        for i in range(self.count):
            r = arr[i]
            out.append({"status": STATUS.get(r.status, str(r.status)), "iters": r.iters, "info": r.info,
                        "nonfinite": bool(r.nonfinite), "timeout": bool(r.timeout), "rnorm": r.rnorm,
                        "scale": r.scale, "tf": r.tf, "bnorm": r.bnorm})
        return out

    def destroy(self):
        if self._h:
            lib().ir_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Factorization:
    """ir_fact: the rounded, factored copy of A (borrows A)."""

    def __init__(self, ctx: Context, h, A: torch.Tensor, lda: int, tf: int):
        self.ctx, self._h, self.A, self.lda, self.tf = ctx, h, A, lda, tf
        self.n = A.shape[0]

    def destroy(self):
        if self._h:
            lib().ir_fact_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def refactor(self, B: torch.Tensor, stream=None):
        Bc, ldb = as_colmajor(B)
        if Bc.shape[0] != self.n or Bc.dtype != self.A.dtype:
            raise ValueError("refactor needs a matrix of the same size and type")
        _check(lib().ir_refactor(self._h, ctypes.c_void_p(Bc.data_ptr()), ldb, _stream_ptr(stream)))
        self.A, self.lda = Bc, ldb

    def solve(self, b: torch.Tensor, x: Optional[torch.Tensor] = None, term: Optional[Term] = None,
              stream=None, report: bool = True):
        bb = b.to(self.A.dtype).contiguous()
        if x is None:
            x = torch.empty_like(bb)
        rep = _Report()
        t = term if term is not None else default_term()
        code = lib().ir_solve(self._h, ctypes.c_void_p(bb.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                              ctypes.byref(t), _stream_ptr(stream), ctypes.byref(rep) if report else None)
        R = _report(rep) if report else None
        if code != 0:
            L = lib()
            err = IRError(code, f"{L.ir_strerror(code).decode()} ({L.ir_last_error().decode()})")
            err.report = R
            raise err
        return x, R

    def solve_many(self, B: torch.Tensor, term: Optional[Term] = None, stream=None):
        """X = A^{-1} B for the columns of B (n x nrhs), each refined by its own IR loop
        (ir_solve_many); returns (X column-major, [Report])."""
        if B.dim() != 2 or B.shape[0] != self.n:
            raise ValueError("B must be n x nrhs")
        Bc = B.to(self.A.dtype).t().contiguous().t()         # column-major, ldb = n
        ldb = max(self.n, 1)
        nrhs = Bc.shape[1]
        X = torch.empty((nrhs, self.n), dtype=self.A.dtype, device=Bc.device).t()
        reps = (_Report * max(nrhs, 1))()
        t = term if term is not None else default_term()
        _check(lib().ir_solve_many(self._h, nrhs, ctypes.c_void_p(Bc.data_ptr()), ldb, ctypes.c_void_p(X.data_ptr()),
                                   max(self.n, 1), ctypes.byref(t), _stream_ptr(stream), reps))
        return X, [_report(reps[j]) for j in range(nrhs)]

    def gmres_reserve(self, basissize: int = 10):
        """Reserve the Krylov basis (mpglu's allocation, Sec. 4.4)."""
        _check(lib().ir_gmres_reserve(self._h, int(basissize)))

    def bicgstab_reserve(self):
        """Reserve the BiCGSTAB vectors (mpblu's allocation, Sec. 4.4)."""
        _check(lib().ir_bicgstab_reserve(self._h))

    def solve_gmres(self, b: torch.Tensor, x: Optional[torch.Tensor] = None, term: Optional[Term] = None,
                    kopts: Optional[KrylovOpts] = None, stream=None, report: bool = True):
        """GMRES-IR (Sec. 4.3): returns (x, Report with khist)."""
        return self._krylov(lib().ir_solve_gmres, b, x, term, kopts, stream, report)

    def solve_bicgstab(self, b: torch.Tensor, x: Optional[torch.Tensor] = None, term: Optional[Term] = None,
                       kopts: Optional[KrylovOpts] = None, stream=None, report: bool = True):
        """BiCGSTAB-IR (Sec. 2.3, 4.2): returns (x, Report with khist)."""
        return self._krylov(lib().ir_solve_bicgstab, b, x, term, kopts, stream, report)

    def _krylov(self, fn, b, x, term, kopts, stream, report):
        bb = b.to(self.A.dtype).contiguous()
        if x is None:
            x = torch.empty_like(bb)
        rep = _Report()
        kh = (ctypes.c_int * MAX_HIST)()
        t = term if term is not None else default_term()
        ko = kopts if kopts is not None else krylov_opts()
        code = fn(self._h, ctypes.c_void_p(bb.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                  ctypes.byref(t), ctypes.byref(ko), _stream_ptr(stream),
                  ctypes.byref(rep) if report else None, kh)
        R = _report(rep) if report else None
        if R is not None:
            R.khist = list(kh[: R.iters])
        if code != 0:
            L = lib()
            err = IRError(code, f"{L.ir_strerror(code).decode()} ({L.ir_last_error().decode()})")
            err.report = R
            raise err
        return x, R

    def schedule(self):
        """(nb, panel_reserve_sms, group) of the factorization (ir_fact_schedule)."""
        nb, r, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().ir_fact_schedule(self._h, ctypes.byref(nb), ctypes.byref(r), ctypes.byref(g)))
        return nb.value, r.value, g.value

    def lu_solve(self, v: torch.Tensor, stream=None) -> torch.Tensor:
        """d = U^{-1} L^{-1} P v in binary32."""
        vv = v.to(torch.float32).contiguous()
        d = torch.empty_like(vv)
        _check(lib().ir_lu_solve(self._h, ctypes.c_void_p(vv.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                 _stream_ptr(stream)))
        return d

    def check_wait_timeout(self, limit_s: float, stream=None) -> int:
        """ir_check_wait_timeout: the solves' bounded wait on a value nobody writes,
        limited to limit_s seconds; returns the status code (6 = IR_ETIMEOUT expected)."""
        return int(lib().ir_check_wait_timeout(self._h, ctypes.c_double(limit_s), _stream_ptr(stream)))

    def pivots(self):
        import numpy as np
        out = np.zeros(self.n, dtype=np.int32)
        _check(lib().ir_fact_pivots(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def factors(self):
        """P A_F = L U as one column-major binary32 array (L strictly below the diagonal)."""
        import numpy as np
        out = np.zeros((self.n, self.n), dtype=np.float32, order="F")
        _check(lib().ir_fact_factors(self._h, out.ctypes.data_as(ctypes.c_void_p), max(self.n, 1)))
        return out

    def info(self):
        info = ctypes.c_int64()
        nf = ctypes.c_int()
        _check(lib().ir_fact_info(self._h, ctypes.byref(info), ctypes.byref(nf)))
        return int(info.value), bool(nf.value)


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(lib().ir_kernel_launches())


def profile_start():
    lib().ir_profile_start()


def profile_stop():
    """{kind: (total_ms, calls)} for the launcher calls since profile_start()."""
    ms = (ctypes.c_double * 32)()
    cnt = (ctypes.c_int * 32)()
    k = lib().ir_profile_stop(ms, cnt, 32)
    if k < 0:
        raise IRError(3, "profile_stop: CUDA error")
    return {lib().ir_profile_kind(i).decode(): (ms[i], cnt[i]) for i in range(k) if cnt[i]}
