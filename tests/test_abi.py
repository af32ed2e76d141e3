"""The C-ABI library builds, loads and exports every function include/ir.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "ir.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ir_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("ir_init", "ir_factor", "ir_refactor", "ir_solve", "ir_solve_host", "ir_lu_solve",
                 "ir_residual", "ir_fact_pivots", "ir_fact_factors", "ir_fact_destroy", "ir_finalize",
                 "ir_gmres_reserve", "ir_solve_gmres", "ir_default_krylov_opts", "ir_solve_bicgstab",
                 "ir_bicgstab_reserve", "ir_fact_schedule", "ir_batch_schedule", "ir_solve_many", "ir_batch_run_escalate",
                 "ir_check_wait_timeout"):
        assert must in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2311_14616_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)          # loads without a GPU (the runtime binds lazily)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_defaults_and_strerror_without_gpu():
    from paper_2311_14616_gb300 import ir
    t = ir.default_term()
    assert (t.Cr, t.Ce, t.Rmax, t.litmax) == (1.0, 1.0, 0.5, 10)
    o = ir.make_opts(ir.F64, ir.F32)
    assert (o.TW, o.TF, o.TR, o.fp16_scale) == (ir.F64, ir.F32, ir.F64, 1)
    assert ir.lib().ir_strerror(4) == b"zero pivot in the factorization"
    k = ir.krylov_opts()
    assert (k.basissize, k.eta, k.Rmax_r) == (10, 1e-8, 1.0)
    assert ctypes.sizeof(ir.KrylovOpts) == 24


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2311_14616_gb300 import ir
    monkeypatch.setattr(ir, "_lib", None)
    monkeypatch.setattr(ir, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="not built"):
        ir.lib()
