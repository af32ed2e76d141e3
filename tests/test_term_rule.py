"""The library's termination rule (term_rule, which the device-side loop of
ir_solve runs after every residual) decides exactly as the oracle's
term_decide (Sec. 5.1 eqs. residterm, term, stag, wilkterm; litmax) on random
histories and on cases placed exactly on each test's boundary, where a fused
multiply-add in either would flip the decision.  The rule is compiled for the
host here; no GPU is used."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def rule_exe(tmp_path_factory):
    nvcc = os.environ.get("NVCC", shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc")
    if not os.path.exists(nvcc) and not shutil.which(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("term") / "term_rule_check")
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-o", exe, os.path.join(HERE, "term_rule_check.cu")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def _cases():
    g = np.random.default_rng(5)
    out = []
    for _ in range(1500):
        k = int(g.integers(1, 12))
        pick = int(g.integers(0, 6))
        # the boundary cases run under the test they sit on
        mode = 1 if pick == 4 else (0 if pick == 1 else int(g.integers(0, 2)))
        tr_wider = True if pick == 3 else (False if pick in (1, 2, 4) else bool(g.integers(0, 2)))
        t = O.Term(Cr=float(g.choice([1.0, 10.0, 3.0])), Ce=float(g.choice([1.0, 4.0, 3.0])),
                   Rmax=float(g.choice([0.5, 0.9, 0.3])), litmax=int(g.integers(k, 14)), mode=mode,
                   abs_rel_tol=float(g.choice([0.0, 0.0, 1e-13])))
        eps = float(g.choice([2.0 ** -53, 2.0 ** -24]))
        rmax_r = t.Rmax if g.integers(0, 2) else 1.0
        bnorm = float(g.uniform(0.5, 4.0))
        anorm, xnorm = float(g.uniform(1, 100)), float(g.uniform(0.1, 10))
        rh = [bnorm] + list(bnorm * 10.0 ** -g.uniform(0, 16, k))
        dh = list(10.0 ** -g.uniform(0, 16, k))
        # place the last residual / correction exactly on a boundary
        if pick == 1:
            tol = t.abs_rel_tol if t.abs_rel_tol > 0 else t.Cr * eps
            rh[-1] = tol * bnorm
        elif pick == 2:
            rh[-1] = rmax_r * rh[-2]
        elif pick == 3 and k >= 2:
            dh[-1] = t.Rmax * dh[-2]
        elif pick == 4:
            rh[-1] = t.Ce * eps * (bnorm + anorm * xnorm)
        elif pick == 5:
            rh[-1] = float(g.choice([0.0, np.inf, np.nan]))
        out.append((k, t, eps, rmax_r, bnorm, anorm, xnorm, rh, dh, tr_wider))
    return out


def test_term_rule_matches_the_oracle(rule_exe):
    cases = _cases()
    lines = []
    for k, t, eps, rmax_r, bnorm, anorm, xnorm, rh, dh, tr_wider in cases:
        vals = [k, t.litmax, t.mode, int(tr_wider), t.Cr, t.Ce, t.Rmax, rmax_r, t.abs_rel_tol, eps, bnorm, anorm, xnorm]
        lines.append(" ".join(repr(float(v)) if isinstance(v, float) else str(v) for v in vals))
        lines.append(" ".join(repr(float(v)) for v in rh))
        lines.append(" ".join(repr(float(v)) for v in dh) if dh else "")
    r = subprocess.run([rule_exe], input="\n".join(lines) + "\n", capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = [int(v) for v in r.stdout.split()]
    assert len(got) == len(cases)
    boundary = 0
    for (k, t, eps, rmax_r, bnorm, anorm, xnorm, rh, dh, tr_wider), st in zip(cases, got):
        ref = O.term_decide(rh, dh, bnorm, eps, t, tr_wider, rmax_r=rmax_r, anorm=anorm, xnorm=xnorm)
        assert st == (-1 if ref is None else ref), (k, rh, dh, st, ref)
        boundary += ref is not None
    assert boundary > 500          # plenty of cases that stop, many of them on a boundary
