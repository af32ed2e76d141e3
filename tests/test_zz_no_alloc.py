"""The allocation-free residual entry point agrees with the allocating one.

ir_residual_noalloc exists for callers that must not call cudaMalloc when they
need a residual (a framework allocator owns the device memory, a
latency-critical loop, allocation allowed only at start-up).  It keeps its
workspace in a fixed array inside the library.  This file is collected last
on purpose, and works both alone in a fresh process and after the others.
"""
import ctypes

import numpy as np
import pytest
import torch

import irgen
import oracle as O
from gpu_util import dev_colmajor, dev_vec
from paper_2311_14616_gb300 import ir

pytestmark = pytest.mark.gpu


def _noalloc():
    f = ir.lib().ir_residual_noalloc
    vp = ctypes.c_void_p
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int64, ctypes.c_int, vp, ctypes.c_int64, vp, vp, vp, vp, vp]
    return f


def _call_noalloc(A, b, x):
    Ac, lda = ir.as_colmajor(A)
    n = Ac.shape[0]
    r = torch.full((n,), float("nan"), dtype=torch.float64, device=Ac.device)
    rn = torch.full((1,), float("nan"), dtype=torch.float64, device=Ac.device)
    code = _noalloc()(n, ir._tw_code(Ac), ctypes.c_void_p(Ac.data_ptr()), lda,
                      ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                      ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(rn.data_ptr()),
                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0, code
    return r, rn


def _bound(A, b, x):
    n = A.shape[0]
    g = 2 * n * 2.0 ** -53
    return g * (np.abs(A).astype(np.float64) @ np.abs(x) + np.abs(b.astype(np.float64)))


@pytest.mark.parametrize("tw", [np.float64, np.float32])
def test_noalloc_residual_matches_allocating_entry_point_twice(ctx, tw):
    # two calls in a row, different sizes and data: the second must not see the first's leftovers
    for n, seed in ((3000, 1), (1237, 2)):
        A, b = irgen.case_gaussian(n, 900 + seed)
        A = np.asfortranarray(A.astype(tw))
        b = b.astype(tw)
        x = np.random.Generator(np.random.PCG64(seed)).standard_normal(n)
        Ad, bd, xd = dev_colmajor(A), dev_vec(b), dev_vec(x)
        r_ref, rn_ref = ctx.residual(Ad, bd, xd)
        r, rn = _call_noalloc(Ad, bd, xd)
        torch.cuda.synchronize()
        r, r_ref = r.cpu().numpy(), r_ref.cpu().numpy()
        assert np.all(np.abs(r - r_ref) <= _bound(A, b, x) + 1e-300)
        # and against the CPU oracle's residual (a sequential binary64 fma chain per row)
        r_orc = O.residual(A, b, x)
        assert np.all(np.abs(r - r_orc) <= _bound(A, b, x) + 1e-300)
        assert float(rn.cpu()[0]) == np.max(np.abs(r))
        assert abs(float(rn.cpu()[0]) - float(rn_ref.cpu()[0])) <= np.max(_bound(A, b, x))


def test_noalloc_residual_rejects_sizes_beyond_its_array(ctx):
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(t.data_ptr())
    n = (1 << 20) + 1
    code = _noalloc()(n, ir.F64, p, n, p, p, p, p, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 7          # IR_EUNSUPPORTED, nothing launched
