"""A CPU model of the panel kernel's algorithm (not of its arithmetic): rows
stay in place and carry position labels, every row holds a window of the
panel that shifts left by one column per step, the pivot row travels as a
record, and the rank-1 update stops at the first 16-column chunk past the
live width, so window entries past it go stale; the record carries only the
header and the live part of the row (16-byte chunks: 17 at the first column,
one fewer every four), so the receivers see stale values past it.  The model
checks the invariants the kernel relies on: the stale entries are never read,
and the labels give LAPACK's interchanges.  fmaf is emulated in binary64 (the product
of two binary32 values is exact there); the same emulation serves every
variant, so variants are compared bit for bit and the model is compared with
the oracle's binary32 LU through its pivots and to a tight tolerance."""
import numpy as np
import pytest

import irgen
import oracle as O

NB = 64


def _fmaf(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def panel_model(P, chunked, live_records=False):
    """Factor the M x nbp panel P (binary32); returns (factors in final row
    order, ipiv) as the kernel writes them.  live_records: the pivot record
    keeps only its first (70 - k) // 4 chunks of 4 (header: |a|, position,
    1/a; then a[0], a[1], ...), everything past them arrives as NaN."""
    M, nbp = P.shape
    a = np.zeros((M, NB), np.float32)
    a[:, :nbp] = P
    pos = np.arange(M)              # current position of each row (rows never move)
    kp = np.full(M, nbp)            # step at which the row became the pivot row (nbp: never)
    Ls = np.zeros((M, NB), np.float32)
    Us = np.zeros((NB, NB), np.float32)
    ipiv = np.zeros(nbp, np.int64)
    for k in range(nbp):
        cand = kp == nbp
        key = np.where(cand, np.abs(a[:, 0]), -1.0)
        best = np.flatnonzero(cand & (key == key.max()))
        w = best[np.argmin(pos[best])]                   # ties: lowest current position
        ppos = pos[w]
        u = a[w].copy()                                  # the pivot row's record
        if live_records:
            nch = (70 - k) // 4                          # chunks sent at step k
            u[4 * nch - 3:] = np.nan                     # record float 3 + i holds a[i]
        ipiv[k] = ppos
        piv = u[0]
        r = np.float32(1.0) / piv
        swap_in = pos == k
        pos[w], kp[w] = k, k
        pos[swap_in & (np.arange(M) != w)] = ppos        # interchange of positions k and ppos
        Us[k] = u
        live = kp == nbp
        l = np.where(live, a[:, 0] * r, np.float32(0)).astype(np.float32)
        Ls[live, k] = l[live]
        new = a.copy()
        for q in range(NB // 4):
            if chunked and q % 4 == 0 and q > 0 and 4 * q >= NB - 1 - k:
                break                                    # this and later chunks hold no live entry
            for i in range(4 * q, 4 * q + 4):
                new[:, i] = _fmaf(-l, np.full(M, u[i + 1], np.float32), a[:, i + 1]) if i < NB - 1 else 0
        a = new
    out = np.zeros((M, nbp), np.float32)
    for s in range(M):
        for c in range(nbp):
            out[pos[s], c] = Ls[s, c] if c < kp[s] else Us[kp[s], c - kp[s]]
    return out, ipiv


@pytest.mark.parametrize("M,nbp,seed", [(64, 64, 0), (200, 64, 1), (97, 44, 2), (80, 20, 3), (70, 1, 4), (130, 64, 5)])
def test_chunked_update_reads_no_stale_entry(M, nbp, seed):
    P = np.random.default_rng(seed).standard_normal((M, nbp)).astype(np.float32)
    full, piv_full = panel_model(P, chunked=False)
    chunk, piv_chunk = panel_model(P, chunked=True)
    assert np.array_equal(piv_full, piv_chunk)
    assert np.array_equal(full.view(np.uint32), chunk.view(np.uint32))


@pytest.mark.parametrize("M,nbp,seed", [(64, 64, 6), (300, 64, 7), (97, 44, 8), (70, 1, 9), (513, 64, 10)])
def test_live_records_carry_every_value_that_is_read(M, nbp, seed):
    """Sending only the live part of the pivot row (the rest arrives as NaN)
    gives the same factors and pivots, bit for bit."""
    P = np.random.default_rng(seed).standard_normal((M, nbp)).astype(np.float32)
    full, piv_full = panel_model(P, chunked=True)
    live, piv_live = panel_model(P, chunked=True, live_records=True)
    assert np.array_equal(piv_full, piv_live)
    assert not np.isnan(live).any()
    assert np.array_equal(full.view(np.uint32), live.view(np.uint32))


@pytest.mark.parametrize("n", [40, 64, 100])
def test_labels_give_lapack_interchanges(n):
    """One panel of a square matrix (n <= 64 columns are one panel; n > 64: the
    first 64 columns): the model's interchanges are the oracle's binary32 LU's,
    and its factors agree with the oracle's to rounding."""
    A, _ = irgen.case_random(n, 900 + n)
    AF = O.cast(A, O.F32)
    nbp = min(n, NB)
    F, ipiv = panel_model(np.ascontiguousarray(AF[:, :nbp]), chunked=True)
    LU, ipiv_o, _ = O.getrf_tf(AF, O.F32)
    assert list(ipiv) == list(ipiv_o[:nbp])
    ref = LU[:, :nbp] if n <= NB else None
    if ref is not None:
        assert np.max(np.abs(F - ref)) <= 64 * 2.0 ** -23 * max(1.0, np.max(np.abs(ref)))


def test_tie_goes_to_the_lowest_current_position():
    P = np.array([[1.0, 2.0], [-3.0, 1.0], [3.0, 5.0], [2.0, 2.0]], np.float32)
    _, ipiv = panel_model(P, chunked=True)
    assert ipiv[0] == 1          # |-3| = |3|: the row at position 1 wins
