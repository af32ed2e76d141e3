"""A CPU model of the cluster solve's tile bookkeeping.  In the cluster
kernel one thread of each CTA issues the TMA loads of the CTA's 128 x 128
factor tiles in advance, walking a tile sequence (first / next), while the
whole CTA consumes tiles in the order of its two solve loops; a tile buffer
is valid only if the two orders agree.  The model walks both, as the kernel
states them, for every block count the cluster path takes (1 .. 32 blocks of
128 rows, clusters of min(blocks, 16) CTAs, CTA c owning blocks c and
c + 16), and checks that they agree and cover exactly the tiles the
triangular solves need."""
import pytest

K_CTAS = 16


def _own(c, C, o):
    return c + o * C


def _seq_first_upper(c, C, nown, nblk):
    bj = nblk - 1
    o = 1 if (nown > 1 and _own(c, C, 1) < bj) else (0 if _own(c, C, 0) < bj else -1)
    return (1, o, bj) if o >= 0 else (2, o, bj)


def _seq_first(c, C, nown, nblk):
    o = 0 if _own(c, C, 0) > 0 else (1 if (nown > 1 and _own(c, C, 1) > 0) else -1)
    if o < 0:
        return _seq_first_upper(c, C, nown, nblk)
    return (0, o, 0)


def _seq_next(q, c, C, nown, nblk):
    ph, o, bj = q
    if ph == 0:
        if o == 0 and nown > 1 and _own(c, C, 1) > bj:
            return (0, 1, bj)
        bj += 1
        o = 0 if _own(c, C, 0) > bj else (1 if (nown > 1 and _own(c, C, 1) > bj) else -1)
        if o < 0:
            return _seq_first_upper(c, C, nown, nblk)
        return (0, o, bj)
    if ph == 1:
        if o == 1 and _own(c, C, 0) < bj:
            return (1, 0, bj)
        bj -= 1
        o = 1 if (nown > 1 and _own(c, C, 1) < bj) else (0 if _own(c, C, 0) < bj else -1)
        return (1, o, bj) if o >= 0 else (2, o, bj)
    return q


def _producer(c, C, nown, nblk):
    """(row block, column block) of every tile the producer loads, in order."""
    out, q = [], _seq_first(c, C, nown, nblk)
    while q[0] < 2:
        out.append((_own(c, C, q[1]), q[2]))
        q = _seq_next(q, c, C, nown, nblk)
        assert len(out) <= 4 * nblk
    return out


def _consumer(c, C, nown, nblk):
    """The tiles in the order the two solve loops apply them."""
    out = []
    for bj in range(nblk - 1):                         # lower: blocks ascending
        if _own(c, C, nown - 1) <= bj:
            break
        for o in range(2):
            if o >= nown or _own(c, C, o) <= bj:
                continue
            out.append((_own(c, C, o), bj))
    for bj in range(nblk - 1, 0, -1):                  # upper: blocks descending
        if _own(c, C, 0) >= bj:
            break
        for oo in range(2):
            o = 1 - oo                                  # the higher block first
            if o >= nown or _own(c, C, o) >= bj:
                continue
            out.append((_own(c, C, o), bj))
    return out


@pytest.mark.parametrize("nblk", list(range(1, 2 * K_CTAS + 1)))
def test_prefetch_order_is_the_apply_order(nblk):
    C = min(nblk, K_CTAS)
    lower, upper, applied = set(), set(), []
    for c in range(C):
        nown = 2 if _own(c, C, 1) < nblk else 1
        prod, cons = _producer(c, C, nown, nblk), _consumer(c, C, nown, nblk)
        assert prod == cons, (c, prod, cons)
        applied += cons
        for (bi, bj) in cons:
            (lower if bi > bj else upper).add((bi, bj))
    assert len(applied) == len(set(applied))
    # together the CTAs apply every off-diagonal tile of L and of U exactly once
    want_lower = {(i, j) for i in range(nblk) for j in range(i)}
    assert lower == want_lower
    assert upper == {(j, i) for (i, j) in want_lower}
