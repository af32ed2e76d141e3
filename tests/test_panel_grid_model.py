"""A CPU model of the exchange of a panel taller than one cluster (the
cooperative launch of k_panel for n > 8192): C CTAs, per column k each writes
its best record into slot [k & 1][its rank] of global memory, arrives on the
column's counter, waits until all C have arrived, then reads every slot
[k & 1][*] and updates before staging column k + 1.  Run under seeded
interleavings, the model checks that every CTA reads the records of the
column it is on (never one a faster CTA has already overwritten with column
k + 2) and that no interleaving stalls."""
import numpy as np
import pytest


def run_exchange(C, ncols, seed):
    rng = np.random.default_rng(seed)
    slot = [[None] * C for _ in range(2)]       # (column, writer) held by each record slot
    count = [0] * ncols
    # per CTA: phase 0 write + arrive, 1 wait, 2 read + update, then the next column
    st = [dict(k=0, ph=0) for _ in range(C)]
    reads_ok = True
    def can(r):
        s = st[r]
        return s["k"] < ncols and (s["ph"] != 1 or count[s["k"]] == C)

    while True:
        ready = [r for r in range(C) if can(r)]
        if not ready:
            break
        r = ready[rng.integers(len(ready))]          # one CTA moves; the others may lag any amount
        s = st[r]
        k = s["k"]
        if s["ph"] == 0:
            slot[k & 1][r] = (k, r)
            count[k] += 1
            s["ph"] = 1
        elif s["ph"] == 1:
            s["ph"] = 2
        else:
            # the headers and the winner's record of column k
            if any(slot[k & 1][q] != (k, q) for q in range(C)):
                reads_ok = False
            s["k"] += 1
            s["ph"] = 0
    finished = all(s["k"] == ncols for s in st)
    return finished, reads_ok


@pytest.mark.parametrize("C", [17, 40, 152])
def test_two_slots_by_column_parity_suffice(C):
    for seed in range(6):
        finished, reads_ok = run_exchange(C, 64, seed)
        assert finished and reads_ok, (C, seed)


def test_one_slot_would_not():
    """With a single slot per CTA a fast CTA overwrites a record a slow one
    has yet to read (the model is sensitive to the hazard it rules out)."""
    rng_bad = False
    for seed in range(10):
        C, ncols = 17, 64
        rng = np.random.default_rng(seed)
        slot = [None] * C
        count = [0] * ncols
        st = [dict(k=0, ph=0) for _ in range(C)]
        while True:
            ready = [r for r in range(C) if st[r]["k"] < ncols and (st[r]["ph"] != 1 or count[st[r]["k"]] == C)]
            if not ready:
                break
            r = ready[rng.integers(len(ready))]
            s = st[r]
            k = s["k"]
            if s["ph"] == 0:
                slot[r] = (k, r)
                count[k] += 1
                s["ph"] = 1
            elif s["ph"] == 1:
                s["ph"] = 2
            else:
                rng_bad |= any(slot[q] != (k, q) for q in range(C))
                s["k"], s["ph"] = k + 1, 0
    assert rng_bad
