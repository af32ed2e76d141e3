"""A CPU model of the group-U12 kernel's pipeline protocol (k_u12_group_tc):
the TMA producer, the MMA issuer, and two epilogue warpgroups that take the
group's block rows in turn, synchronised by a ring of operand stages, a ring
of 8 TMEM accumulators (one per block pair) and the in-order publication of
each block's U.  Every role advances only when the barrier it waits on would
let it; the model runs the roles in every interleaving a seeded scheduler
picks and checks that all of them finish (no circular wait), that each
accumulator is read only after its product and overwritten only after it was
read, and that a block's U is published before any product that needs it."""
import numpy as np
import pytest

ACC = 8


def run_model(G, stages, seed):
    pairs = [(c, a) for c in range(1, G) for a in range(c)]
    qa_of = {p: i for i, p in enumerate(pairs)}
    rng = np.random.default_rng(seed)
    published = set()                 # blocks whose U is out
    stage_full = [None] * stages      # pair loaded into each stage
    acc = [None] * ACC                # pair whose product sits in each accumulator (None: free)
    acc_read = set()                  # pairs whose accumulator was read
    prod_i = mma_i = 0
    epi = [dict(rows=list(range(e, G, 2)), r=0, a=0) for e in range(2)]

    def producer():
        nonlocal prod_i
        if prod_i >= len(pairs):
            return False
        c, a = pairs[prod_i]
        s = prod_i % stages
        if a not in published or stage_full[s] is not None:
            return False
        stage_full[s] = (c, a)
        prod_i += 1
        return True

    def mma():
        nonlocal mma_i
        if mma_i >= len(pairs):
            return False
        p = pairs[mma_i]
        s, slot = mma_i % stages, mma_i % ACC
        if stage_full[s] != p or acc[slot] is not None:
            return False
        assert p[1] in published                     # U_a is out before its product
        acc[slot] = p
        stage_full[s] = None                          # the stage is free again
        mma_i += 1
        return True

    def epilogue(e):
        st = epi[e]
        if st["r"] >= len(st["rows"]):
            return False
        c = st["rows"][st["r"]]
        if st["a"] < c:
            p = (c, st["a"])
            slot = qa_of[p] % ACC
            if acc[slot] != p:
                return False                          # product not there yet
            acc_read.add(p)
            acc[slot] = None                          # released
            st["a"] += 1
            return True
        published.add(c)                              # solved and published
        st["r"] += 1
        st["a"] = 0
        return True

    roles = [producer, mma, lambda: epilogue(0), lambda: epilogue(1)]
    while True:
        order = rng.permutation(len(roles))
        if not any(roles[i]() for i in order):
            break
    done = prod_i == len(pairs) and mma_i == len(pairs) and all(st["r"] == len(st["rows"]) for st in epi)
    return done, published, acc_read, pairs


@pytest.mark.parametrize("G", list(range(1, 17)))
@pytest.mark.parametrize("stages", [2, 3, 4])
def test_u12_pipeline_never_waits_in_a_circle(G, stages):
    for seed in range(5):
        done, published, acc_read, pairs = run_model(G, stages, seed + 100 * G)
        assert done, (G, stages, seed)
        assert published == set(range(G))
        assert acc_read == set(pairs)
