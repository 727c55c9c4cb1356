"""The reading behind the GPU's balanced-split build, checked on the CPU: ADS+
insertion (series added one by one in row order, a leaf split on its most
balanced segment when it first overflows: the oracle's tree) gives the same
leaves as a level-by-level bulk construction in which every node over capacity
decides its segment on its first leaf_size + 1 series in row order and is then
partitioned stably by that segment's next bit.  The bulk construction here is
plain numpy over the oracle's FP64 symbols, independent of the GPU code."""
import numpy as np
import pytest

import datagen
import oracle


def bulk_leaves(S, card, cap):
    """Leaves (ids in depth-first order, sizes including empty leaves) of the
    level-by-level construction."""
    cbits = card.bit_length() - 1
    root = np.zeros(len(S), np.int64)
    for i in range(16):
        root = (root << 1) | ((S[:, i] >> (cbits - 1)) & 1)
    order = np.argsort(root, kind="stable")
    # a node: (ids in row order, bits taken per segment)
    nodes = [(order[root[order] == r], np.ones(16, np.int64)) for r in np.unique(root)]
    while True:
        nxt, split_any = [], False
        for ids, bits in nodes:
            if len(ids) <= cap or (bits >= cbits).all():
                nxt.append((ids, bits))
                continue
            first = S[ids[:cap + 1]]
            best, best_bal = -1, None
            for g in range(16):
                if bits[g] >= cbits:
                    continue
                ones = int(((first[:, g] >> (cbits - 1 - bits[g])) & 1).sum())
                bal = abs(2 * ones - (cap + 1))
                if best < 0 or bal < best_bal:
                    best, best_bal = g, bal
            bit = (S[ids, best] >> (cbits - 1 - bits[best])) & 1
            nb = bits.copy()
            nb[best] += 1
            nxt += [(ids[bit == 0], nb), (ids[bit == 1], nb)]
            split_any = True
        nodes = nxt
        if not split_any:
            break
    return (np.concatenate([ids for ids, _ in nodes]), np.array([len(ids) for ids, _ in nodes]))


@pytest.mark.parametrize("kind,N,n,card,cap,dup", [
    ("walk", 3000, 64, 256, 20, False), ("walk", 2000, 64, 16, 7, True), ("sine", 3000, 128, 256, 50, False),
    ("walk", 500, 32, 4, 1, True), ("walk", 3000, 256, 256, 100, True), ("walk", 20000, 256, 256, 40, False)])
def test_bulk_levels_equal_insertion_order(kind, N, n, card, cap, dup):
    X = datagen.rows(kind, 11, 0, N, n)
    if dup:
        X[N // 3: N // 3 + 2 * cap + 3] = X[0]
    _, S = oracle.summarize(X, card=card)
    ids, sizes = bulk_leaves(S.astype(np.int64), card, cap)
    ix = oracle.ISAXIndex(X, card=card, leaf_size=cap)
    np.testing.assert_array_equal(sizes, ix.leaf_sizes())
    np.testing.assert_array_equal(ids, ix.leaf_ids())
