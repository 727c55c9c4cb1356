"""Randomised properties of the oracle's iSAX index (CPU, hypothesis): on
small random collections of any cardinality, leaf capacity and amount of
duplication, its exact search returns the brute-force answer, its leaves
partition the collection (row order inside a leaf, capacity respected except by
leaves of identical words), and the level-by-level bulk split builds the same
leaves as its one-by-one insertion."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402
from test_split_levels import bulk_leaves  # noqa: E402


@settings(max_examples=60, deadline=None)
@given(seed=st.integers(0, 2**31 - 1), N=st.integers(1, 300), n=st.sampled_from([16, 32, 64]),
       card=st.sampled_from([2, 4, 16, 256]), cap=st.integers(1, 40), dup=st.integers(0, 60),
       k=st.integers(1, 8))
def test_index_properties(seed, N, n, card, cap, dup, k):
    rng = np.random.default_rng(seed)
    X = np.cumsum(rng.standard_normal((N, n)), axis=1)
    X = (X - X.mean(axis=1, keepdims=True)) / np.maximum(X.std(axis=1, keepdims=True), 1e-12)
    X = X.astype(np.float32)
    if dup and N > 1:
        X[rng.integers(0, N, size=min(dup, N))] = X[0]
    ix = oracle.ISAXIndex(X, card=card, leaf_size=cap)
    ids, sizes = ix.leaf_ids(), ix.leaf_sizes()
    assert np.array_equal(np.sort(ids), np.arange(N)) and sizes.sum() == N
    _, S = oracle.summarize(X, card=card)
    off = np.concatenate([[0], np.cumsum(sizes)])
    for a, b in zip(off[:-1], off[1:]):
        assert (np.diff(ids[a:b]) > 0).all()
        if b - a > cap:  # only a leaf of identical words may exceed its capacity
            assert (S[ids[a:b]] == S[ids[a]]).all()
    bids, bsizes = bulk_leaves(S.astype(np.int64), card, cap)
    assert np.array_equal(bids, ids) and np.array_equal(bsizes, sizes)
    Q = np.vstack([X[rng.integers(0, N)] + 0.05 * rng.standard_normal(n).astype(np.float32),
                   rng.standard_normal(n).astype(np.float32)])
    kk = min(k, N)
    ref_i, ref_d = oracle.bruteforce_knn(X, Q, kk)
    for b in range(len(Q)):
        i, d, _ = ix.query(Q[b], kk)
        assert np.array_equal(i, ref_i[b])
        np.testing.assert_allclose(d, ref_d[b], rtol=0, atol=0)
