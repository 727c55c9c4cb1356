"""The CPU oracle pinned to what the paper and mathematics fix (not to itself):
closed forms, library special cases, published tables, invariants and brute
force on tiny inputs.  CPU only."""
import math
import os

import numpy as np
import pytest

import datagen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- breakpoints
def test_breakpoints_are_normal_quantiles():
    b = oracle.breakpoints(256)
    t = np.arange(1, 256)
    for bt, tt in zip(b, t):
        assert abs(0.5 * math.erfc(-bt / math.sqrt(2)) - tt / 256) < 1e-15
    from scipy.stats import norm
    np.testing.assert_allclose(b, norm.ppf(t / 256), rtol=0, atol=1e-14)
    assert b[127] == 0.0
    np.testing.assert_array_equal(b, -b[::-1])
    assert (np.diff(b) > 0).all()


@pytest.mark.parametrize("bits", range(1, 8))
def test_breakpoints_nest_across_cardinalities(bits):
    card = 1 << bits
    step = 256 // card
    np.testing.assert_array_equal(oracle.breakpoints(card), oracle.breakpoints(256)[step - 1::step])


def test_breakpoints_match_published_sax_table():
    with open(os.path.join(GOLDEN, "sax_breakpoints_lin2003.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            card, vals = line.split(":")
            ref = np.array([float(v) for v in vals.split()])
            np.testing.assert_allclose(oracle.breakpoints(int(card)), ref, rtol=0, atol=0.005)


# ---------------------------------------------------------------- PAA, SAX
@pytest.mark.parametrize("c", [0.5, -1.25, 3.0, 0.0])
def test_paa_of_constant_series(c):
    x = np.full(256, c, dtype=np.float32)
    np.testing.assert_array_equal(oracle.paa(x), np.full(16, c))


def test_paa_of_ramp_is_closed_form():
    n, w = 256, 16
    m = n // w
    a, b = -3.0, 0.0234375  # dyadic: every x_j and partial sum exact
    x = (a + b * np.arange(n)).astype(np.float32)
    ref = a + b * (np.arange(w) * m + (m - 1) / 2)
    np.testing.assert_array_equal(oracle.paa(x), ref)


def test_paa_matches_numpy_segment_means():
    X = datagen.rows("walk", 2, 0, 50, 256)
    P, _ = oracle.summarize(X)
    ref = X.astype(np.float64).reshape(50, 16, 16).mean(axis=2)
    np.testing.assert_allclose(P, ref, rtol=0, atol=1e-14)


def test_symbol_on_and_around_breakpoints():
    b = oracle.breakpoints(256)
    for t in [1, 17, 127, 128, 200, 255]:
        v = b[t - 1]
        assert oracle.symbol(v, b) == t  # on a breakpoint: upper region
        assert oracle.symbol(np.nextafter(v, -np.inf), b) == t - 1
    assert oracle.symbol(-1e9, b) == 0 and oracle.symbol(1e9, b) == 255


@pytest.mark.parametrize("bits", [1, 2, 4, 7])
def test_symbols_have_the_prefix_property(bits):
    rng = np.random.default_rng(bits)
    vals = rng.normal(size=500) * 1.5
    b256, bc = oracle.breakpoints(256), oracle.breakpoints(1 << bits)
    for v in vals:
        assert oracle.symbol(v, bc) == oracle.symbol(v, b256) >> (8 - bits)


def test_summarize_symbols_follow_the_region_definition():
    X = datagen.rows("walk", 4, 0, 100, 128)
    P, S = oracle.summarize(X)
    edges = np.concatenate([[-np.inf], oracle.breakpoints(256), [np.inf]])
    assert ((edges[S] <= P) & (P < edges[S.astype(int) + 1])).all()


# ---------------------------------------------------------------- lower bounds
def test_lb_closed_form_for_constant_series():
    n = 256
    b = oracle.breakpoints(256)
    c1 = -0.5
    x = np.full(n, 1.0, dtype=np.float32)
    qpaa = np.full(16, c1)
    _, S = oracle.summarize(x)
    s = int(S[0, 0])
    assert b[s - 1] <= 1.0 < b[s]
    lb2 = oracle.lb2_series(qpaa, S[0], n, b)
    assert lb2 == pytest.approx(n * (b[s - 1] - c1) ** 2, rel=1e-14)
    # query above the series' region: distance to the region's upper edge
    qpaa2 = np.full(16, 3.5)
    assert oracle.lb2_series(qpaa2, S[0], n, b) == pytest.approx(n * (3.5 - b[s]) ** 2, rel=1e-14)
    # query PAA inside the region: zero
    assert oracle.lb2_series(np.full(16, 1.0), S[0], n, b) == 0.0


@pytest.mark.parametrize("n", [16, 64, 256])
def test_lb_never_exceeds_ed_all_pairs(n):
    X = np.concatenate([datagen.rows("walk", 10 + n, 0, 120, n), datagen.rows("sine", 10 + n, 0, 80, n)])
    b = oracle.breakpoints(256)
    P, S = oracle.summarize(X)
    N = len(X)
    for i in range(N):
        d2 = ((X.astype(np.float64) - X[i].astype(np.float64)) ** 2).sum(axis=1)
        for j in range(N):
            lb2 = oracle.lb2_series(P[i], S[j], n, b)
            assert lb2 <= d2[j] * (1 + 1e-12) + 1e-12, (i, j, lb2, d2[j])


def test_node_bound_is_below_member_bounds():
    n = 256
    X = datagen.rows("walk", 21, 0, 200, n)
    b = oracle.breakpoints(256)
    P, S = oracle.summarize(X)
    rng = np.random.default_rng(0)
    for _ in range(300):
        i, j = rng.integers(0, len(X), 2)
        bits = rng.integers(1, 9, 16).astype(np.uint8)
        val = (S[j].astype(np.uint16) >> (8 - bits)).astype(np.uint16)
        lbn = oracle.lb2_node(P[i], val, bits, n, b)
        lbs = oracle.lb2_series(P[i], S[j], n, b)
        assert lbn <= lbs
        if (bits == 8).all():
            assert lbn == lbs
        if (bits == 1).all():
            # root-level region: only the sign of each segment is known
            ref = n / 16 * sum(
                (min(0.0, P[i][g]) if val[g] == 1 else max(0.0, P[i][g])) ** 2 for g in range(16))
            assert lbn == pytest.approx(ref, rel=1e-13, abs=1e-300)


# ---------------------------------------------------------------- brute force
def test_ed2_matches_direct_sum():
    x, q = datagen.rows("walk", 30, 0, 2, 256)
    ref = math.fsum((float(a) - float(c)) ** 2 for a, c in zip(x, q))
    assert oracle.ed2(x, q) == pytest.approx(ref, rel=1e-14)


@pytest.mark.parametrize("k", [1, 7, 40])
def test_bruteforce_matches_scipy_cdist(k):
    from scipy.spatial.distance import cdist
    X = datagen.rows("walk", 31, 0, 3000, 64)
    Q, _ = datagen.queries("walk", 31, 3000, 64, 32, 6, 6, 0.05)
    idx, d2 = oracle.bruteforce_knn(X, Q, k)
    D = cdist(Q.astype(np.float64), X.astype(np.float64), "sqeuclidean")
    for b in range(len(Q)):
        order = np.lexsort((np.arange(len(X)), D[b]))[:k]
        np.testing.assert_array_equal(idx[b], order)
        np.testing.assert_allclose(d2[b], D[b][order], rtol=1e-12, atol=1e-12)


def test_bruteforce_ties_go_to_the_lower_index():
    X = datagen.rows("walk", 40, 0, 100, 32)
    X[[70, 12, 55]] = X[3]
    idx, d2 = oracle.bruteforce_knn(X, X[3], 4)
    np.testing.assert_array_equal(idx[0], [3, 12, 55, 70])
    np.testing.assert_array_equal(d2[0], [0, 0, 0, 0])


def test_bruteforce_threading_is_invisible():
    X = datagen.rows("sine", 41, 0, 2000, 128)
    Q, _ = datagen.queries("sine", 41, 2000, 128, 42, 4, 4, 0.1)
    a = oracle.bruteforce_knn(X, Q, 9, nthreads=1)
    b = oracle.bruteforce_knn(X, Q, 9, nthreads=7)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_noisy_member_is_its_own_nearest_neighbour():
    N, n = 20000, 256
    X = datagen.rows("walk", 0, 0, N, n)
    Q, src = datagen.queries("walk", 0, N, n, 1, 0, 10, 0.01)
    idx, _ = oracle.bruteforce_knn(X, Q, 1)
    np.testing.assert_array_equal(idx[:, 0], src)


# ---------------------------------------------------------------- iSAX index
def _check_index_equals_bruteforce(X, Q, ks, leaf_size, card=256):
    ix = oracle.ISAXIndex(X, card=card, leaf_size=leaf_size)
    for k in ks:
        ref_i, ref_d = oracle.bruteforce_knn(X, Q, k)
        for b in range(len(Q)):
            i, d, st = ix.query(Q[b], k)
            np.testing.assert_array_equal(i, ref_i[b])
            np.testing.assert_array_equal(d, ref_d[b])
    return ix


@pytest.mark.parametrize("kind,n", [("walk", 256), ("walk", 64), ("sine", 128)])
def test_index_equals_bruteforce(kind, n):
    N = 6000
    X = datagen.rows(kind, 50, 0, N, n)
    Q, _ = datagen.queries(kind, 50, N, n, 51, 8, 8, 0.1)
    ix = _check_index_equals_bruteforce(X, Q, [1, 5, 30], leaf_size=40)
    sizes = ix.leaf_sizes()
    assert sizes.sum() == N and ix.leaves == len(sizes)


def test_index_prunes_on_random_walks():
    N = 20000
    X = datagen.rows("walk", 52, 0, N, 256)
    Q, _ = datagen.queries("walk", 52, N, 256, 53, 5, 5, 0.01)
    ix = oracle.ISAXIndex(X, leaf_size=100)
    refined = [ix.query(q, 1)[2].series_ed for q in Q]
    assert np.mean(refined) < 0.5 * N


def test_index_with_duplicates_constants_and_small_card():
    N, n = 900, 64
    X = datagen.rows("walk", 54, 0, N, n)
    X[100:400] = X[5]          # 301 identical rows: an unsplittable leaf
    X[500:520] = 0.0           # constant rows
    Q = np.concatenate([X[[5, 510, 7]], datagen.rows("walk", 55, 0, 3, n)])
    _check_index_equals_bruteforce(X, Q, [1, 3, 350], leaf_size=25)
    _check_index_equals_bruteforce(X, Q, [1, 12], leaf_size=25, card=4)


def test_index_tiny_collections():
    for N in [1, 2, 3]:
        X = datagen.rows("walk", 56, 0, N, 32)
        Q = datagen.rows("walk", 57, 0, 2, 32)
        _check_index_equals_bruteforce(X, Q, [1, N], leaf_size=1)


def test_index_leaves_respect_capacity():
    N = 5000
    X = datagen.rows("walk", 58, 0, N, 128)
    ix = oracle.ISAXIndex(X, leaf_size=30)
    assert ix.leaf_sizes().max() <= 30


def _words(rows):
    """Series of length 16 (one point per segment, so PAA = the values): 0.1 has
    symbol 2 (binary 10) and 1.0 symbol 3 (binary 11) at cardinality 4, whose
    breakpoints are -0.674, 0, 0.674.  Every series has root key 1...1 and the
    extra bit of a segment is 1 exactly where the value is 1.0."""
    X = np.full((len(rows), 16), 0.1, dtype=np.float32)
    for r, segs in enumerate(rows):
        X[r, list(segs)] = 1.0
    return X


@pytest.mark.parametrize("rows,cap,sizes,ids", [
    # capacity 2.  Insert 0,1,2: over capacity -> split {0,1,2}: segment 0 has
    # ones {0,2}, segment 1 ones {1,2} (both |2*2-3| = 1), the rest none: the tie
    # goes to segment 0 -> {1} | {0,2}.  3 joins {1}.  4 makes {0,2,4}: segment 0
    # is at full cardinality; segments 1 and 2 tie (one 1 each) -> segment 1:
    # {0,4} | {2}.  5 makes {0,4,5}: segments 0, 1 full; segment 2 -> {0,5} | {4}.
    ([[0], [1], [0, 1], [], [0, 2], [0]], 2, [2, 2, 1, 1], [1, 3, 0, 5, 4, 2]),
    # capacity 3: the split is decided on the first cap+1 members only.  {0..3}:
    # segment 1 has ones {0,1} (|4-4| = 0), segment 0 ones {1} (2) -> segment 1:
    # {2,3} | {0,1}.  4, 5 make {2,3,4,5}: segment 0 ones {4,5} -> {2,3} | {4,5};
    # 6 joins {4,5}.  (All seven at once would have chosen segment 0 first.)
    ([[1], [0, 1], [], [], [0], [0], [0]], 3, [2, 3, 2], [2, 3, 4, 5, 6, 0, 1]),
    # capacity 1, two identical words: every split sends both to child 0 and
    # leaves an empty child 1, segment after segment, until all 16 segments are
    # at full cardinality; the leaf then stays over capacity.
    ([[], []], 1, [2] + [0] * 16, [0, 1]),
])
def test_split_rule_worked_examples(rows, cap, sizes, ids):
    """ADS+ leaf split (Section II): on overflow a leaf splits on the segment
    whose extra bit divides its series most evenly (ties: lowest segment),
    decided when the leaf first holds cap+1 series in insertion order."""
    ix = oracle.ISAXIndex(_words(rows), card=4, leaf_size=cap)
    np.testing.assert_array_equal(ix.leaf_sizes(), sizes)
    assert ix.leaves == len(sizes)
    np.testing.assert_array_equal(ix.leaf_ids(), ids)


def test_leaf_ids_partition_the_collection():
    N = 4000
    X = datagen.rows("walk", 59, 0, N, 64)
    ix = oracle.ISAXIndex(X, leaf_size=40)
    ids, sizes = ix.leaf_ids(), ix.leaf_sizes()
    assert np.array_equal(np.sort(ids), np.arange(N))
    assert sizes.sum() == N
    for a, b in zip(np.cumsum(sizes) - sizes, np.cumsum(sizes)):
        assert (np.diff(ids[a:b]) > 0).all()  # insertion order inside a leaf
