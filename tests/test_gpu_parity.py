"""GPU path (through the C ABI) against the CPU oracle, element by element, on
seeded inputs shaped like the paper's workloads.  Indices must match exactly
(ties to the lower row); distances within 1e-5 relative."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import datagen
import oracle
import paper_2009_01614_gb300 as pkg

pytestmark = pytest.mark.gpu

RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def check_knn(got_i, got_d, X, Q, k):
    ref_i, ref_d2 = oracle.bruteforce_knn(X, Q, k)
    got_i = np.asarray(got_i).reshape(len(Q), k)
    got_d = np.asarray(got_d, dtype=np.float64).reshape(len(Q), k)
    bad = np.nonzero((got_i != ref_i).any(axis=1))[0]
    assert len(bad) == 0, "queries %s: got %s want %s (d %s vs %s)" % (
        bad[:5], got_i[bad[:3]], ref_i[bad[:3]], got_d[bad[:3]], np.sqrt(ref_d2[bad[:3]]))
    np.testing.assert_allclose(got_d, np.sqrt(ref_d2), rtol=RTOL, atol=1e-30)


def run(X, Q, k, card=256, leaf_size=2000, device=True, batch=True):
    Xt = torch.from_numpy(X).cuda() if device else X
    ix = pkg.Index(Xt, cardinality=card, leaf_size=leaf_size)
    Qt = torch.from_numpy(Q).cuda() if device else Q
    if batch:
        i, d = ix.query_batch(Qt, k)
    else:
        outs = [ix.query(Qt[b], k) for b in range(len(Q))]
        i = [o[0] for o in outs]
        d = [o[1] for o in outs]
        if device:
            i, d = torch.stack(i), torch.stack(d)
    if device:
        i, d = i.cpu().numpy(), d.cpu().numpy()
    return ix, np.asarray(i), np.asarray(d)


# ---------------------------------------------------------------- generator
@pytest.mark.parametrize("kind,n", [("walk", 256), ("sine", 128), ("walk", 48)])
def test_device_generator_is_bit_identical(kind, n):
    N = 3000
    out = torch.empty((N, n), dtype=torch.float32, device="cuda")
    datagen.rows_device(kind, 9, 1000, N, n, out.data_ptr())
    torch.cuda.synchronize()
    ref = datagen.rows(kind, 9, 1000, N, n)
    np.testing.assert_array_equal(out.cpu().numpy(), ref)


# ---------------------------------------------------------------- summarize
@pytest.mark.parametrize("card", [4, 16, 256])
def test_breakpoint_table_equals_oracle(card):
    X = datagen.rows("walk", 1, 0, 500, 64)
    ix = pkg.Index(torch.from_numpy(X).cuda(), cardinality=card, leaf_size=50)
    bp = ix.export()["breakpoints"]
    np.testing.assert_array_equal(bp, oracle.breakpoints(card).astype(np.float32))


@pytest.mark.parametrize("kind,n,N", [("walk", 256, 40000), ("sine", 128, 20000), ("walk", 48, 5000),
                                      ("walk", 1024, 3000), ("walk", 16, 5000)])
def test_summarize_parity(kind, n, N):
    X = datagen.rows(kind, 2, 0, N, n)
    sax, paa = pkg.summarize(torch.from_numpy(X).cuda())
    sax, paa = sax.cpu().numpy(), paa.cpu().numpy()
    P64, S64 = oracle.summarize(X)
    m = n // 16
    eps = 1.01 * (m + 1) * 2.0**-24 * np.abs(X).max()
    assert np.abs(paa - P64).max() <= eps
    beta = oracle.breakpoints(256)
    diff = sax != S64
    if diff.any():  # only where the FP64 PAA is within the fp32 error of a breakpoint
        near = np.min(np.abs(P64[diff][:, None] - beta[None, :]), axis=1)
        assert (near <= eps + 1e-7).all()
    assert diff.mean() < 1e-3


def test_summarize_host_buffers_match_device():
    X = datagen.rows("walk", 3, 0, 3000, 256)
    s1, p1 = pkg.summarize(X)
    s2, p2 = pkg.summarize(torch.from_numpy(X).cuda())
    np.testing.assert_array_equal(s1, s2.cpu().numpy())
    np.testing.assert_array_equal(p1, p2.cpu().numpy())


# ---------------------------------------------------------------- build
def expected_leaves(keys, L, root_bits=16, keybits=64):
    """Leaf starts of the documented rule: split every node holding more than
    L series on its next key bit (round-robin over segments), root always;
    runs of identical keys cut into pieces of L."""
    N = len(keys)
    starts = []

    def rec(b, e, depth):
        if b >= e:
            return
        if depth >= root_bits and e - b <= L:
            starts.append(b)
            return
        if depth >= keybits:
            starts.extend(range(b, e, L))
            return
        bit = np.uint64(1) << np.uint64(63 - depth)
        ones = (keys[b:e] & bit) != 0
        mid = b + int(np.argmax(ones)) if ones.any() else e
        rec(b, mid, depth + 1)
        rec(mid, e, depth + 1)

    rec(0, N, 0)
    return np.array(starts + [N], dtype=np.int64)


def keys_of(sax, cbits):
    key = np.zeros(len(sax), dtype=np.uint64)
    for pl in range(4):
        b = cbits - 1 - pl
        plane = np.zeros(len(sax), dtype=np.uint64)
        if b >= 0:
            for i in range(16):
                plane |= ((sax[:, i].astype(np.uint64) >> np.uint64(b)) & np.uint64(1)) << np.uint64(15 - i)
        key = (key << np.uint64(16)) | plane
    return key


@pytest.mark.parametrize("in_place", [False, True])
@pytest.mark.parametrize("N,leaf,card", [(30000, 100, 256), (5000, 7, 256), (20000, 500, 16),
                                         (4001, 2000, 256), (1, 5, 256), (3000, 1, 4)])
def test_build_invariants(N, leaf, card, in_place):
    """Leaf order, envelopes and leaf boundaries; with the rows read in place the
    SAX words and row ids are put in leaf order by the radix sort's last pass."""
    n = 128
    X = datagen.rows("walk", 4, 0, N, n)
    X[N // 3: N // 3 + min(N // 4, 2 * leaf + 3)] = X[0]  # a long run of identical words
    ix = pkg.Index(torch.from_numpy(X).cuda(), cardinality=card, leaf_size=leaf, rows_in_place=in_place)
    ex = ix.export()
    orig = ex["orig"].astype(np.int64)
    assert np.array_equal(np.sort(orig), np.arange(N))
    sax_ref, _ = pkg.summarize(torch.from_numpy(X).cuda(), cardinality=card)
    sax_ref = sax_ref.cpu().numpy()
    np.testing.assert_array_equal(ex["sax"], sax_ref[orig])
    lb = ex["leaf_begin"].astype(np.int64)
    assert lb[0] == 0 and lb[-1] == N and (np.diff(lb) > 0).all()
    info = ix.info()
    assert info["leaves"] == len(lb) - 1 and info["max_leaf"] == np.diff(lb).max()
    assert np.diff(lb).max() <= leaf
    for l in range(len(lb) - 1):
        s = ex["sax"][lb[l]:lb[l + 1]]
        np.testing.assert_array_equal(ex["env"][l, :16], s.min(axis=0))
        np.testing.assert_array_equal(ex["env"][l, 16:], s.max(axis=0))
    cbits = card.bit_length() - 1
    keys = keys_of(ex["sax"], cbits)
    assert (keys[1:] >= keys[:-1]).all()
    # stable: equal keys keep ascending original rows
    same = keys[1:] == keys[:-1]
    assert (orig[1:][same] > orig[:-1][same]).all()
    np.testing.assert_array_equal(lb, expected_leaves(keys, leaf, keybits=16 * min(cbits, 4)))


def test_build_from_host_equals_device():
    X = datagen.rows("sine", 5, 0, 8000, 128)
    a = pkg.Index(X, leaf_size=64).export()
    b = pkg.Index(torch.from_numpy(X).cuda(), leaf_size=64).export()
    for key in a:
        np.testing.assert_array_equal(a[key], b[key])


# ---------------------------------------------------------------- queries
def test_config0_shape_exact_1nn():
    """100,000 random walks x 256, leaf 2000; 90 fresh walks + 10 noisy members."""
    N, n = 100000, 256
    X = datagen.rows("walk", 0, 0, N, n)
    Q, src = datagen.queries("walk", 0, N, n, 1, 90, 10, 0.01)
    ix, i, d = run(X, Q, 1)
    check_knn(i, d, X, Q, 1)
    np.testing.assert_array_equal(i[90:, 0], src[90:])


@pytest.mark.parametrize("k", [10, 100])
def test_knn_random_walks(k):
    N, n = 60000, 256
    X = datagen.rows("walk", 6, 0, N, n)
    Q, _ = datagen.queries("walk", 6, N, n, 7, 12, 8, 0.05)
    ix, i, d = run(X, Q, k, leaf_size=500)
    check_knn(i, d, X, Q, k)


@pytest.mark.parametrize("sigma", [0.01, 0.1, 0.5, 1.0])
def test_knn_sinusoids_by_hardness(sigma):
    N, n = 30000, 256
    X = datagen.rows("sine", 0, 0, N, n)
    Q, _ = datagen.queries("sine", 0, N, n, 3, 0, 12, sigma)
    Xt = torch.from_numpy(X).cuda()
    ix = pkg.Index(Xt, leaf_size=300)
    for k in [1, 10, 100]:
        i, d = ix.query_batch(torch.from_numpy(Q).cuda(), k)
        check_knn(i.cpu().numpy(), d.cpu().numpy(), X, Q, k)


@pytest.mark.parametrize("n", [16, 48, 128, 512, 1024])
def test_lengths(n):
    N = 6000
    X = datagen.rows("walk", 8, 0, N, n)
    Q, _ = datagen.queries("walk", 8, N, n, 9, 5, 5, 0.1)
    ix, i, d = run(X, Q, 3, leaf_size=150)
    check_knn(i, d, X, Q, 3)


@pytest.mark.parametrize("card", [2, 4, 16, 64])
def test_cardinalities(card):
    N, n = 8000, 128
    X = datagen.rows("walk", 10, 0, N, n)
    Q, _ = datagen.queries("walk", 10, N, n, 11, 5, 5, 0.1)
    ix, i, d = run(X, Q, 4, card=card, leaf_size=100)
    check_knn(i, d, X, Q, 4)


@pytest.mark.parametrize("N,leaf,k", [(1, 2000, 1), (2, 2000, 2), (5, 1, 5), (1999, 2000, 7),
                                      (2000, 2000, 1), (2001, 2000, 3), (6000, 2000, 1),
                                      (3000, 1, 2), (700, 700, 700)])
def test_sizes_and_leaf_edges(N, leaf, k):
    n = 64
    X = datagen.rows("walk", 12, 0, N, n)
    Q = np.concatenate([datagen.rows("walk", 13, 0, 3, n), X[: min(N, 2)]])
    ix, i, d = run(X, Q, k, leaf_size=leaf)
    check_knn(i, d, X, Q, k)


def test_duplicates_constants_and_ties():
    N, n = 9000, 128
    X = datagen.rows("walk", 14, 0, N, n)
    X[100:2600] = X[7]      # 2501 identical rows
    X[5000:5100] = 0.0      # constant rows
    X[8000] = X[20]         # a single duplicate
    Q = np.concatenate([X[[7, 5000, 20, 21]], datagen.rows("walk", 15, 0, 4, n)])
    for k in [1, 2, 50]:
        ix, i, d = run(X, Q, k, leaf_size=300)
        check_knn(i, d, X, Q, k)
    assert i[0, 0] == 7 and i[2, 0] == 20 and i[2, 1] == 8000


def test_single_equals_batch_and_host_equals_device():
    N, n = 20000, 256
    X = datagen.rows("walk", 16, 0, N, n)
    Q, _ = datagen.queries("walk", 16, N, n, 17, 6, 6, 0.1)
    _, i1, d1 = run(X, Q, 5, leaf_size=400, batch=True)
    _, i2, d2 = run(X, Q, 5, leaf_size=400, batch=False)
    _, i3, d3 = run(X, Q, 5, leaf_size=400, device=False)
    np.testing.assert_array_equal(i1, i2)
    np.testing.assert_array_equal(d1, d2)
    np.testing.assert_array_equal(i1, i3)
    np.testing.assert_array_equal(d1, d3)
    check_knn(i1, d1, X, Q, 5)


def test_stats_are_consistent():
    N, n = 100000, 256
    X = datagen.rows("walk", 0, 0, N, n)
    Q, _ = datagen.queries("walk", 0, N, n, 1, 10, 0, 0.01)
    ix = pkg.Index(torch.from_numpy(X).cuda())
    _, _, st = ix.query_batch(torch.from_numpy(Q).cuda(), 1, stats=True)
    for s in st:
        assert s["leaves_total"] == ix.info()["leaves"]
        assert 0 <= s["leaves_scanned"] <= s["leaves_queued"] < s["leaves_total"]
        assert s["series_refined"] <= N and s["series_lb"] <= N
        assert s["window"] >= 1 and s["candidates"] >= s["window"]
        assert s["reruns"] == 0


def test_invalid_inputs_on_gpu():
    X = datagen.rows("walk", 18, 0, 1000, 64)
    bad = X.copy()
    bad[500, 3] = np.nan
    with pytest.raises(pkg.ISAXError) as e:
        pkg.Index(torch.from_numpy(bad).cuda())
    assert e.value.status == 1 and "non-finite" in e.value.message
    bad[500, 3] = np.inf
    with pytest.raises(pkg.ISAXError):
        pkg.Index(bad)
    ix = pkg.Index(torch.from_numpy(X).cuda(), leaf_size=50)
    q = X[0].copy()
    q[10] = np.inf
    with pytest.raises(pkg.ISAXError) as e:
        ix.query(q, 1)
    assert "non-finite" in e.value.message
    with pytest.raises(pkg.ISAXError):
        ix.query(X[0], 1001)
    with pytest.raises(pkg.ISAXError):
        ix.query(X[0], 0)
    # the index stays usable after rejected calls
    i, d = ix.query(X[1], 1)
    assert i[0] == 1 and d[0] == 0.0


def test_candidate_overflow_rerun():
    """1.2M identical rows tie at distance 0: more candidates than the initial
    buffer holds, so the query reruns with a larger one and still returns the
    lowest rows."""
    N, n = 1_200_000, 16
    X = torch.zeros((N, n), dtype=torch.float32, device="cuda")
    ix = pkg.Index(X, leaf_size=2000)
    i, d, st = ix.query(torch.zeros(n, device="cuda"), 3, stats=True)
    assert i.cpu().tolist() == [0, 1, 2] and d.cpu().tolist() == [0.0, 0.0, 0.0]
    assert st["reruns"] >= 1


@pytest.mark.parametrize("kind,k", [("walk", 1), ("walk", 10), ("sine", 5)])
def test_flat_scan_equals_messi_and_oracle(kind, k):
    """The ParIS-style flat scan bounds every series outside the approximate
    answer and returns the same answer as MESSI's pruned, ordered search."""
    N, n = 60_000, 256
    X = datagen.rows(kind, 31, 0, N, n)
    Q, _ = datagen.queries(kind, 31, N, n, 32, 12, 8, 0.1)
    ix = pkg.Index(torch.from_numpy(X).cuda(), leaf_size=500)
    L = ix.info()["leaves"]
    got_i, got_d = [], []
    for q in Q:
        i1, d1, s1 = ix.query(q, k, stats=True)
        i2, d2, s2 = ix.query_flat(q, k, stats=True)
        np.testing.assert_array_equal(i2, i1)
        np.testing.assert_array_equal(d2, d1)
        assert s2["series_lb"] == N - s2["approx_series"]
        assert s2["leaves_queued"] == s2["leaves_scanned"] <= L
        assert s2["series_lb"] >= s1["series_lb"]
        got_i.append(i2)
        got_d.append(d2)
    check_knn(np.array(got_i), np.array(got_d), X, Q, k)


def test_rows_on_host_give_the_same_answers():
    """Rows kept in pinned host memory (read over the CPU-GPU link) give the
    same answers on every query path as rows in device memory."""
    N, n = 40_000, 256
    X = datagen.rows("walk", 33, 0, N, n)
    Q, _ = datagen.queries("walk", 33, N, n, 34, 10, 6, 0.05)
    a = pkg.Index(torch.from_numpy(X).cuda(), leaf_size=400)
    b = pkg.Index(torch.from_numpy(X).cuda(), leaf_size=400, rows_on_host=True)
    assert b.info()["device_bytes"] < a.info()["device_bytes"] - N * n * 4 + 1
    # built from host memory read in place (page-locked by the build), rows to host
    c = pkg.Index(X, leaf_size=400, rows_on_host=True)
    ea, eb = np.empty((a.info()["N"], 16), np.uint8), np.empty((a.info()["N"], 16), np.uint8)
    pkg.isax_index_export(a._h, ea.ctypes.data)
    pkg.isax_index_export(c._h, eb.ctypes.data)
    np.testing.assert_array_equal(ea, eb)
    for k in (1, 10):
        i1, d1 = a.query_batch(Q, k)
        i2, d2 = b.query_batch(Q, k)
        np.testing.assert_array_equal(i2, i1)
        np.testing.assert_array_equal(d2, d1)
        i3, d3 = b.query_batch_bf16(Q, k)
        np.testing.assert_array_equal(i3, i1)
        np.testing.assert_array_equal(d3, d1)
        i4, d4 = b.query_flat(Q[0], k)
        np.testing.assert_array_equal(i4, i1[0])
        i5, d5 = c.query_batch(Q, k)
        np.testing.assert_array_equal(i5, i1)
        np.testing.assert_array_equal(d5, d1)
        check_knn(i2, d2, X, Q, k)
    c.close()
    b.close()
    a.close()


@pytest.mark.parametrize("n,card", [(256, 256), (192, 16), (64, 256)])
def test_rows_in_place_give_the_same_answers(n, card):
    """An index that reads the caller's rows in place (by original row index,
    nothing copied) answers every query path exactly like the index that copies
    the rows into leaf order, and like the oracle; it holds no row bytes."""
    N = 30_000
    X = datagen.rows("walk", 41, 0, N, n)
    Q, _ = datagen.queries("walk", 41, N, n, 42, 12, 6, 0.05)
    Xd = torch.from_numpy(X).cuda()
    a = pkg.Index(Xd, cardinality=card, leaf_size=300)
    b = pkg.Index(Xd, cardinality=card, leaf_size=300, rows_in_place=True)
    assert b.info()["device_bytes"] <= a.info()["device_bytes"] - N * n * 4
    ea, eb = np.empty((N, 16), np.uint8), np.empty((N, 16), np.uint8)
    oa, ob = np.empty(N, np.uint32), np.empty(N, np.uint32)
    pkg.isax_index_export(a._h, ea.ctypes.data, oa.ctypes.data)
    pkg.isax_index_export(b._h, eb.ctypes.data, ob.ctypes.data)
    np.testing.assert_array_equal(ea, eb)
    np.testing.assert_array_equal(oa, ob)
    for k in (1, 7):
        i1, d1 = a.query_batch(Q, k)
        i2, d2 = b.query_batch(Q, k)
        np.testing.assert_array_equal(i2, i1)
        np.testing.assert_array_equal(d2, d1)
        check_knn(i2, d2, X, Q, k)
        for qi in (0, len(Q) - 1):
            i3, d3 = b.query(Q[qi], k)
            np.testing.assert_array_equal(i3, i1[qi])
            np.testing.assert_array_equal(d3, d1[qi])
            i4, d4 = b.query_flat(Q[qi], k)
            np.testing.assert_array_equal(i4, i1[qi])
            np.testing.assert_array_equal(d4, d1[qi])
        if n % 64 == 0:
            i5, d5 = b.query_batch_bf16(Q, k)
            np.testing.assert_array_equal(i5, i1)
            np.testing.assert_array_equal(d5, d1)
    b.close()
    a.close()
    # the index keeps the tensor alive on its own
    c = pkg.Index(torch.from_numpy(X).cuda(), cardinality=card, leaf_size=300, rows_in_place=True)
    i6, d6 = c.query_batch(Q, 1)
    check_knn(i6, d6, X, Q, 1)
    c.close()


def test_trim_memory_between_builds():
    """Cached pool memory handed back to the driver between two builds of the
    same collection from host memory: same answers, and a bad device ordinal is
    rejected."""
    N, n = 20_000, 128
    X = datagen.rows("walk", 51, 0, N, n)
    Q, _ = datagen.queries("walk", 51, N, n, 52, 8, 4, 0.05)
    a = pkg.Index(X, leaf_size=200)
    i1, d1 = a.query_batch(Q, 3)
    a.close()
    pkg.isax_trim_memory(0)
    b = pkg.Index(X, leaf_size=200)
    i2, d2 = b.query_batch(Q, 3)
    np.testing.assert_array_equal(i2, i1)
    np.testing.assert_array_equal(d2, d1)
    check_knn(i2, d2, X, Q, 3)
    b.close()
    with pytest.raises(pkg.ISAXError):
        pkg.isax_trim_memory(4096)


# ---------------------------------------------------------------- balanced split (ADS+)
def _far_from_breakpoints(X, card):
    """The rows whose FP64 segment means all lie farther than four times the
    fp32 PAA error bound from every breakpoint: on them the GPU's fp32 symbols
    and the oracle's FP64 symbols agree, so both sides build the same tree."""
    P64, _ = oracle.summarize(X, card=card)
    m = X.shape[1] // 16
    eps = 1.01 * (m + 1) * 2.0**-24 * np.abs(X).max()
    beta = np.sort(oracle.breakpoints(card))
    j = np.clip(np.searchsorted(beta, P64), 1, len(beta) - 1)
    near = np.minimum(np.abs(P64 - beta[j - 1]), np.abs(P64 - beta[j])) if len(beta) > 1 else np.abs(P64 - beta[0])
    return np.ascontiguousarray(X[(near > 4 * eps + 1e-7).all(axis=1)])


@pytest.mark.parametrize("kind,N,n,card,cap,dup", [
    ("walk", 3000, 64, 256, 20, False), ("walk", 2000, 64, 16, 7, True), ("sine", 3000, 128, 256, 50, False),
    ("walk", 600, 32, 4, 1, True), ("walk", 4000, 256, 256, 100, True), ("walk", 40000, 256, 256, 300, False)])
def test_balanced_split_tree_equals_oracle(kind, N, n, card, cap, dup):
    """ADS+ node splitting on the GPU (level by level over the whole collection)
    forms exactly the oracle's leaves (series inserted one by one, a leaf split
    when it overflows): the same members in the same depth-first order, empty
    leaves dropped; a run of identical words beyond capacity stays one leaf.
    Answers equal brute force on every query path, and a query equal to a
    collection row descends to that row's leaf."""
    X = _far_from_breakpoints(datagen.rows(kind, 11, 0, N, n), card)
    if dup:
        X[len(X) // 3: len(X) // 3 + 2 * cap + 3] = X[0]
    N = len(X)
    Xd = torch.from_numpy(X).cuda()
    ix = pkg.Index(Xd, cardinality=card, leaf_size=cap, split="balanced")
    ex = ix.export()
    orig = ex["orig"].astype(np.int64)
    _, S64 = oracle.summarize(X, card=card)
    np.testing.assert_array_equal(ex["sax"], S64[orig])  # precondition: the same symbols
    ox = oracle.ISAXIndex(X, card=card, leaf_size=cap)
    np.testing.assert_array_equal(orig, ox.leaf_ids())
    sizes = ox.leaf_sizes()
    lb = ex["leaf_begin"].astype(np.int64)
    np.testing.assert_array_equal(np.diff(lb), sizes[sizes > 0])
    info = ix.info()
    assert info["leaves"] == (sizes > 0).sum() and info["max_leaf"] == sizes.max()
    for l in range(0, len(lb) - 1, max(1, (len(lb) - 1) // 50)):
        s = ex["sax"][lb[l]:lb[l + 1]]
        np.testing.assert_array_equal(ex["env"][l, :16], s.min(axis=0))
        np.testing.assert_array_equal(ex["env"][l, 16:], s.max(axis=0))

    Q, _ = datagen.queries(kind, 11, N, n, 12, 10, 6, 0.05)
    for k in (1, 5):
        i, d = ix.query_batch(torch.from_numpy(Q).cuda(), k)
        check_knn(i.cpu().numpy(), d.cpu().numpy(), X, Q, k)
        for qi in (0, len(Q) - 1):
            i2, d2 = ix.query(Q[qi], k)
            np.testing.assert_array_equal(i2, i.cpu().numpy()[qi])
            i3, d3 = ix.query_flat(Q[qi], k)
            np.testing.assert_array_equal(i3, i.cpu().numpy()[qi])
    pos = np.empty(N, np.int64)
    pos[orig] = np.arange(N)
    for r in np.linspace(0, N - 1, 12).astype(np.int64):
        _, _, st = ix.query(X[r], 1, stats=True)
        leaf_r = int(np.searchsorted(lb, pos[r], side="right")) - 1
        assert st["approx_leaf"] <= leaf_r <= st["approx_leaf"] + 4, (r, leaf_r, st["approx_leaf"])
    ix.close()


def test_balanced_split_with_every_row_store():
    """The balanced split combines with rows in place, rows in host memory and a
    host input: the same leaves and the same answers."""
    N, n = 30_000, 128
    X = datagen.rows("walk", 43, 0, N, n)
    Q, _ = datagen.queries("walk", 43, N, n, 44, 10, 6, 0.05)
    Xd = torch.from_numpy(X).cuda()
    a = pkg.Index(Xd, leaf_size=200, split="balanced")
    ea = a.export()
    others = [pkg.Index(Xd, leaf_size=200, split="balanced", rows_in_place=True),
              pkg.Index(Xd, leaf_size=200, split="balanced", rows_on_host=True),
              pkg.Index(X, leaf_size=200, split="balanced")]
    i1, d1 = a.query_batch(Q, 3)
    check_knn(i1, d1, X, Q, 3)
    i0, d0 = a.query_batch_bf16(Q, 3)  # the tensor-core filtered batch on the same leaves
    np.testing.assert_array_equal(i0, i1)
    np.testing.assert_array_equal(d0, d1)
    srv = pkg.Server(slots=4)  # the resident server on the same index
    cid = srv.add(a)
    for t, q in enumerate(Q):
        srv.submit(cid, q, 3, t)
    got = {}
    for _ in range(400):
        for r in srv.poll(64, wait_ms=50):
            got[r["tag"]] = r
        if len(got) == len(Q):
            break
    assert len(got) == len(Q)
    for t in range(len(Q)):
        assert got[t]["status"] == 0
        np.testing.assert_array_equal(got[t]["idx"], i1[t])
        np.testing.assert_array_equal(got[t]["dist"], d1[t])
    srv.close()
    for b in others:
        eb = b.export()
        for key in ("orig", "leaf_begin", "sax", "env"):
            np.testing.assert_array_equal(eb[key], ea[key])
        i2, d2 = b.query_batch(Q, 3)
        np.testing.assert_array_equal(i2, i1)
        np.testing.assert_array_equal(d2, d1)
        b.close()
    a.close()
