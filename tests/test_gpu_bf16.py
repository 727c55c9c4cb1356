"""The batched path with the tensor-core (BF16) filter, through the C ABI,
against the CPU oracle's brute force (indices exact, ties to the lower row;
distances within 1e-5 relative) and against the plain batch path (identical
indices and distances): the filter only drops rows whose filtered distance
minus its error bound already exceeds an upper bound of the k-th best."""
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
    assert len(bad) == 0, "queries %s: got %s want %s" % (bad[:5], got_i[bad[:3]], ref_i[bad[:3]])
    np.testing.assert_allclose(got_d, np.sqrt(ref_d2), rtol=RTOL, atol=1e-30)


def both(X, Q, k, leaf_size=2000, stats=False):
    ix = pkg.Index(torch.from_numpy(X).cuda(), leaf_size=leaf_size)
    Qt = torch.from_numpy(Q).cuda()
    i1, d1 = ix.query_batch(Qt, k)
    out = ix.query_batch_bf16(Qt, k, stats=stats)
    i2, d2 = out[0], out[1]
    np.testing.assert_array_equal(i2.cpu().numpy(), i1.cpu().numpy())
    np.testing.assert_array_equal(d2.cpu().numpy(), d1.cpu().numpy())
    return ix, i2.cpu().numpy(), d2.cpu().numpy(), (out[2] if stats else None)


@pytest.mark.parametrize("k", [1, 10])
def test_config0_shape(k):
    """100,000 z-normalised random walks x 256, leaf size 2000; 90 fresh walks
    and 10 members with N(0, 0.01) noise."""
    N, n = 100_000, 256
    X = datagen.rows("walk", 0, 0, N, n)
    Q, src = datagen.queries("walk", 0, N, n, 1, 90, 10, 0.01)
    _, i, d, st = both(X, Q, k, stats=True)
    check_knn(i, d, X, Q, k)
    np.testing.assert_array_equal(i[90:, 0], src[90:])
    for s in st:
        assert 0 <= s["leaves_queued"] == s["leaves_scanned"] < s["leaves_total"]
        assert s["window"] >= 1 and s["reruns"] == 0


def test_many_queries_per_leaf_and_ragged_tiles():
    """300 queries (more than one 256-query work item per leaf), leaves of 500
    rows (ragged 128-row tiles), a collection size that is not a tile multiple."""
    N, n = 30_011, 256
    X = datagen.rows("walk", 21, 0, N, n)
    Q, _ = datagen.queries("walk", 21, N, n, 22, 200, 100, 0.2)
    _, i, d, _ = both(X, Q, 5, leaf_size=500)
    check_knn(i, d, X, Q, 5)


@pytest.mark.parametrize("n,N", [(64, 20000), (128, 20000), (192, 12000), (512, 8000), (2048, 3000)])
def test_lengths(n, N):
    X = datagen.rows("walk", 23, 0, N, n)
    Q, _ = datagen.queries("walk", 23, N, n, 24, 40, 20, 0.1)
    _, i, d, _ = both(X, Q, 3, leaf_size=300)
    check_knn(i, d, X, Q, 3)


@pytest.mark.parametrize("sigma", [0.01, 0.5, 1.0])
def test_sinusoids_by_hardness(sigma):
    N, n = 40_000, 256
    X = datagen.rows("sine", 25, 0, N, n)
    Q, _ = datagen.queries("sine", 25, N, n, 26, 0, 48, sigma)
    _, i, d, _ = both(X, Q, 10, leaf_size=1000)
    check_knn(i, d, X, Q, 10)


def test_duplicates_and_ties():
    N, n = 9000, 128
    X = datagen.rows("walk", 14, 0, N, n)
    X[100:2600] = X[7]
    X[5000:5100] = 0.0
    X[8000] = X[20]
    Q = np.concatenate([X[[7, 5000, 20, 21]], datagen.rows("walk", 15, 0, 4, n)])
    for k in [1, 2, 50]:
        _, i, d, _ = both(X, Q, k, leaf_size=300)
        check_knn(i, d, X, Q, k)
    assert i[0, 0] == 7 and i[2, 0] == 20 and i[2, 1] == 8000


def test_two_passes_and_host_buffers():
    """5000 queries run as two passes (at most 4096 per pass); host buffers in
    and out give the same answers as device buffers."""
    N, n = 20_000, 128
    X = datagen.rows("walk", 27, 0, N, n)
    Q, _ = datagen.queries("walk", 27, N, n, 28, 4000, 1000, 0.05)
    ix = pkg.Index(torch.from_numpy(X).cuda(), leaf_size=400)
    i1, d1 = ix.query_batch(Q, 2)
    i2, d2 = ix.query_batch_bf16(Q, 2)
    i3, d3 = ix.query_batch_bf16(torch.from_numpy(Q).cuda(), 2)
    np.testing.assert_array_equal(i2, i1)
    np.testing.assert_array_equal(d2, d1)
    np.testing.assert_array_equal(i3.cpu().numpy(), i1)
    np.testing.assert_array_equal(d3.cpu().numpy(), d1)
    sel = np.arange(0, 5000, 97)
    check_knn(i2[sel], d2[sel], X, Q[sel], 2)


def test_window_overflow_falls_back_to_the_single_query_path():
    """200,000 identical rows: every row ties at distance 0, the per-query
    window overflows and the query is answered again alone."""
    N, n = 200_000, 64
    X = torch.zeros((N, n), dtype=torch.float32, device="cuda")
    ix = pkg.Index(X, leaf_size=2000)
    i, d, st = ix.query_batch_bf16(torch.zeros((2, n), device="cuda"), 3, stats=True)
    assert i.cpu().tolist() == [[0, 1, 2], [0, 1, 2]]
    assert d.cpu().tolist() == [[0.0] * 3] * 2
    assert all(s["reruns"] >= 1 for s in st)


def test_invalid_inputs():
    X = datagen.rows("walk", 29, 0, 2000, 96)
    ix = pkg.Index(torch.from_numpy(X).cuda(), leaf_size=100)
    with pytest.raises(pkg.ISAXError) as e:
        ix.query_batch_bf16(X[:4], 1)
    assert e.value.status == 1 and "multiple of 64" in e.value.message
    X4 = datagen.rows("walk", 29, 0, 500, 4096)
    with pytest.raises(pkg.ISAXError) as e:
        pkg.Index(torch.from_numpy(X4).cuda(), leaf_size=100).query_batch_bf16(X4[:2], 1)
    assert "at most 2048" in e.value.message
    X = datagen.rows("walk", 29, 0, 2000, 64)
    ix = pkg.Index(torch.from_numpy(X).cuda(), leaf_size=100)
    q = X[:3].copy()
    q[1, 5] = np.nan
    with pytest.raises(pkg.ISAXError) as e:
        ix.query_batch_bf16(q, 1)
    assert "non-finite" in e.value.message
    with pytest.raises(pkg.ISAXError):
        ix.query_batch_bf16(X[:3], 1025)
    i, d = ix.query_batch_bf16(X[:3], 1)
    assert i[:, 0].tolist() == [0, 1, 2]


def test_filter_error_bound_holds_on_the_tensor_cores():
    """The bound the filter prunes with, E = c_xq X Q + c_sq (X^2 + Q^2), covers
    the tensor-core dot product of BF16-rounded z-normalised series against
    the exact FP64 dot product of the fp32 series."""
    n = 256
    X = datagen.rows("walk", 30, 0, 128, n)
    Q = np.concatenate([datagen.rows("walk", 31, 0, 200, n), X[:56]])
    a = torch.from_numpy(X).to(torch.bfloat16).cuda().contiguous()
    b = torch.from_numpy(Q).to(torch.bfloat16).cuda().contiguous()
    D = torch.empty(128, 256, dtype=torch.float32, device="cuda")
    pkg.isax_tc_selftest(a.data_ptr(), b.data_ptr(), 256, D.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
    exact = X.astype(np.float64) @ Q.astype(np.float64).T
    xn = np.sqrt((X.astype(np.float64) ** 2).sum(1))[:, None]
    qn = np.sqrt((Q.astype(np.float64) ** 2).sum(1))[None, :]
    u, ub = 2.0 ** -24, 2.0 ** -8
    c_dot = (2 * ub + ub * ub) + n * 2.0 ** -21 * (1 + ub) ** 2
    err = np.abs(D.cpu().numpy().astype(np.float64) - exact)
    assert (err <= c_dot * xn * qn).all()
    # and it is not vacuous: the observed error reaches a fair part of it
    assert err.max() > 0.01 * (c_dot * xn * qn).max()
