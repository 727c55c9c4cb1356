"""The allocation-free query entry point (isax_query_knn_noalloc), called
through the C ABI, must give the regular query's answers.  It serves callers
that cannot allocate device memory while they query: a runtime that owns every
byte of the GPU through its own pool, or a latency-critical serving thread for
which an allocation may block on the driver.  Its scratch is a fixed array
inside the library that every call reuses, so each query is answered twice in a
row, and the allocator hooks count every device allocation the library makes
while those calls run (there must be none).  Collected last on purpose: it must
pass both alone in a fresh process and after every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import datagen
import paper_2009_01614_gb300 as pkg

pytestmark = pytest.mark.gpu

RTOL = 1e-5
ISAX_ERR_OOM = 2
MAX_CANDIDATES = 262144


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


class _CountingHooks:
    """Allocator hooks that count calls.  The allocation hook returns NULL, so a
    call that tried to allocate would also fail with ISAX_ERR_OOM."""

    def __init__(self):
        self.allocs = 0
        self.frees = 0
        self._a = pkg.ALLOC_FN(self._alloc)
        self._f = pkg.FREE_FN(self._free)

    def _alloc(self, nbytes, stream, ctx):
        self.allocs += 1
        return None

    def _free(self, ptr, stream, ctx):
        self.frees += 1

    def __enter__(self):
        assert pkg.lib().isax_set_allocator(self._a, self._f, None) == 0
        return self

    def __exit__(self, *exc):
        pkg.lib().isax_set_allocator(ctypes.cast(None, pkg.ALLOC_FN), ctypes.cast(None, pkg.FREE_FN),
                                     None)
        return False


def _call(fn, handle, q, k, on_device):
    """Run one query through the raw C entry point `fn`: (status, idx, dist)."""
    if on_device:
        qd = torch.from_numpy(q).cuda()
        idx = torch.empty(k, dtype=torch.int64, device="cuda")
        dist = torch.empty(k, dtype=torch.float32, device="cuda")
        flags = pkg.MEM_INPUT_DEVICE | pkg.MEM_OUTPUT_DEVICE
        stream = torch.cuda.current_stream().cuda_stream
        rc = fn(handle, qd.data_ptr(), k, flags, idx.data_ptr(), dist.data_ptr(), None, stream)
        torch.cuda.synchronize()
        return rc, idx.cpu().numpy(), dist.cpu().numpy()
    qh = np.ascontiguousarray(q, dtype=np.float32)
    idx = np.empty(k, np.int64)
    dist = np.empty(k, np.float32)
    rc = fn(handle, qh.ctypes.data, k, 0, idx.ctypes.data, dist.ctypes.data, None, None)
    return rc, idx, dist


def _check_against_regular(ix, Q, ks):
    """Every query of Q, for each k: the regular answer first (it may allocate),
    then two allocation-free calls in a row under the counting hooks."""
    lib = pkg.lib()
    for k in ks:
        for b, q in enumerate(Q):
            on_device = bool(b % 2)
            rc, ref_i, ref_d = _call(lib.isax_query_knn, ix.handle, q, k, on_device)
            assert rc == 0, pkg.isax_last_error()
            with _CountingHooks() as hooks:
                for _ in range(2):  # the shared scratch keeps the previous call's contents
                    rc, got_i, got_d = _call(lib.isax_query_knn_noalloc, ix.handle, q, k, on_device)
                    assert rc == 0, pkg.isax_last_error()
                    np.testing.assert_array_equal(got_i, ref_i)
                    np.testing.assert_allclose(got_d, ref_d, rtol=RTOL, atol=0)
            assert hooks.allocs == 0 and hooks.frees == 0, (hooks.allocs, hooks.frees)


@pytest.mark.parametrize("in_place,split", [(False, "round-robin"), (True, "round-robin"), (False, "balanced")])
def test_noalloc_query_matches_regular_query_twice_in_a_row(in_place, split):
    N, n = 50000, 256
    X = datagen.rows("walk", 21, 0, N, n)
    Q, _ = datagen.queries("walk", 21, N, n, 22, 3, 3, 0.05)
    ix = pkg.Index(torch.from_numpy(X).cuda(), leaf_size=500, rows_in_place=in_place, split=split)
    _check_against_regular(ix, Q, (1, 10))
    ix.close()


@pytest.mark.parametrize("n", [48, 128, 512, 1024])
def test_noalloc_query_matches_regular_query_at_other_lengths(n):
    # 48: the generic distance path (n not a multiple of 128); 128, 512, 1024:
    # the vectorised paths with 1, 4 and 8 float4 per lane; 1024 also fills
    # the query slot of the fixed array more than any shorter length
    N = 12000
    X = datagen.rows("walk", 31, 0, N, n)
    Q, _ = datagen.queries("walk", 31, N, n, 32, 2, 2, 0.05)
    ix = pkg.Index(torch.from_numpy(X).cuda(), leaf_size=300)
    _check_against_regular(ix, Q, (1, 7))
    ix.close()


def test_noalloc_query_reports_candidate_overflow_then_recovers():
    # 300,000 identical rows and a query equal to them: every row is at distance
    # 0, so every refined row stays a candidate for the final ordering, more than
    # the fixed array holds.  The regular query reruns with more room; this
    # entry point reports ISAX_ERR_OOM instead.
    n = 16
    row = datagen.rows("walk", 41, 0, 1, n)[0]
    X = np.tile(row, (300_000, 1)).astype(np.float32)
    ix = pkg.Index(torch.from_numpy(X).cuda(), leaf_size=2000)
    lib = pkg.lib()
    rc, _, _ = _call(lib.isax_query_knn_noalloc, ix.handle, row.copy(), 1, False)
    assert rc == ISAX_ERR_OOM
    msg = pkg.isax_last_error()
    assert "more than %d candidates" % MAX_CANDIDATES in msg and "use isax_query_knn" in msg, msg
    rc, ref_i, ref_d = _call(lib.isax_query_knn, ix.handle, row.copy(), 1, False)
    assert rc == 0 and ref_i[0] == 0 and ref_d[0] == 0.0
    ix.close()
    # the next call on the shared array still answers correctly
    N2, n2 = 20000, 256
    X2 = datagen.rows("walk", 42, 0, N2, n2)
    Q2, _ = datagen.queries("walk", 42, N2, n2, 43, 2, 1, 0.05)
    ix2 = pkg.Index(torch.from_numpy(X2).cuda(), leaf_size=400)
    _check_against_regular(ix2, Q2, (1, 5))
    ix2.close()


def test_noalloc_query_rejects_an_index_beyond_its_limit():
    N, n = 600_000, 16  # leaf_size 1: one leaf per series, more than the 524288 it serves
    X = torch.from_numpy(datagen.rows("walk", 23, 0, N, n)).cuda()
    ix = pkg.Index(X, leaf_size=1)
    assert ix.info()["leaves"] > 524288
    q = np.zeros(n, np.float32)
    idx = np.empty(1, np.int64)
    dist = np.empty(1, np.float32)
    rc = pkg.lib().isax_query_knn_noalloc(ix.handle, q.ctypes.data, 1, 0, idx.ctypes.data,
                                          dist.ctypes.data, None, None)
    assert rc == 1
    assert "at most 524288" in pkg.isax_last_error()
    ix.close()
