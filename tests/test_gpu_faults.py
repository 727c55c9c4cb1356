"""Failure handling without a GPU fault (the library's status contract):

- a bounded device wait that runs out (an mbarrier nothing arrives on, with no
  copy in flight; a grid barrier short of one arrival) returns
  ISAX_ERR_TIMEOUT and leaves the device usable;
- a query whose control block reports a wait that gave up surfaces
  ISAX_ERR_TIMEOUT through every query entry point (single, batch, BF16
  batch, allocation-free, served), and the next query answers normally;
- a device allocation that fails (an allocator hook that returns NULL at its
  j-th call) makes build, query, batch, BF16 batch and server creation return
  ISAX_ERR_OOM, leaks nothing that was allocated, and leaves the index
  answering."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import datagen
import oracle
import paper_2009_01614_gb300 as pkg

pytestmark = pytest.mark.gpu

OK, OOM, TIMEOUT = 0, 2, 4


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _data(N=20000, n=256, seed=71):
    X = datagen.rows("walk", seed, 0, N, n)
    Q, _ = datagen.queries("walk", seed, N, n, seed + 1, 6, 4, 0.05)
    return X, Q


def _check(i, d, X, Q, k):
    ri, rd2 = oracle.bruteforce_knn(X, Q, k)
    np.testing.assert_array_equal(np.asarray(i).reshape(len(Q), k), ri)
    np.testing.assert_allclose(np.asarray(d, dtype=np.float64).reshape(len(Q), k), np.sqrt(rd2), rtol=1e-5)


def test_bounded_waits_run_out_and_the_device_stays_usable():
    for kind in (0, 1):
        assert pkg.isax_selftest_wait(kind, 1, 100000) == OK
        assert pkg.isax_selftest_wait(kind, 0, 2000) == TIMEOUT
        assert "gave up" in pkg.isax_last_error()
    X, Q = _data()
    ix = pkg.Index(torch.from_numpy(X).cuda(), leaf_size=300)
    i, d = ix.query_batch(Q, 3)
    _check(i, d, X, Q, 3)
    ix.close()


def _expect_timeout(fn):
    pkg.isax_debug_inject_timeout(1)
    with pytest.raises(pkg.ISAXError) as e:
        fn()
    assert e.value.status == TIMEOUT
    pkg.isax_debug_inject_timeout(0)


def test_a_stalled_query_surfaces_as_timeout_through_every_entry_point():
    X, Q = _data()
    ix = pkg.Index(torch.from_numpy(X).cuda(), leaf_size=300)
    k = 4
    _expect_timeout(lambda: ix.query(Q[0], k))
    i, d = ix.query(Q[0], k)  # the next query answers
    _check(i[None], d[None], X, Q[:1], k)
    _expect_timeout(lambda: ix.query_batch(Q[:3], k))    # concurrent single-query slots
    _expect_timeout(lambda: ix.query_batch(Q, k))        # chunked batch path
    _expect_timeout(lambda: ix.query_batch_bf16(Q, k))   # tensor-core filtered batch
    i, d = ix.query_batch(Q, k)
    _check(i, d, X, Q, k)
    # allocation-free entry point
    lib = pkg.lib()
    idx = np.empty(k, np.int64)
    dist = np.empty(k, np.float32)
    q = np.ascontiguousarray(Q[1])
    pkg.isax_debug_inject_timeout(1)
    assert lib.isax_query_knn_noalloc(ix.handle, q.ctypes.data, k, 0, idx.ctypes.data, dist.ctypes.data,
                                      None, None) == TIMEOUT
    assert lib.isax_query_knn_noalloc(ix.handle, q.ctypes.data, k, 0, idx.ctypes.data, dist.ctypes.data,
                                      None, None) == OK
    _check(idx[None], dist[None], X, Q[1:2], k)
    # served query: the request's status
    srv = pkg.Server(slots=2)
    srv.add(ix)
    pkg.isax_debug_inject_timeout(1)
    srv.submit(0, Q[2], k, 7)
    r = srv.poll(1, 10000)[0]
    assert r["status"] == TIMEOUT
    srv.submit(0, Q[2], k, 8)
    r = srv.poll(1, 10000)[0]
    assert r["status"] == OK
    _check(r["idx"][None], r["dist"][None], X, Q[2:3], k)
    srv.close()
    ix.close()


class _Hooks:
    """Device allocations through torch's caching allocator, counted; the
    fail_at-th allocation (0-based, counted from arm()) returns NULL."""

    def __init__(self):
        self.live = {}
        self.calls = 0
        self.fail_at = -1
        self._a = pkg.ALLOC_FN(self._alloc)
        self._f = pkg.FREE_FN(self._free)

    def _alloc(self, nbytes, stream, ctx):
        c = self.calls
        self.calls += 1
        if c == self.fail_at:
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), 0, stream or 0)
        self.live[p] = int(nbytes)
        return p

    def _free(self, ptr, stream, ctx):
        assert ptr in self.live, "free of a pointer the hook never returned"
        del self.live[ptr]
        torch.cuda.caching_allocator_delete(ptr)

    def arm(self, j):
        self.calls = 0
        self.fail_at = j

    def install(self):
        assert pkg.lib().isax_set_allocator(self._a, self._f, None) == 0

    def remove(self):
        pkg.lib().isax_set_allocator(ctypes.cast(None, pkg.ALLOC_FN), ctypes.cast(None, pkg.FREE_FN), None)


def _fails_cleanly(hooks, fn, max_calls=200, caches_on_index=False):
    """fn() under a failure at every allocation index in turn: each either
    succeeds or raises ISAX_ERR_OOM; returns how many indices failed.  A failed
    call must leave no allocation behind, except (caches_on_index) what the
    index keeps for later calls: then the bytes held after a failure never
    exceed what the successful call holds, so repeated failures accumulate
    nothing (and closing the index returns all of it)."""
    failed, held = 0, []
    start = dict(hooks.live)
    for j in range(max_calls):
        before = dict(hooks.live)
        hooks.arm(j)
        try:
            res = fn()
        except pkg.ISAXError as e:
            assert e.status == OOM, e
            if not caches_on_index:
                assert hooks.live == before, "allocations leaked after a failed call (failure at %d)" % j
            held.append(sum(hooks.live.values()) - sum(start.values()))
            failed += 1
            continue
        finally:
            hooks.arm(-1)
        ok_bytes = sum(hooks.live.values()) - sum(start.values())
        assert all(h <= ok_bytes for h in held), (held, ok_bytes)
        return failed, res
    raise AssertionError("still failing after %d allocations" % max_calls)


def test_failed_allocations_return_oom_and_leak_nothing():
    X, Q = _data()
    Xd = torch.from_numpy(X).cuda()
    hooks = _Hooks()
    hooks.install()
    try:
        # build: every allocation index in turn fails, until the build needs no more
        n_fail, ix = _fails_cleanly(hooks, lambda: pkg.Index(Xd, leaf_size=300))
        assert n_fail >= 5
        # a single query's first use and a batch's scratch, then the BF16 copy and its scratch
        k = 5
        # (the BF16 copy of the collection, made by the first BF16 batch, stays on
        # the index for later calls even when the batch's own scratch then fails)
        for fn, cached in ((lambda: ix.query(Q[0], k), False), (lambda: ix.query_batch(Q, k), False),
                           (lambda: ix.query_batch_bf16(Q, k), True)):
            _fails_cleanly(hooks, fn, caches_on_index=cached)
            i, d = ix.query_batch(Q, k)   # still answers
            _check(i, d, X, Q, k)
        held = len(hooks.live)
        assert held > 0
        ix.close()
        assert hooks.live == {}, "the index did not return everything it allocated"
        # server slots: creation fails cleanly, then serves
        ix = pkg.Index(Xd, leaf_size=300)

        def make_server():
            srv = pkg.Server(slots=2)
            try:
                srv.add(ix)
                srv.submit(0, Q[0], k, 1)
                r = srv.poll(1, 10000)[0]
            finally:
                srv.close()
            if r["status"] != OK:
                raise pkg.ISAXError(r["status"], "served query failed")
            return r
        _fails_cleanly(hooks, make_server)
        ix.close()
        assert hooks.live == {}
    finally:
        hooks.remove()
    torch.cuda.synchronize()
