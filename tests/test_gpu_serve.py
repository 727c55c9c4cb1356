"""The resident query server (isax_server_*): several collections of different
series lengths stay on the device; requests with different k arrive alone or in
a mix, are admitted into in-flight slots as slots and candidate memory free up,
and every answer equals the single-query answer (and the oracle's)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import datagen
import oracle
import paper_2009_01614_gb300 as pkg

pytestmark = pytest.mark.gpu

RTOL = 1e-5
COLLS = [("walk", 10, 30_000, 256, 800), ("walk", 11, 40_000, 128, 1000), ("walk", 12, 8_000, 1024, 300)]


@pytest.fixture(scope="module")
def collections():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    out = []
    for c, (kind, seed, N, n, leaf) in enumerate(COLLS):
        X = datagen.rows(kind, seed, 0, N, n)
        # the server holds indexes of both kinds: rows copied, rows read in place
        out.append((X, pkg.Index(torch.from_numpy(X).cuda(), leaf_size=leaf, rows_in_place=c % 2 == 1)))
    yield out
    for _, ix in out:
        ix.close()


def make_requests(collections, count, seed):
    """Config-4 style: collection uniform, k in {1, 10, 100}, half fresh walks,
    half members with noise sigma ~ U[0.01, 0.5]."""
    rng = np.random.default_rng(seed)
    reqs = []
    for t in range(count):
        c = int(rng.integers(len(collections)))
        kind, dseed, N, n, _ = COLLS[c]
        k = int(rng.choice([1, 10, 100]))
        if rng.random() < 0.5:
            q = datagen.rows(kind, 1000 + seed, t, 1, n)[0]
        else:
            q = datagen.queries(kind, dseed, N, n, 2000 + seed * 1000 + t, 0, 1,
                                float(rng.uniform(0.01, 0.5)))[0][0]
        reqs.append((t, c, k, q))
    return reqs


def collect(srv, count, timeout_polls=2000):
    got = {}
    for _ in range(timeout_polls):
        for r in srv.poll(64, wait_ms=50):
            got[r["tag"]] = r
        if len(got) == count:
            break
    assert len(got) == count
    return got


def test_alone_equals_mixed_equals_single_query(collections):
    reqs = make_requests(collections, 90, 1)
    srv = pkg.Server(slots=12)
    for _, ix in collections:
        srv.add(ix)
    alone = {}
    for t, c, k, q in reqs:
        srv.submit(c, q, k, t)
        alone.update(collect(srv, 1))
    srv2 = pkg.Server(slots=12)
    for _, ix in collections:
        srv2.add(ix)
    for t, c, k, q in reqs:
        srv2.submit(c, q, k, t)
    mixed = collect(srv2, len(reqs))
    assert srv2.info()["max_in_flight"] > 1  # the mix really overlapped
    for t, c, k, q in reqs:
        a, m = alone[t], mixed[t]
        assert a["status"] == 0 and m["status"] == 0
        np.testing.assert_array_equal(m["idx"], a["idx"])
        np.testing.assert_array_equal(m["dist"], a["dist"])
        i1, d1 = collections[c][1].query(q, k)
        np.testing.assert_array_equal(m["idx"], i1)
        np.testing.assert_array_equal(m["dist"], d1)
        assert a["submit_s"] <= a["start_s"] <= a["done_s"]
    # a sample against the oracle
    for t, c, k, q in reqs[::9]:
        X = collections[c][0]
        ri, rd2 = oracle.bruteforce_knn(X, q[None, :], k)
        np.testing.assert_array_equal(mixed[t]["idx"], ri[0])
        np.testing.assert_allclose(mixed[t]["dist"], np.sqrt(rd2[0]), rtol=RTOL, atol=1e-30)
    srv.close()
    srv2.close()


def test_admission_by_candidate_memory(collections):
    """A budget that holds three k = 100 candidate buffers keeps at most three
    such requests in flight; all finish with the single-query answer."""
    per = (4096 + 256 * 100) * 12
    srv = pkg.Server(slots=16, candidate_budget=3 * per)
    for _, ix in collections:
        srv.add(ix)
    reqs = [(t, c, 100, q) for (t, c, _, q) in make_requests(collections, 30, 2)]
    for t, c, k, q in reqs:
        srv.submit(c, q, k, t)
    got = collect(srv, len(reqs))
    info = srv.info()
    assert 1 <= info["max_in_flight"] <= 3 and info["reserved_bytes"] == 0
    for t, c, k, q in reqs:
        i1, d1 = collections[c][1].query(q, k)
        np.testing.assert_array_equal(got[t]["idx"], i1)
        np.testing.assert_array_equal(got[t]["dist"], d1)
    srv.close()


def test_candidate_overflow_reruns_in_the_server():
    N, n = 200_000, 64
    ix = pkg.Index(torch.zeros((N, n), dtype=torch.float32, device="cuda"), leaf_size=2000)
    srv = pkg.Server(slots=2)
    srv.add(ix)
    srv.submit(0, np.zeros(n, np.float32), 3, 7)
    r = collect(srv, 1)[7]
    assert r["status"] == 0 and r["reruns"] >= 1
    assert r["idx"].tolist() == [0, 1, 2] and r["dist"].tolist() == [0.0, 0.0, 0.0]
    srv.close()
    ix.close()


def test_invalid_requests(collections):
    srv = pkg.Server(slots=2)
    srv.add(collections[0][1])
    q = np.zeros(256, np.float32)
    with pytest.raises(pkg.ISAXError):
        srv.submit(1, q, 1, 0)          # no such collection
    with pytest.raises(pkg.ISAXError):
        srv.submit(0, q, 0, 0)          # k out of range
    bad = datagen.rows("walk", 10, 0, 1, 256)[0].copy()
    bad[3] = np.nan
    srv.submit(0, bad, 1, 5)            # rejected on the device
    r = collect(srv, 1)[5]
    assert r["status"] == 1
    with pytest.raises(pkg.ISAXError):
        srv.add(collections[1][1])      # after the first submit
    srv.close()
