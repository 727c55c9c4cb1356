"""The allocation-free query entry point (isax_query_knn_noalloc), called
through the C ABI, must give the regular query's answers.  It serves callers
that cannot allocate device memory while they query (a runtime owning the GPU
pool, a latency-critical serving thread, code recorded into a CUDA graph), so
its scratch is a fixed array inside the library that every call reuses; the
test therefore calls it twice in a row on each query.  Collected last on
purpose: it must pass both alone in a fresh process and after every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import datagen
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


def _call(fn, handle, q, k, on_device):
    """Run one query through the raw C entry point `fn`; returns numpy arrays."""
    if on_device:
        qd = torch.from_numpy(q).cuda()
        idx = torch.empty(k, dtype=torch.int64, device="cuda")
        dist = torch.empty(k, dtype=torch.float32, device="cuda")
        flags = pkg.MEM_INPUT_DEVICE | pkg.MEM_OUTPUT_DEVICE
        stream = torch.cuda.current_stream().cuda_stream
        rc = fn(handle, qd.data_ptr(), k, flags, idx.data_ptr(), dist.data_ptr(), None, stream)
        assert rc == 0, pkg.isax_last_error()
        return idx.cpu().numpy(), dist.cpu().numpy()
    qh = np.ascontiguousarray(q, dtype=np.float32)
    idx = np.empty(k, np.int64)
    dist = np.empty(k, np.float32)
    rc = fn(handle, qh.ctypes.data, k, 0, idx.ctypes.data, dist.ctypes.data, None, None)
    assert rc == 0, pkg.isax_last_error()
    return idx, dist


@pytest.mark.parametrize("in_place,split", [(False, "round-robin"), (True, "round-robin"), (False, "balanced")])
def test_noalloc_query_matches_regular_query_twice_in_a_row(in_place, split):
    N, n = 50000, 256
    X = datagen.rows("walk", 21, 0, N, n)
    Q, _ = datagen.queries("walk", 21, N, n, 22, 3, 3, 0.05)
    ix = pkg.Index(torch.from_numpy(X).cuda(), leaf_size=500, rows_in_place=in_place, split=split)
    lib = pkg.lib()
    for k in (1, 10):
        for b, q in enumerate(Q):
            on_device = bool(b % 2)
            ref_i, ref_d = _call(lib.isax_query_knn, ix.handle, q, k, on_device)
            for _ in range(2):  # the shared scratch keeps the previous call's contents
                got_i, got_d = _call(lib.isax_query_knn_noalloc, ix.handle, q, k, on_device)
                np.testing.assert_array_equal(got_i, ref_i)
                np.testing.assert_allclose(got_d, ref_d, rtol=RTOL, atol=0)
    ix.close()


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
