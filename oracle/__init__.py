"""CPU oracle for exact Euclidean k-NN with an iSAX index (FP64).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  The GPU library never
links, imports or calls it, and the two share no code (only the seeded input
generator in ``datagen/`` feeds both).

Functions and the passages they follow (Peng, Fatourou, Palpanas, "Data Series
Indexing Gone Parallel"):

- ``breakpoints``      N(0,1) quantiles splitting the y-axis into equiprobable
                       symbol regions (Section II, iSAX Representation).
- ``paa`` / ``summarize``  PAA segment means and iSAX symbols (Section II).
- ``ed2``              squared Euclidean distance (Section II, Similarity Search).
- ``lb2_series`` / ``lb2_node``  iSAX lower-bound distances used for pruning
                       (Section III, ParIS/ParIS+ and MESSI query answering).
- ``bruteforce_knn``   the definition of the exact answer: the k rows of
                       smallest distance, ties by lower row index.
- ``ISAXIndex``        ADS+-style tree (Section II, ADS+ Index) and MESSI's
                       exact search (Section III, MESSI Approach).

Every function above is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle.py`` (closed forms, library special cases, invariants and
brute force on tiny inputs); the tree shape and pruning counts are reported,
not pinned ("parity unpinned": the paper prints no tree or pruning figures).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


class Stats(ctypes.Structure):
    _fields_ = [("leaves_total", ctypes.c_int64), ("leaves_queued", ctypes.c_int64),
                ("leaves_visited", ctypes.c_int64), ("series_lb", ctypes.c_int64),
                ("series_ed", ctypes.c_int64)]


def lib():
    global _lib
    if _lib is None:
        _build.build()
        L = ctypes.CDLL(_build.LIB)
        fp = ctypes.POINTER(ctypes.c_float)
        dp = ctypes.POINTER(ctypes.c_double)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u16p = ctypes.POINTER(ctypes.c_uint16)
        i64p = ctypes.POINTER(ctypes.c_int64)
        c_int, i64 = ctypes.c_int, ctypes.c_int64
        L.or_breakpoints.argtypes = [c_int, dp]
        L.or_paa.argtypes = [fp, c_int, c_int, dp]
        L.or_symbol.argtypes = [ctypes.c_double, dp, c_int]
        L.or_symbol.restype = c_int
        L.or_summarize.argtypes = [fp, i64, c_int, c_int, c_int, dp, dp, u8p]
        L.or_ed2.argtypes = [fp, fp, c_int]
        L.or_ed2.restype = ctypes.c_double
        L.or_lb2_series.argtypes = [dp, u8p, c_int, c_int, dp, c_int]
        L.or_lb2_series.restype = ctypes.c_double
        L.or_lb2_node.argtypes = [dp, u16p, u8p, c_int, c_int, dp, c_int, c_int]
        L.or_lb2_node.restype = ctypes.c_double
        L.or_bruteforce.argtypes = [fp, i64, c_int, fp, c_int, c_int, c_int, i64p, dp]
        L.or_bruteforce.restype = c_int
        L.or_index_build.argtypes = [fp, i64, c_int, c_int, c_int, c_int]
        L.or_index_build.restype = ctypes.c_void_p
        L.or_index_free.argtypes = [ctypes.c_void_p]
        L.or_index_leaves.argtypes = [ctypes.c_void_p]
        L.or_index_leaves.restype = i64
        L.or_index_leaf_sizes.argtypes = [ctypes.c_void_p, i64p]
        L.or_index_leaf_sizes.restype = i64
        L.or_index_leaf_ids.argtypes = [ctypes.c_void_p, i64p]
        L.or_index_leaf_ids.restype = i64
        L.or_index_query.argtypes = [ctypes.c_void_p, fp, c_int, i64p, dp, ctypes.POINTER(Stats)]
        L.or_index_query.restype = c_int
        _lib = L
    return _lib


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def breakpoints(card=256):
    """beta_t = Phi^{-1}(t / card), t = 1..card-1 (FP64)."""
    out = np.empty(card - 1, dtype=np.float64)
    lib().or_breakpoints(card, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def paa(x, w=16):
    x, xp = _f32(x)
    out = np.empty(w, dtype=np.float64)
    lib().or_paa(xp, x.shape[-1], w, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def symbol(v, beta):
    beta, bp = _f64(beta)
    return lib().or_symbol(float(v), bp, len(beta) + 1)


def summarize(X, w=16, card=256, beta=None):
    """(PAA FP64 [N, w], symbols uint8 [N, w]) of the rows of X."""
    X, xp = _f32(np.atleast_2d(X))
    if beta is None:
        beta = breakpoints(card)
    beta, bp = _f64(beta)
    N, n = X.shape
    P = np.empty((N, w), dtype=np.float64)
    S = np.empty((N, w), dtype=np.uint8)
    lib().or_summarize(xp, N, n, w, card, bp, P.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       S.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return P, S


def ed2(x, q):
    x, xp = _f32(x)
    q, qp = _f32(q)
    return lib().or_ed2(xp, qp, x.shape[-1])


def lb2_series(qpaa, sym, n, beta):
    qpaa, qp = _f64(qpaa)
    sym, sp = _u8(sym)
    beta, bp = _f64(beta)
    return lib().or_lb2_series(qp, sp, len(qpaa), n, bp, len(beta) + 1)


def lb2_node(qpaa, val, bits, n, beta):
    qpaa, qp = _f64(qpaa)
    val = np.ascontiguousarray(val, dtype=np.uint16)
    bits, bitp = _u8(bits)
    beta, bp = _f64(beta)
    card = len(beta) + 1
    cbits = card.bit_length() - 1
    return lib().or_lb2_node(qp, val.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)), bitp,
                             len(qpaa), n, bp, card, cbits)


def bruteforce_knn(X, Q, k, nthreads=0):
    """Exact k-NN by a full scan: (indices int64 [B, k], squared distances FP64
    [B, k]) ascending by (distance, index)."""
    X, xp = _f32(np.atleast_2d(X))
    Q, qp = _f32(np.atleast_2d(Q))
    N, n = X.shape
    B = Q.shape[0]
    idx = np.empty((B, k), dtype=np.int64)
    d2 = np.empty((B, k), dtype=np.float64)
    rc = lib().or_bruteforce(xp, N, n, qp, B, k, nthreads,
                             idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                             d2.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise RuntimeError("or_bruteforce rc=%d" % rc)
    return idx, d2


class ISAXIndex:
    """Single-threaded ADS+-style iSAX tree with MESSI's exact k-NN search."""

    def __init__(self, X, w=16, card=256, leaf_size=2000):
        self.X, xp = _f32(np.atleast_2d(X))  # kept alive: the C index borrows it
        N, n = self.X.shape
        self.n = n
        self._h = lib().or_index_build(xp, N, n, w, card, leaf_size)
        if not self._h:
            raise ValueError("invalid index parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_index_free(h)
            self._h = None

    @property
    def leaves(self):
        return int(lib().or_index_leaves(self._h))

    def leaf_sizes(self):
        m = int(lib().or_index_leaf_sizes(self._h, None))
        out = np.empty(m, dtype=np.int64)
        lib().or_index_leaf_sizes(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
        return out

    def leaf_ids(self):
        """Member ids of every leaf, leaf after leaf in depth-first order (root
        children by key, child 0 first), ids inside a leaf in insertion order;
        split with np.cumsum(leaf_sizes())."""
        out = np.empty(self.X.shape[0], dtype=np.int64)
        m = int(lib().or_index_leaf_ids(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        assert m == len(out)
        return out

    def query(self, q, k=1):
        """(indices int64 [k], squared distances FP64 [k], Stats)."""
        q, qp = _f32(q)
        idx = np.empty(k, dtype=np.int64)
        d2 = np.empty(k, dtype=np.float64)
        st = Stats()
        rc = lib().or_index_query(self._h, qp, k, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  d2.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  ctypes.byref(st))
        if rc != 0:
            raise RuntimeError("or_index_query rc=%d" % rc)
        return idx, d2, st
