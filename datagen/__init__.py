"""Seeded synthetic inputs shared by the CPU oracle and the GPU path.

Every row is a pure function of (seed, row index), generated bit-identically on
the host (``libdghost.so``) and on the device (``libdgcuda.so``); see
``dg_core.h`` for the generator and the workload recipes.  This module holds
none of the indexing method's arithmetic.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_host = None
_cuda = None


def _host_lib():
    global _host
    if _host is None:
        if not os.path.exists(_build.HOST_LIB):
            _build.build(cuda=False)
        lib = ctypes.CDLL(_build.HOST_LIB)
        i64, u64, c_int = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int
        fp = ctypes.POINTER(ctypes.c_float)
        for name in ("dg_host_random_walks", "dg_host_sinusoids"):
            f = getattr(lib, name)
            f.argtypes = [u64, i64, i64, c_int, fp, c_int]
            f.restype = c_int
        lib.dg_host_rows_at.argtypes = [c_int, u64, ctypes.POINTER(ctypes.c_int64), i64, c_int, fp,
                                        c_int]
        lib.dg_host_rows_at.restype = c_int
        lib.dg_host_noisy.argtypes = [fp, u64, i64, i64, c_int, ctypes.POINTER(ctypes.c_double), fp]
        lib.dg_host_noisy.restype = c_int
        lib.dg_host_pick_members.argtypes = [u64, i64, i64, u64, ctypes.POINTER(ctypes.c_int64)]
        lib.dg_host_pick_members.restype = None
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.dg_host_philox.argtypes = [u32p, u32p, u32p]
        lib.dg_host_ln.argtypes = [ctypes.c_double]
        lib.dg_host_ln.restype = ctypes.c_double
        dp = ctypes.POINTER(ctypes.c_double)
        lib.dg_host_sincos_turns.argtypes = [ctypes.c_double, dp, dp]
        lib.dg_host_normal_pair.argtypes = [u64, u64, ctypes.c_uint32, ctypes.c_uint32, dp, dp]
        _host = lib
    return _host


def _cuda_lib():
    global _cuda
    if _cuda is None:
        if not os.path.exists(_build.CUDA_LIB):
            raise RuntimeError("device generator not built: run __graft_entry__.build()")
        lib = ctypes.CDLL(_build.CUDA_LIB)
        for name in ("dg_cuda_random_walks", "dg_cuda_sinusoids"):
            f = getattr(lib, name)
            f.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                          ctypes.c_void_p, ctypes.c_void_p]
            f.restype = ctypes.c_int
        _cuda = lib
    return _cuda


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


KINDS = ("walk", "sine")


def rows(kind, seed, row0, count, n, nthreads=0):
    """Rows [row0, row0+count) of collection (kind, seed) as float32 [count, n]."""
    out = np.empty((count, n), dtype=np.float32)
    if count == 0:
        return out
    lib = _host_lib()
    f = lib.dg_host_random_walks if kind == "walk" else lib.dg_host_sinusoids
    rc = f(seed, row0, count, n, _fptr(out), nthreads)
    if rc != 0:
        raise RuntimeError("dg_host rows failed rc=%d" % rc)
    return out


def rows_at(kind, seed, idx, n, nthreads=0):
    """Arbitrary rows (by index, any order) of a collection, regenerated."""
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64).ravel())
    out = np.empty((len(idx), n), dtype=np.float32)
    if len(idx) == 0:
        return out
    rc = _host_lib().dg_host_rows_at(0 if kind == "walk" else 1, seed,
                                     idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(idx),
                                     n, _fptr(out), nthreads)
    if rc != 0:
        raise RuntimeError("dg_host_rows_at failed rc=%d" % rc)
    return out


def rows_device(kind, seed, row0, count, n, dev_ptr, stream_ptr=0):
    """Fill a device buffer (float32 [count, n], 16-byte aligned) with the same rows."""
    lib = _cuda_lib()
    f = lib.dg_cuda_random_walks if kind == "walk" else lib.dg_cuda_sinusoids
    rc = f(seed, row0, count, n, ctypes.c_void_p(dev_ptr), ctypes.c_void_p(stream_ptr))
    if rc != 0:
        raise RuntimeError("dg_cuda rows failed rc=%d" % rc)


def noisy(members, qseed, qid0, sigma):
    """znorm(members[b] + sigma[b] * N(0,1)) with noise stream (qseed, qid0 + b)."""
    members = np.ascontiguousarray(members, dtype=np.float32)
    B, n = members.shape
    sig = np.ascontiguousarray(np.broadcast_to(np.asarray(sigma, dtype=np.float64), (B,)))
    out = np.empty_like(members)
    rc = _host_lib().dg_host_noisy(_fptr(members), qseed, qid0, B, n,
                                   sig.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _fptr(out))
    if rc != 0:
        raise RuntimeError("dg_host_noisy failed rc=%d" % rc)
    return out


def pick_members(qseed, qid0, count, N):
    out = np.empty(count, dtype=np.int64)
    _host_lib().dg_host_pick_members(qseed, qid0, count, N,
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return out


def queries(kind, data_seed, N, n, qseed, n_fresh, n_member, sigma):
    """Query workload: n_fresh fresh rows of (kind, qseed), then n_member noisy
    copies of uniformly picked members of collection (kind, data_seed).
    Returns (Q float32 [n_fresh + n_member, n], member index or -1 per query)."""
    fresh = rows(kind, qseed, 0, n_fresh, n)
    qid0 = n_fresh
    pick = pick_members(qseed, qid0, n_member, N)
    members = rows_at(kind, data_seed, pick, n) if n_member else np.empty((0, n), np.float32)
    noisy_q = noisy(members, qseed, qid0, sigma) if n_member else members
    Q = np.concatenate([fresh, noisy_q], axis=0)
    src = np.concatenate([np.full(n_fresh, -1, np.int64), pick])
    return Q, src


# building blocks, exposed for the generator's own tests
def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    _host_lib().dg_host_philox(c, k, o)
    return [int(v) for v in o]


def ln(x):
    return _host_lib().dg_host_ln(float(x))


def sincos_turns(u):
    s, c = ctypes.c_double(), ctypes.c_double()
    _host_lib().dg_host_sincos_turns(float(u), ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def normal_pair(seed, row, draw, tag=0):
    a, b = ctypes.c_double(), ctypes.c_double()
    _host_lib().dg_host_normal_pair(seed, row, draw, tag, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value
