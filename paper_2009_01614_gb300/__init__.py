"""Python binding of libisaxgpu.so, the sm_103a exact k-NN engine over data
series with an iSAX index (Peng, Fatourou, Palpanas, "Data Series Indexing Gone
Parallel": ParIS / ParIS+ / MESSI).

The C entry points are re-exported under their own names (``isax_build_index``,
``isax_query_knn``, ...) with argument marshalling only; ``Index`` is a small
convenience wrapper over them for numpy arrays and torch tensors.  Every step of
the build and of the query runs in the library's CUDA kernels; there is no CPU
fallback, and importing the binding fails loudly when the library is missing.
"""
import ctypes
import os

from . import build as _build

__all__ = [
    "ISAXError", "BuildParams", "QueryStats", "IndexInfo", "Index", "MEM_INPUT_DEVICE",
    "MEM_OUTPUT_DEVICE", "W", "MAX_K", "lib", "build",
    "isax_build_index", "isax_query_knn", "isax_query_knn_batch", "isax_free_index",
    "isax_last_error", "isax_get_index_info", "isax_index_export", "isax_summarize",
    "isax_set_allocator", "isax_trim_memory", "isax_profile", "isax_profile_report", "isax_launch_count",
    "isax_query_knn_noalloc", "isax_tc_selftest", "isax_query_knn_batch_bf16",
    "isax_prepare_bf16", "isax_query_knn_flat", "isax_exact_d2", "isax_selftest_wait",
    "isax_debug_inject_timeout", "Server", "ServerParams", "ServerResult", "ServerInfo",
    "isax_server_create", "isax_server_add_collection", "isax_server_submit", "isax_server_poll",
    "isax_server_get_info", "isax_server_clock", "isax_server_destroy",
]

W = 16
BUILD_ROWS_HOST = 4
BUILD_ROWS_IN_PLACE = 8
BUILD_SPLIT_BALANCED = 16
MAX_K = 1024
MAX_LEN = 4096
MEM_INPUT_DEVICE = 1
MEM_OUTPUT_DEVICE = 2

STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "cuda error", 4: "timeout",
          5: "internal error"}


class ISAXError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s (%d): %s" % (STATUS.get(status, "?"), status, message))
        self.status = status
        self.message = message


class BuildParams(ctypes.Structure):
    _fields_ = [("w", ctypes.c_int32), ("cardinality", ctypes.c_int32),
                ("leaf_size", ctypes.c_int32), ("mem_flags", ctypes.c_uint32)]


class QueryStats(ctypes.Structure):
    _fields_ = [("leaves_total", ctypes.c_int64), ("leaves_queued", ctypes.c_int64),
                ("leaves_scanned", ctypes.c_int64), ("series_lb", ctypes.c_int64),
                ("series_refined", ctypes.c_int64), ("approx_series", ctypes.c_int64),
                ("candidates", ctypes.c_int64),
                ("window", ctypes.c_int64), ("approx_leaf", ctypes.c_int32),
                ("reruns", ctypes.c_int32), ("ed_floats", ctypes.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class ServerParams(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("candidate_budget", ctypes.c_int64)]


class ServerResult(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("collection", ctypes.c_int32), ("k", ctypes.c_int32),
                ("status", ctypes.c_int32), ("reruns", ctypes.c_int32),
                ("submit_s", ctypes.c_double), ("start_s", ctypes.c_double),
                ("done_s", ctypes.c_double), ("stats", QueryStats)]


class ServerInfo(ctypes.Structure):
    _fields_ = [("collections", ctypes.c_int32), ("slots", ctypes.c_int32),
                ("queued", ctypes.c_int64), ("in_flight", ctypes.c_int32),
                ("max_in_flight", ctypes.c_int32), ("reserved_bytes", ctypes.c_int64),
                ("budget_bytes", ctypes.c_int64), ("submitted", ctypes.c_int64),
                ("completed", ctypes.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class IndexInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("n", ctypes.c_int32), ("w", ctypes.c_int32),
                ("cardinality", ctypes.c_int32), ("leaf_size", ctypes.c_int32),
                ("leaves", ctypes.c_int64), ("max_leaf", ctypes.c_int32),
                ("device", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
                ("maxabs", ctypes.c_float)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


def build():
    """Compile libisaxgpu.so (sm_103a) in-tree if it is missing or stale."""
    return _build.build()


def lib():
    """The loaded C library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libisaxgpu.so is not built (%s): run paper_2009_01614_gb300.build()"
                               % _build.LIB)
        L = ctypes.CDLL(_build.LIB)
        vp, i64, i32, u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
        st = ctypes.c_int
        L.isax_set_allocator.argtypes = [ALLOC_FN, FREE_FN, vp]
        L.isax_set_allocator.restype = st
        L.isax_trim_memory.argtypes = [i32]
        L.isax_trim_memory.restype = st
        L.isax_build_index.argtypes = [vp, i64, i32, ctypes.POINTER(BuildParams), vp,
                                       ctypes.POINTER(vp)]
        L.isax_build_index.restype = st
        L.isax_query_knn.argtypes = [vp, vp, i32, u32, vp, vp, ctypes.POINTER(QueryStats), vp]
        L.isax_query_knn.restype = st
        L.isax_query_knn_batch.argtypes = [vp, vp, i32, i32, u32, vp, vp,
                                           ctypes.POINTER(QueryStats), vp]
        L.isax_query_knn_batch.restype = st
        L.isax_free_index.argtypes = [vp]
        L.isax_free_index.restype = None
        L.isax_last_error.argtypes = []
        L.isax_last_error.restype = ctypes.c_char_p
        L.isax_get_index_info.argtypes = [vp, ctypes.POINTER(IndexInfo)]
        L.isax_get_index_info.restype = st
        L.isax_index_export.argtypes = [vp, vp, vp, vp, vp, vp]
        L.isax_index_export.restype = st
        L.isax_summarize.argtypes = [vp, i64, i32, i32, u32, vp, vp, vp]
        L.isax_summarize.restype = st
        L.isax_profile.argtypes = [i32]
        L.isax_profile.restype = st
        L.isax_profile_report.argtypes = [ctypes.POINTER(KernelTime), i32]
        L.isax_profile_report.restype = i32
        L.isax_query_knn_noalloc.argtypes = [vp, vp, i32, u32, vp, vp,
                                             ctypes.POINTER(QueryStats), vp]
        L.isax_query_knn_noalloc.restype = st
        L.isax_launch_count.argtypes = []
        L.isax_launch_count.restype = ctypes.c_uint64
        L.isax_tc_selftest.argtypes = [vp, vp, i32, vp, vp]
        L.isax_tc_selftest.restype = st
        L.isax_query_knn_flat.argtypes = [vp, vp, i32, u32, vp, vp, ctypes.POINTER(QueryStats), vp]
        L.isax_query_knn_flat.restype = st
        L.isax_query_knn_batch_bf16.argtypes = [vp, vp, i32, i32, u32, vp, vp,
                                                ctypes.POINTER(QueryStats), vp]
        L.isax_query_knn_batch_bf16.restype = st
        L.isax_prepare_bf16.argtypes = [vp, vp]
        L.isax_prepare_bf16.restype = st
        L.isax_server_create.argtypes = [ctypes.POINTER(ServerParams), ctypes.POINTER(vp)]
        L.isax_server_create.restype = st
        L.isax_server_add_collection.argtypes = [vp, vp, ctypes.POINTER(i32)]
        L.isax_server_add_collection.restype = st
        L.isax_server_submit.argtypes = [vp, i32, vp, i32, ctypes.c_uint64]
        L.isax_server_submit.restype = st
        L.isax_server_poll.argtypes = [vp, ctypes.POINTER(ServerResult), vp, vp, i32, i32, i32]
        L.isax_server_poll.restype = i32
        L.isax_server_get_info.argtypes = [vp, ctypes.POINTER(ServerInfo)]
        L.isax_server_get_info.restype = st
        L.isax_server_clock.argtypes = []
        L.isax_server_clock.restype = ctypes.c_double
        L.isax_exact_d2.argtypes = [vp, vp, i32, i32, u32, vp, vp, vp]
        L.isax_exact_d2.restype = st
        L.isax_selftest_wait.argtypes = [i32, i32, i32, vp]
        L.isax_selftest_wait.restype = st
        L.isax_debug_inject_timeout.argtypes = [i32]
        L.isax_debug_inject_timeout.restype = st
        L.isax_server_destroy.argtypes = [vp]
        L.isax_server_destroy.restype = None
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise ISAXError(status, lib().isax_last_error().decode())


# ------------------------------------------------------------------ raw C ABI
def isax_trim_memory(device=0):
    """Hand the device memory cached by the library's pool back to the driver."""
    _check(lib().isax_trim_memory(int(device)))


def isax_set_allocator(alloc_fn, free_fn, ctx=None):
    _check(lib().isax_set_allocator(alloc_fn, free_fn, ctx))


def isax_build_index(series_ptr, N, n, params=None, stream=0):
    """Returns the index handle (int)."""
    out = ctypes.c_void_p()
    p = ctypes.byref(params) if params is not None else None
    _check(lib().isax_build_index(series_ptr, N, n, p, stream, ctypes.byref(out)))
    return out.value


def isax_query_knn(index, q_ptr, k, mem_flags, out_idx_ptr, out_dist_ptr, stats=None, stream=0):
    _check(lib().isax_query_knn(index, q_ptr, k, mem_flags, out_idx_ptr, out_dist_ptr,
                                ctypes.byref(stats) if stats is not None else None, stream))


def isax_query_knn_noalloc(index, q_ptr, k, mem_flags, out_idx_ptr, out_dist_ptr, stats=None,
                           stream=0):
    """The query of isax_query_knn on the library's built-in scratch: for
    callers that must not allocate device memory (see include/isax.h)."""
    _check(lib().isax_query_knn_noalloc(index, q_ptr, k, mem_flags, out_idx_ptr, out_dist_ptr,
                                        ctypes.byref(stats) if stats is not None else None,
                                        stream))


def isax_query_knn_batch(index, Q_ptr, B, k, mem_flags, out_idx_ptr, out_dist_ptr, stats=None,
                         stream=0):
    _check(lib().isax_query_knn_batch(index, Q_ptr, B, k, mem_flags, out_idx_ptr, out_dist_ptr,
                                      stats, stream))


def isax_query_knn_flat(index, q_ptr, k, mem_flags, out_idx_ptr, out_dist_ptr, stats=None, stream=0):
    _check(lib().isax_query_knn_flat(index, q_ptr, k, mem_flags, out_idx_ptr, out_dist_ptr, stats,
                                     stream))


def isax_exact_d2(index, Q_ptr, B, k, mem_flags, idx_ptr, out_d2_ptr, stream=0):
    """FP64 squared distances of rows idx[b][j] to queries Q[b], definition order."""
    _check(lib().isax_exact_d2(index, Q_ptr, B, k, mem_flags, idx_ptr, out_d2_ptr, stream))


def isax_selftest_wait(kind, satisfied, max_polls, stream=0):
    """Make a bounded device wait run out (or not); returns the status code."""
    return lib().isax_selftest_wait(kind, satisfied, max_polls, stream)


def isax_debug_inject_timeout(queries):
    _check(lib().isax_debug_inject_timeout(queries))


def isax_query_knn_batch_bf16(index, Q_ptr, B, k, mem_flags, out_idx_ptr, out_dist_ptr, stats=None,
                              stream=0):
    _check(lib().isax_query_knn_batch_bf16(index, Q_ptr, B, k, mem_flags, out_idx_ptr, out_dist_ptr,
                                           stats, stream))


def isax_prepare_bf16(index, stream=0):
    _check(lib().isax_prepare_bf16(index, stream))


def isax_free_index(index):
    lib().isax_free_index(index)


def isax_server_create(slots=0, candidate_budget=0):
    p = ServerParams(int(slots), int(candidate_budget))
    h = ctypes.c_void_p()
    _check(lib().isax_server_create(ctypes.byref(p), ctypes.byref(h)))
    return h.value


def isax_server_add_collection(server, index):
    cid = ctypes.c_int32()
    _check(lib().isax_server_add_collection(server, index, ctypes.byref(cid)))
    return cid.value


def isax_server_submit(server, collection, q_ptr, k, tag):
    _check(lib().isax_server_submit(server, collection, q_ptr, k, tag))


def isax_server_poll(server, out, idx_ptr, dist_ptr, max_results, stride, wait_ms):
    return int(lib().isax_server_poll(server, out, idx_ptr, dist_ptr, max_results, stride, wait_ms))


def isax_server_get_info(server):
    info = ServerInfo()
    _check(lib().isax_server_get_info(server, ctypes.byref(info)))
    return info


def isax_server_clock():
    return float(lib().isax_server_clock())


def isax_server_destroy(server):
    lib().isax_server_destroy(server)


def isax_last_error():
    return lib().isax_last_error().decode()


def isax_get_index_info(index):
    info = IndexInfo()
    _check(lib().isax_get_index_info(index, ctypes.byref(info)))
    return info


def isax_index_export(index, sax_ptr=None, orig_ptr=None, leaf_begin_ptr=None, env_ptr=None,
                      bp_ptr=None):
    _check(lib().isax_index_export(index, sax_ptr, orig_ptr, leaf_begin_ptr, env_ptr, bp_ptr))


def isax_summarize(series_ptr, N, n, cardinality, mem_flags, out_sax_ptr, out_paa_ptr, stream=0):
    _check(lib().isax_summarize(series_ptr, N, n, cardinality, mem_flags, out_sax_ptr,
                                out_paa_ptr, stream))


def isax_profile(mode):
    """0 off, 1 (or True) time every kernel, 2 time the index-build kernels only."""
    _check(lib().isax_profile(int(mode)))


def isax_profile_report():
    """{kernel name: (timed launches, total ms)} of the launches timed since
    isax_profile(True)."""
    n = lib().isax_profile_report(None, 0)
    arr = (KernelTime * max(n, 1))()
    n = lib().isax_profile_report(arr, n)
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(n)}


def isax_launch_count():
    return int(lib().isax_launch_count())


def isax_tc_selftest(a_ptr, b_ptr, n_cols, d_ptr, stream=0):
    """d [128][n_cols] fp32 = a [128][256] bf16 . b [n_cols][256] bf16 ^T on the
    tensor cores (device pointers)."""
    _check(lib().isax_tc_selftest(a_ptr, b_ptr, n_cols, d_ptr, stream))


# ------------------------------------------------------------------ convenience
def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _buffer(x):
    """(pointer, on_device, keepalive, shape) of a contiguous float32 array/tensor."""
    if _is_torch(x):
        import torch
        if x.dtype != torch.float32:
            raise TypeError("expected float32")
        x = x.contiguous()
        return x.data_ptr(), x.is_cuda, x, tuple(x.shape)
    import numpy as np
    a = np.ascontiguousarray(x, dtype=np.float32)
    return a.ctypes.data, False, a, a.shape


def _stream_of(t, stream):
    if stream is not None:
        return stream
    if _is_torch(t) and t.is_cuda:
        import torch
        return torch.cuda.current_stream(t.device).cuda_stream
    return 0


class Index:
    """An iSAX index resident in device memory.

    ``Index(series, cardinality=256, leaf_size=2000)`` builds from a float32
    [N, n] numpy array (host) or torch tensor (host or CUDA).  With
    ``rows_on_host=True`` the leaf-ordered rows live in pinned host memory after
    the build (ISAX_BUILD_ROWS_HOST).  With ``rows_in_place=True`` (a contiguous
    CUDA tensor) the index reads the rows in ``series`` itself and copies none
    (ISAX_BUILD_ROWS_IN_PLACE); it keeps a reference to the tensor, which must not
    be modified while the index lives.  ``split="balanced"`` forms the leaves by
    ADS+ node splitting (ISAX_BUILD_SPLIT_BALANCED) instead of the default
    round-robin split of the sorted keys."""

    def __init__(self, series, cardinality=256, leaf_size=2000, stream=None, rows_on_host=False,
                 rows_in_place=False, split="round-robin"):
        if split not in ("round-robin", "balanced"):
            raise ValueError("split must be 'round-robin' or 'balanced'")
        ptr, on_dev, keep, shape = _buffer(series)
        if len(shape) != 2:
            raise ValueError("series must be 2-D [N, n]")
        if rows_in_place and (not on_dev or keep is not series):
            raise ValueError("rows_in_place needs a contiguous float32 CUDA tensor")
        N, n = shape
        flags = ((MEM_INPUT_DEVICE if on_dev else 0) | (BUILD_ROWS_HOST if rows_on_host else 0) |
                 (BUILD_ROWS_IN_PLACE if rows_in_place else 0) |
                 (BUILD_SPLIT_BALANCED if split == "balanced" else 0))
        p = BuildParams(W, cardinality, leaf_size, flags)
        self._h = None
        self._rows = keep if rows_in_place else None
        self._h = isax_build_index(ptr, N, n, p, _stream_of(keep, stream))
        self.N, self.n = N, n
        self.cardinality, self.leaf_size, self.split = cardinality, leaf_size, split

    def close(self):
        if self._h:
            isax_free_index(self._h)
            self._h = None
        self._rows = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def info(self):
        return isax_get_index_info(self._h).as_dict()

    def export(self):
        import numpy as np
        inf = isax_get_index_info(self._h)
        sax = np.empty((inf.N, W), np.uint8)
        orig = np.empty(inf.N, np.uint32)
        lb = np.empty(inf.leaves + 1, np.uint32)
        env = np.empty((inf.leaves, 2 * W), np.uint8)
        bp = np.empty(inf.cardinality - 1, np.float32)
        isax_index_export(self._h, sax.ctypes.data, orig.ctypes.data, lb.ctypes.data,
                          env.ctypes.data, bp.ctypes.data)
        return {"sax": sax, "orig": orig, "leaf_begin": lb, "env": env, "breakpoints": bp}

    def query(self, q, k=1, stats=False, stream=None):
        """Exact k-NN of one query: (indices int64 [k], distances float32 [k]
        [, stats dict]).  A CUDA tensor query returns CUDA tensors."""
        return self._run(q, k, stats, stream, batch=False)

    def query_batch(self, Q, k=1, stats=False, stream=None):
        return self._run(Q, k, stats, stream, batch=True)

    def query_flat(self, q, k=1, stats=False, stream=None):
        """Same answer as query, by the ParIS flat scan (every series bounded)."""
        return self._run(q, k, stats, stream, batch=False, flat=True)

    def query_batch_bf16(self, Q, k=1, stats=False, stream=None):
        """Same answers as query_batch, through the tensor-core (BF16) filter."""
        return self._run(Q, k, stats, stream, batch="bf16")

    def exact_d2(self, Q, idx, stream=None):
        """FP64 squared distances [B, k] of the original rows idx [B, k] to the
        queries Q [B, n], summed in the definition's order (isax_exact_d2):
        the values by which row shards' answers merge exactly.  CUDA tensors
        in give a CUDA float64 tensor out; otherwise a numpy array."""
        import numpy as np
        if _is_torch(Q) and Q.is_cuda and _is_torch(idx) and idx.is_cuda:
            import torch
            Qc = Q.contiguous()
            Ic = idx.to(torch.int64).contiguous()
            if Qc.dim() != 2 or Qc.shape[1] != self.n or Ic.dim() != 2 or Ic.shape[0] != Qc.shape[0]:
                raise ValueError("queries must be [B, %d] and idx [B, k]" % self.n)
            out = torch.empty(Ic.shape, dtype=torch.float64, device=Qc.device)
            isax_exact_d2(self._h, Qc.data_ptr(), Ic.shape[0], Ic.shape[1],
                          MEM_INPUT_DEVICE | MEM_OUTPUT_DEVICE, Ic.data_ptr(), out.data_ptr(),
                          _stream_of(Qc, stream))
            return out
        ptr, on_dev, keep, shape = _buffer(Q)
        if len(shape) != 2 or shape[1] != self.n:
            raise ValueError("queries must be [B, %d]" % self.n)
        if _is_torch(idx):
            idx = idx.detach().cpu().numpy()
        I = np.ascontiguousarray(idx, dtype=np.int64)
        if I.ndim != 2 or I.shape[0] != shape[0]:
            raise ValueError("idx must be [B, k]")
        B, k = I.shape
        out = np.empty((B, k), np.float64)
        if on_dev:
            keep = keep.detach().cpu().numpy()
            ptr = keep.ctypes.data
        isax_exact_d2(self._h, ptr, B, k, 0, I.ctypes.data, out.ctypes.data, _stream_of(None, stream))
        return out

    def prepare_bf16(self, stream=None):
        """Build the BF16 copy of the collection used by query_batch_bf16."""
        isax_prepare_bf16(self._h, _stream_of(None, stream))

    def _run(self, q, k, want_stats, stream, batch, flat=False):
        ptr, on_dev, keep, shape = _buffer(q)
        B = shape[0] if batch else 1
        if (batch and (len(shape) != 2 or shape[1] != self.n)) or (not batch and shape[-1] != self.n):
            raise ValueError("query length must be %d" % self.n)
        st = _stream_of(keep, stream)
        oshape = (B, k) if batch else (k,)
        if on_dev:
            import torch
            idx = torch.empty(oshape, dtype=torch.int64, device=keep.device)
            dist = torch.empty(oshape, dtype=torch.float32, device=keep.device)
            ip, dp, flags = idx.data_ptr(), dist.data_ptr(), MEM_INPUT_DEVICE | MEM_OUTPUT_DEVICE
        else:
            import numpy as np
            idx = np.empty(oshape, np.int64)
            dist = np.empty(oshape, np.float32)
            ip, dp, flags = idx.ctypes.data, dist.ctypes.data, 0
        # the counters only when asked for (NULL otherwise)
        stats = (QueryStats * B)() if want_stats else None
        one = stats[0] if want_stats else None
        if flat:
            isax_query_knn_flat(self._h, ptr, k, flags, ip, dp, one, st)
        elif batch == "bf16":
            isax_query_knn_batch_bf16(self._h, ptr, B, k, flags, ip, dp, stats, st)
        elif batch:
            isax_query_knn_batch(self._h, ptr, B, k, flags, ip, dp, stats, st)
        else:
            isax_query_knn(self._h, ptr, k, flags, ip, dp, one, st)
        if want_stats:
            s = [x.as_dict() for x in stats]
            return idx, dist, (s if batch else s[0])
        return idx, dist


def summarize(series, cardinality=256, stream=None):
    """(symbols uint8 [N, 16], PAA float32 [N, 16]) from the GPU summarisation
    kernel alone; host arrays in, host arrays out (or CUDA tensors in/out)."""
    ptr, on_dev, keep, shape = _buffer(series)
    N, n = shape
    st = _stream_of(keep, stream)
    if on_dev:
        import torch
        sax = torch.empty((N, W), dtype=torch.uint8, device=keep.device)
        paa = torch.empty((N, W), dtype=torch.float32, device=keep.device)
        isax_summarize(ptr, N, n, cardinality, MEM_INPUT_DEVICE | MEM_OUTPUT_DEVICE,
                       sax.data_ptr(), paa.data_ptr(), st)
    else:
        import numpy as np
        sax = np.empty((N, W), np.uint8)
        paa = np.empty((N, W), np.float32)
        isax_summarize(ptr, N, n, cardinality, 0, sax.ctypes.data, paa.ctypes.data, st)
    return sax, paa


class Server:
    """A resident query server over several indexes (isax_server_*): requests
    are admitted into in-flight slots as they arrive (continuous batching) and
    each returns the same answer as the single query.

    ``Server(slots=16, candidate_budget=256 << 20)``; ``add(index)`` -> id
    (before the first submit; the index must outlive the server);
    ``submit(collection, q, k, tag)`` with a host array q; ``poll(max, wait_ms)``
    -> list of dicts (tag, collection, k, status, reruns, submit_s, start_s,
    done_s, stats, idx, dist)."""

    def __init__(self, slots=16, candidate_budget=256 << 20):
        self._h = None
        self._h = isax_server_create(slots, candidate_budget)
        self._indexes = []
        self._stride = 0
        self._bufs = None

    def add(self, index):
        cid = isax_server_add_collection(self._h, index._h)
        self._indexes.append(index)
        return cid

    def submit(self, collection, q, k=1, tag=0):
        import numpy as np
        q = np.ascontiguousarray(q, dtype=np.float32)
        isax_server_submit(self._h, collection, q.ctypes.data, int(k), int(tag))
        self._stride = max(self._stride, int(k))

    def poll(self, max_results=256, wait_ms=0):
        import numpy as np
        stride = max(self._stride, 1)
        if self._bufs is None or self._bufs[0] < max_results or self._bufs[1] < stride:
            self._bufs = (max_results, stride, (ServerResult * max_results)(),
                          np.empty((max_results, stride), np.int64),
                          np.empty((max_results, stride), np.float32))
        _, st, out, idx, dist = self._bufs
        m = isax_server_poll(self._h, out, idx.ctypes.data, dist.ctypes.data, max_results, st,
                             int(wait_ms))
        res = []
        for i in range(m):
            r = out[i]
            res.append({"tag": int(r.tag), "collection": int(r.collection), "k": int(r.k),
                        "status": int(r.status), "reruns": int(r.reruns),
                        "submit_s": r.submit_s, "start_s": r.start_s, "done_s": r.done_s,
                        "stats": r.stats.as_dict(),
                        "idx": idx[i, :r.k].copy(), "dist": dist[i, :r.k].copy()})
        return res

    def info(self):
        return isax_server_get_info(self._h).as_dict()

    @staticmethod
    def clock():
        return isax_server_clock()

    def close(self):
        if self._h is not None:
            isax_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
