"""The C-ABI library loads, exports every entry point include/isax.h declares,
and rejects invalid arguments before touching a device.  CPU only: no compute
call reaches the GPU here."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2009_01614_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return pkg.lib()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(isax_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ["isax_build_index", "isax_query_knn", "isax_query_knn_batch", "isax_free_index",
              "isax_last_error", "isax_get_index_info", "isax_index_export", "isax_summarize",
              "isax_set_allocator"]:
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def _expect(status, code, needle):
    assert status == code, (status, pkg.isax_last_error())
    assert needle in pkg.isax_last_error()


def test_build_rejects_bad_arguments(lib):
    X = np.zeros((4, 32), np.float32)
    out = ctypes.c_void_p()
    p = pkg.BuildParams(16, 256, 10, 0)
    bp = ctypes.byref(p)
    ptr = X.ctypes.data
    _expect(lib.isax_build_index(ptr, 4, 32, bp, None, None), 1, "out is NULL")
    _expect(lib.isax_build_index(None, 4, 32, bp, None, ctypes.byref(out)), 1, "series is NULL")
    _expect(lib.isax_build_index(ptr, 0, 32, bp, None, ctypes.byref(out)), 1, "N must be")
    _expect(lib.isax_build_index(ptr, 1 << 32, 32, bp, None, ctypes.byref(out)), 1, "N must be")
    for n in [0, 8, 24, 4112]:
        _expect(lib.isax_build_index(ptr, 4, n, bp, None, ctypes.byref(out)), 1, "n must be")
    for card in [0, 1, 3, 512]:
        q = pkg.BuildParams(16, card, 10, 0)
        _expect(lib.isax_build_index(ptr, 4, 32, ctypes.byref(q), None, ctypes.byref(out)), 1,
                "cardinality")
    q = pkg.BuildParams(8, 256, 10, 0)
    _expect(lib.isax_build_index(ptr, 4, 32, ctypes.byref(q), None, ctypes.byref(out)), 1, "w must be 16")
    q = pkg.BuildParams(16, 256, 0, 0)
    _expect(lib.isax_build_index(ptr, 4, 32, ctypes.byref(q), None, ctypes.byref(out)), 1, "leaf_size")
    q = pkg.BuildParams(16, 256, 10, 32)
    _expect(lib.isax_build_index(ptr, 4, 32, ctypes.byref(q), None, ctypes.byref(out)), 1, "mem_flags")
    # the balanced split is a known flag, alone and with the row stores: argument checks pass it
    for fl in (pkg.BUILD_SPLIT_BALANCED, pkg.BUILD_SPLIT_BALANCED | pkg.BUILD_ROWS_HOST):
        q = pkg.BuildParams(16, 256, 10, fl)
        st = lib.isax_build_index(ptr, 4, 32, ctypes.byref(q), None, ctypes.byref(out))
        assert st != 1 or "mem_flags" not in pkg.isax_last_error(), pkg.isax_last_error()
        if st == 0:
            pkg.isax_free_index(out.value)
    # rows read in place need device-resident series, and exclude rows in host memory
    q = pkg.BuildParams(16, 256, 10, pkg.BUILD_ROWS_IN_PLACE)
    _expect(lib.isax_build_index(ptr, 4, 32, ctypes.byref(q), None, ctypes.byref(out)), 1,
            "ISAX_MEM_INPUT_DEVICE")
    q = pkg.BuildParams(16, 256, 10, pkg.BUILD_ROWS_IN_PLACE | pkg.BUILD_ROWS_HOST | pkg.MEM_INPUT_DEVICE)
    _expect(lib.isax_build_index(ptr, 4, 32, ctypes.byref(q), None, ctypes.byref(out)), 1,
            "exclude each other")
    _expect(lib.isax_build_index(ptr + 4, 4, 32, bp, None, ctypes.byref(out)), 1, "aligned")
    assert out.value is None


def test_query_rejects_bad_arguments(lib):
    q = np.zeros(32, np.float32)
    i = np.zeros(4, np.int64)
    d = np.zeros(4, np.float32)
    _expect(lib.isax_query_knn(None, q.ctypes.data, 1, 0, i.ctypes.data, d.ctypes.data, None, None),
            1, "index is NULL")
    _expect(lib.isax_query_knn_batch(None, q.ctypes.data, 1, 1, 0, i.ctypes.data, d.ctypes.data,
                                     None, None), 1, "index is NULL")
    _expect(lib.isax_get_index_info(None, None), 1, "NULL")
    _expect(lib.isax_index_export(None, None, None, None, None, None), 1, "NULL")
    lib.isax_free_index(None)  # no-op


def test_summarize_and_allocator_validation(lib):
    X = np.zeros((4, 32), np.float32)
    _expect(lib.isax_summarize(X.ctypes.data, 4, 20, 256, 0, None, None, None), 1, "n must be")
    _expect(lib.isax_summarize(X.ctypes.data, 4, 32, 6, 0, None, None, None), 1, "cardinality")
    _expect(lib.isax_set_allocator(pkg.ALLOC_FN(lambda *a: 0), ctypes.cast(None, pkg.FREE_FN), None),
            1, "both hooks")
    assert lib.isax_set_allocator(ctypes.cast(None, pkg.ALLOC_FN), ctypes.cast(None, pkg.FREE_FN),
                                  None) == 0


def test_product_path_has_no_oracle_dependency():
    for dirpath, _, files in os.walk(os.path.join(ROOT, "paper_2009_01614_gb300")):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.replace("Oracle", "").lower() or f.endswith(".md"), f


def test_tc_selftest_validation(lib):
    a = np.zeros((128, 256), np.uint16)
    _expect(lib.isax_tc_selftest(a.ctypes.data, a.ctypes.data, 24, a.ctypes.data, None), 1,
            "multiple of 16")
    _expect(lib.isax_tc_selftest(None, a.ctypes.data, 32, a.ctypes.data, None), 1, "NULL")


def test_server_argument_validation(lib):
    assert lib.isax_server_create(None, None) == 1
    p = pkg.ServerParams(-1, 0)
    h = ctypes.c_void_p()
    assert lib.isax_server_create(ctypes.byref(p), ctypes.byref(h)) == 1
    p = pkg.ServerParams(300, 0)
    assert lib.isax_server_create(ctypes.byref(p), ctypes.byref(h)) == 1
    assert lib.isax_server_submit(None, 0, None, 1, 0) == 1
    assert lib.isax_server_add_collection(None, None, None) == 1
    assert lib.isax_server_poll(None, None, None, None, 1, 1, 0) == -1
    assert lib.isax_server_get_info(None, None) == 1
    lib.isax_server_destroy(None)  # no-op
    assert lib.isax_server_clock() > 0


def test_failure_check_entry_points_validate_arguments(lib):
    # rejected before any device work
    _expect(lib.isax_selftest_wait(2, 0, 10, None), 1, "kind must be")
    _expect(lib.isax_selftest_wait(0, 0, 0, None), 1, "max_polls")
    _expect(lib.isax_debug_inject_timeout(-1), 1, "queries must be")
    assert lib.isax_debug_inject_timeout(0) == 0


def test_exact_d2_validates_arguments(lib):
    q = np.zeros(32, np.float32)
    i = np.zeros(4, np.int64)
    d = np.zeros(4, np.float64)
    _expect(lib.isax_exact_d2(None, q.ctypes.data, 1, 1, 0, i.ctypes.data, d.ctypes.data, None), 1,
            "index is NULL")
