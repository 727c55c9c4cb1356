"""The bounds-checked build (-DISAX_CHECKS): its kernels verify that every
position, row and list entry they touch lies inside its array, and record a
violation in a device word.  A small workload of each query path runs on it,
answers are compared with the CPU oracle, and the word must stay 0.  Runs in a
child process, which loads the checked library in place of the normal one."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, os, sys
sys.path.insert(0, os.environ["ROOT"])
import importlib
import numpy as np
import torch
import datagen, oracle
import paper_2009_01614_gb300 as pkg
b = importlib.import_module("paper_2009_01614_gb300.build")
pkg._build.LIB = b.build_checked()
pkg._lib = None
lib = pkg.lib()
lib.isax_checks_enabled.restype = __import__("ctypes").c_int32
word = __import__("ctypes").c_uint32(0)
out = {"enabled": lib.isax_checks_enabled(), "cases": []}
def check(i, d, X, Q, k):
    ri, rd2 = oracle.bruteforce_knn(X, Q, k)
    ok = np.array_equal(np.asarray(i).reshape(len(Q), k), ri) and np.allclose(
        np.asarray(d, dtype=np.float64).reshape(len(Q), k), np.sqrt(rd2), rtol=1e-5, atol=0)
    return bool(ok)
torch.cuda.set_device(0)
for kind, N, n, card, leaf in [("walk", 30000, 256, 256, 300), ("sine", 12000, 128, 16, 200), ("walk", 5000, 48, 256, 100)]:
    X = datagen.rows(kind, 81, 0, N, n)
    Q, _ = datagen.queries(kind, 81, N, n, 82, 6, 6, 0.05)
    for in_place in (False, True):
        ix = pkg.Index(torch.from_numpy(X).cuda(), cardinality=card, leaf_size=leaf, rows_in_place=in_place)
        k = 5
        single = [ix.query(q, k) for q in Q]
        res = {"kind": kind, "n": n, "in_place": in_place,
               "single": check([s[0] for s in single], [s[1] for s in single], X, Q, k)}
        i, d = ix.query_batch(Q, k)
        res["batch"] = check(i, d, X, Q, k)
        flat = [ix.query_flat(q, k) for q in Q]
        res["flat"] = check([s[0] for s in flat], [s[1] for s in flat], X, Q, k)
        if n % 64 == 0:
            i, d = ix.query_batch_bf16(Q, k)
            res["bf16"] = check(i, d, X, Q, k)
        ix.close()
        torch.cuda.synchronize()
        assert lib.isax_check_word(__import__("ctypes").byref(word)) == 0
        res["check_word"] = word.value
        out["cases"].append(res)
print(json.dumps(out))
'''


def test_checked_build_answers_exactly_and_records_no_violation():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    env = dict(os.environ)
    env["ROOT"] = ROOT
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["enabled"] == 1
    assert len(out["cases"]) == 6
    for c in out["cases"]:
        assert c["check_word"] == 0, c
        assert all(v for key, v in c.items() if key in ("single", "batch", "flat", "bf16")), c
