"""bench.py's output contract, checked on the CPU through its reference arm
(the oracle timed on the host cores, on a small sample), and the refusal of its
GPU arm to run without a GPU (no CPU fallback)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(args, env=None, timeout=300):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=e,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    r = _bench(["--impl", "reference", "--N", "20000", "--steps", "2", "--warmup", "1", "--queries", "10"])
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "queries/s"
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["data"] == "synthetic" and d["dtype"] == "f64"
    assert "workload" in d["config"] and d["config"]["N"] == 20000
    assert "NOT larger than L2" in d["config"]["l2"]  # a small check says so
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    # a step is the timed sample; value = the step's queries / the sample's time
    # scaled to N by rows
    q = d["config"]["queries_per_step"]
    scaled = d["ms_per_step"] * d["config"]["N"] / d["sample_rows"]
    assert abs(d["ms_per_step_scaled_to_N"] - scaled) <= 1e-6 * scaled
    assert abs(q / (scaled / 1e3) - d["value"]) <= 1e-6 * d["value"]


def test_reference_arm_runs_on_rank_0_only():
    r = _bench(["--impl", "reference", "--N", "20000", "--steps", "1", "--warmup", "0"], env={"RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_gpu_arm_refuses_to_run_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = _bench(["--steps", "1", "--warmup", "3", "--N", "20000", "--no-e2e", "--no-cpu-baseline",
                "--no-serving", "--no-host-rows", "--batch", "0"], timeout=900)
    assert r.returncode != 0
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_query_roofline_arithmetic():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    # the row values the refinement read (an abandoned row counts what it read)
    acc = {"series_lb": 814_000_000, "series_refined": 7_650_000, "ed_floats": 1_200_000_000}
    r = bench.query_roofline(acc, 100, 151_497, 256, 13.1, 6701.5)
    b = 32 * 151_497 + 16 * 8_140_000 + 4 * 12_000_000
    assert r["algorithmic_bytes_per_query"] == pytest.approx(b)
    assert r["mean_query_ms"] == pytest.approx(0.131)
    assert r["achieved"] == pytest.approx(b / 0.131e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6701.5)
    assert bench.query_roofline(acc, 0, 1, 256, 0.0, 6701.5) is None


def test_traffic_entries_resolve_to_kernel_sources():
    """Every measured-traffic entry names a kernel whose source the bench can
    hash, and an entry is returned only under the hash it was taken on."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod2", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    entries = [l.split() for l in open(os.path.join(ROOT, "profiles", "traffic.txt"))
               if l.strip() and not l.startswith("#")]
    assert entries
    for label, digest, nbytes, source in (e[:4] for e in entries):
        kernel = label.split(":")[0]
        h = bench.kernel_source_hash(kernel)
        assert len(h) == 16 and float(nbytes) > 0 and source.startswith("ncu:")
        got = bench.traffic_from_profile(kernel, label)
        assert (got is not None) == (h == digest)
        if got is not None:
            assert got == (float(nbytes), source)
