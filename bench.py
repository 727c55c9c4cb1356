#!/usr/bin/env python3
"""Benchmark: exact k-NN over an in-memory data-series collection with the
GPU iSAX index.

Workload (one "step" = the whole hot path once): build the index over
100,000,000 z-normalised random walks of length 256 fp32 (w = 16, cardinality
256, leaf size 2000: PAA + SAX summarisation, radix bucketing, leaves, SAX
words and ids into leaf order, envelopes), then answer 100 exact 1-NN queries
one by one (90 fresh random walks + 10 collection members with N(0, 0.01^2)
noise, re-normalised).  The collection is generated on the device by the seeded
generator before timing and is resident in HBM when the timed region starts;
it is larger than L2, and every build streams all of it.  By default the index
reads the rows in the collection array itself (`--rows in-place`: the paper's
in-memory layout, leaves hold iSAX words and row ids); `--rows copy` makes
every build also copy the rows into leaf order, and the JSON line reports that
variant too (`rows_copied`).

Printed JSON line: `value` = queries per second of the whole job (all ranks'
queries / wall time of the timed steps, builds included); `e2e` = the same job
through the C ABI with host buffers (the 102.4 GB collection copied from pinned
host memory by every build, queries and answers through host memory);
`roofline` = the dominant kernel's algorithmic bytes per launch / its mean
CUDA-event duration; `scan_roofline` = the same for a single query's
lower-bound scan and refinement, one launch (16 B per series bounded + 4 B
per row value refined; MESSI queries here, the ParIS flat scan under
`ablation_flat_scan`); `query_roofline` = a
whole query's algorithmic bytes (leaf envelopes, SAX words bounded, rows
refined) over its mean latency; `cpu_baseline` = the CPU oracle's FP64 brute
force on a sample of the same workload.  `--impl reference` times that oracle
alone.

With --gpus N > 1 (torchrun, one process per GPU) the collection is N times
larger and sharded by rows: rank r holds rows [r N, (r + 1) N) of the one
seeded collection (N = --N per rank) and builds its own index over them; every
query is answered on every shard, each rank attaches the FP64 squared distance
of its k answers (isax_exact_d2), one NCCL all-gather per step carries every
query's k (row, distance, squared distance) triples of all ranks, and each rank
merges them by (FP64 squared distance, global row): the exact answer over the
whole collection.  Per-GPU work is fixed as N grows ("scaling": "weak"); `value`
counts each query once.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact k-NN queries/s @100M x256 vs plain path; p50/p99 latency; % HBM roofline"
UNIT = "queries/s"
HBM_FALLBACK = 6800.0


L2_BYTES = 129 * 1000 * 1000  # GB300 L2 (129 MB)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--N", type=int, default=100_000_000)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--queries", type=int, default=100)
    ap.add_argument("--k", type=int, default=1)
    ap.add_argument("--leaf", type=int, default=2000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-rows", type=int, default=4_000_000)
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving leg (three resident collections, Poisson arrivals)")
    ap.add_argument("--serve-scale", type=float, default=1.0,
                    help="serving workload: scale the three collections' sizes (1.0: 40M x 256, "
                         "80M x 128, 10M x 1024)")
    ap.add_argument("--serve-requests", type=int, default=3000,
                    help="serving workload: requests per arrival rate")
    ap.add_argument("--no-hardness", action="store_true",
                    help="skip the query-hardness leg (50M sinusoid series, member queries by noise level)")
    ap.add_argument("--no-floor", action="store_true",
                    help="skip the measured GPU brute-force floor and the host round-trip latency")
    ap.add_argument("--no-host-rows", action="store_true",
                    help="skip the leg with the index's rows in host memory")
    ap.add_argument("--workload", choices=["walk", "hardness", "serving"], default="walk",
                    help="hardness: the sinusoid collection, member queries by noise level and k")
    ap.add_argument("--rows", choices=["in-place", "copy"], default="in-place",
                    help="in-place: the index reads the rows in the collection array by row id "
                         "(nothing copied); copy: each build also copies the rows into leaf order")
    ap.add_argument("--batch", type=int, default=1024,
                    help="batched leg: time the plain and the BF16-filtered batch paths on "
                         "batches of this size and of 4x this size, k = 1 and 10 (0: skip)")
    return ap.parse_args()


def workload_config(a, world=1):
    return {
        "workload": "random-walk collection %d x %d fp32 z-normalised (seed = rank), iSAX w=16 "
                    "card=256 leaf=%d; per step: full index build + %d exact %d-NN queries "
                    "(%d fresh walks + %d noisy members, sigma 0.01)" % (
                        a.N, a.n, a.leaf, a.queries, a.k, a.queries - a.queries // 10,
                        a.queries // 10),
        "N": a.N, "n": a.n, "w": 16, "cardinality": 256, "leaf_size": a.leaf, "k": a.k,
        "rows": ("read in place in the collection array by row id (leaves hold iSAX words and "
                 "row ids)" if a.rows == "in-place" else "copied into leaf order by every build"),
        "queries_per_step": a.queries,
        "gpus_sharing_the_collection": world,
        "collection_rows": a.N * world,
        "l2": ("inputs larger than L2: the %.1f GB collection is streamed by every build"
               % (a.N * a.n * 4 / 1e9) if a.N * a.n * 4 > L2_BYTES else
               "inputs NOT larger than L2 (%.3f GB collection): a small check, not a bench value"
               % (a.N * a.n * 4 / 1e9)),
        "parallelism": ("row shards of one %d x %d collection, one per GPU; one all-gather of every "
                        "query's k (row, distance, FP64 squared distance) per step, exact merge" % (a.N * world, a.n)
                        if world > 1 else "one GPU"),
    }


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK, "fallback"


def make_queries(a, world):
    """The step's queries over the whole (world x N row) collection: fresh walks
    of seed 1, then members of the collection with sigma 0.01 noise."""
    import datagen
    nq_member = a.queries // 10
    Q, src = datagen.queries("walk", 0, a.N * world, a.n, 1, a.queries - nq_member, nq_member, 0.01)
    return Q, src


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.p = None
        self.path = os.path.join("/tmp", "isax_clocks_%d_%d.csv" % (os.getpid(), gpu))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu),
                                       "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def host_available_bytes():
    """MemAvailable of this host, in bytes (None if unknown)."""
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return None


# ------------------------------------------------------------------ roofline
def kernel_bytes(name, a, launches, acc):
    """Algorithmic bytes of all timed launches of a kernel (None if not modelled).
    Build kernels run once per step (rs_* and os_scatter once per radix pass); the query
    kernels' bytes come from the per-query counters: 16 B per SAX word bounded
    plus 4 B per row value the refinement read outside the approximate answer
    (q_scan_refine: the scan and the refinement in one launch; an abandoned row
    counts the part read), the leaf envelopes and the approximate answer's rows
    (q_front)."""
    N, n = a.N, a.n
    row = 4 * n
    per_launch = {
        "permute": N * (2 * row + 2 * 16 + 4 + 4),   # rows, SAX words, ids gathered
        "summarize": N * (row + 16 + 8 + 4),         # rows read; SAX, key, id written
        "rs_scatter": N * (8 + 4) * 2,               # keys and ids read and written
        "rs_hist": N * 8,
        # one-sweep pass: keys and ids read and written; the last of the 8 passes
        # of a build with the rows in place also gathers the SAX words and writes
        # them and the ids in leaf order (averaged over the 8 launches)
        "os_scatter": N * (8 + 4) * 2 + N * (16 + 16 + 4) // 8,
        "os_hist": N * 8,                            # every pass's digit histogram in one read of the keys
        "permute_sax": N * (4 + 2 * 16 + 4),         # ids read, SAX words gathered, ids written
    }
    if name in per_launch:
        return per_launch[name] * launches
    if name == "q_scan_refine":
        # SAX words bounded, and the row floats actually read outside the
        # approximate answer (early abandoning stops a row before its end)
        return 16 * acc["series_lb"] + 4 * (acc["ed_floats"] - n * acc["approx_series"])
    if name == "q_front":
        # every leaf's envelope and the approximate answer's rows
        return 32 * acc["leaves_total"] + row * acc["approx_series"]
    return None


def query_roofline(acc, n_queries, leaves, n, q_time_ms, hbm):
    """A whole query against HBM: algorithmic bytes per query = 32 per leaf
    (every leaf's envelope is bounded) + 16 per SAX word bounded + 4 per row
    value read by the refinement (approximate-answer rows included; an
    abandoned row counts the part read), over the mean CUDA-event latency of a
    query."""
    if not n_queries or not q_time_ms:
        return None
    b = (32.0 * leaves + 16.0 * acc["series_lb"] / n_queries + 4.0 * acc["ed_floats"] / n_queries)
    t = q_time_ms / n_queries / 1e3
    return {"bound": "hbm", "algorithmic_bytes_per_query": b, "mean_query_ms": t * 1e3,
            "achieved": b / t / 1e9, "peak": hbm, "unit": "GB/s", "frac": b / t / 1e9 / hbm}


def kernel_source_hash(kernel):
    """Hash of what a kernel is compiled from: the text of its __global__
    definition (`<kernel>_kernel` in the file that defines it: q_* and bq_* in
    isax_query.cu, tc_* in isax_tc.cu, the rest in isax_build.cu), of the device
    body it wraps (`<kernel>_body`, if any) and of the shared device-helper
    header."""
    import re
    kernel = {"summarize": "summarize_vec"}.get(kernel, kernel)  # launch name -> kernel name
    # a kernel whose device body carries another name (the scan's body, whose
    # refinement step it calls, is hashed with that step below)
    body_name = {"q_scan_refine": "q_series_lb"}.get(kernel, kernel)
    src = os.path.join(ROOT, "paper_2009_01614_gb300", "csrc")
    own = ("isax_query.cu" if kernel.startswith(("q_", "bq_")) else
           "isax_tc.cu" if kernel.startswith("tc_") else "isax_build.cu")
    text = open(os.path.join(src, own)).read()
    def definition(pattern):
        m = re.search(pattern, text)
        if m is None:
            return None
        i = text.index("{", m.end())
        depth = 0
        for j in range(i, len(text)):
            depth += {"{": 1, "}": -1}.get(text[j], 0)
            if depth == 0:
                return text[m.start():j + 1]
        return None

    body = definition(r"__global__[^;{]*?\b%s_kernel\s*\(" % re.escape(kernel))
    if body is None:
        raise KeyError("no __global__ definition of %s_kernel in %s" % (kernel, own))
    # a kernel that wraps a device body (shared with its batched form) is hashed with it
    inner = definition(r"__device__[^;{]*?\b%s_body\s*\(" % re.escape(body_name))
    if kernel == "q_scan_refine":
        inner = (inner or "") + (definition(r"__device__[^;{]*?\bq_refine_claimed\s*\(") or "")
    h = hashlib.sha256(body.encode() + (inner or "").encode())
    h.update(open(os.path.join(src, "isax_kernels_util.cuh"), "rb").read())
    return h.hexdigest()[:16]


def traffic_from_profile(kernel, label=None):
    """dram bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source (its hash is recorded next to the figure); label
    picks one of several workloads of the same kernel."""
    try:
        digest = kernel_source_hash(kernel)
    except KeyError:
        return None
    label = label or kernel
    prof = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(prof):
        return None
    for line in open(prof):
        parts = line.split()
        if len(parts) >= 4 and parts[0] == label and parts[1] == digest:
            return float(parts[2]), parts[3]
    return None


def scan_roofline(prof, series_lb_total, refined_floats_total, hbm, workload):
    """The HBM fraction of a single query's lower-bound scan and refinement
    (one launch, q_scan_refine): 16 B per series bounded + 4 B per row value
    the refinement read outside the approximate answer, over the traced
    launches / their summed CUDA-event time (events around each launch: a
    little above the kernel's own duration)."""
    if "q_scan_refine" not in prof:
        return None
    cnt, ms = prof["q_scan_refine"]
    sax = 16 * series_lb_total / cnt
    rows = 4 * refined_floats_total / cnt
    per_launch = sax + rows
    achieved = per_launch / (ms / cnt / 1e3) / 1e9
    tr = traffic_from_profile("q_scan_refine", "q_scan_refine:" + workload)
    return {"kernel": "q_scan_refine", "bound": "hbm", "launches": cnt, "avg_launch_ms": ms / cnt,
            "algorithmic_bytes_per_launch": per_launch, "sax_bytes_per_launch": sax,
            "row_bytes_per_launch": rows, "achieved": achieved, "peak": hbm,
            "unit": "GB/s", "frac": achieved / hbm,
            "traffic": tr[0] if tr else None, "traffic_source": tr[1] if tr else None}


# ------------------------------------------------------------------ ablation
def ablation_leg(a, X, Qd, pkg, torch, stream):
    """The step's queries answered three ways: MESSI (leaf envelopes prune
    leaves, leaves visited in bound order) and the ParIS flat scan (every series
    of the SAX array bounded in storage order) on one index, then MESSI on an
    index whose leaves come from ADS+ node splitting (the split on the most
    balanced segment) instead of the round-robin split.  Answers must agree.
    Per-query CUDA-event latency and pruning counters; for the first two, one
    more pass with every kernel traced for the lower-bound scan's HBM fraction."""
    import numpy as np
    sp = stream.cuda_stream
    in_place = a.rows == "in-place"
    ix = pkg.Index(X, cardinality=256, leaf_size=a.leaf, stream=sp, rows_in_place=in_place)
    out = {}
    answers = {}

    def measure(fn):
        fn(Qd[0], a.k, stream=sp)  # capture its graph
        lat, st_all, ans = [], [], []
        for b in range(len(Qd)):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            i, d, st = fn(Qd[b], a.k, stats=True, stream=sp)
            e1.record(stream)
            e1.synchronize()
            lat.append(e0.elapsed_time(e1))
            st_all.append(st)
            ans.append((i.cpu().numpy(), d.cpu().numpy()))
        res = {
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "queries_per_s": len(lat) / (sum(lat) / 1e3),
            "series_bounded_per_query": float(np.mean([s["series_lb"] for s in st_all])),
            "series_refined_per_query": float(np.mean([s["series_refined"] for s in st_all])),
            "leaves_scanned_per_query": float(np.mean([s["leaves_scanned"] for s in st_all])),
            "approx_series_per_query": float(np.mean([s["approx_series"] for s in st_all])),
        }
        return res, st_all, ans

    for mode in ("messi", "flat"):
        fn = ix.query if mode == "messi" else ix.query_flat
        out[mode], st_all, answers[mode] = measure(fn)
        pkg.isax_profile(1)
        for b in range(len(Qd)):
            fn(Qd[b], a.k, stream=sp)
        torch.cuda.synchronize()
        pkg.isax_profile(0)
        out[mode]["scan_roofline"] = scan_roofline(
            pkg.isax_profile_report(), sum(s["series_lb"] for s in st_all),
            sum(s["ed_floats"] - a.n * s["approx_series"] for s in st_all), peaks()[0],
            "%s_%dMx%d" % (mode, a.N // 1000000, a.n))
    out["same_answers"] = all(np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
                              for x, y in zip(answers["messi"], answers["flat"]))
    out["messi_speedup"] = out["flat"]["latency_ms"]["p50"] / out["messi"]["latency_ms"]["p50"]
    info = ix.info()
    out["messi"]["leaves"], out["messi"]["max_leaf"] = info["leaves"], info["max_leaf"]
    ix.close()

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ib = pkg.Index(X, cardinality=256, leaf_size=a.leaf, stream=sp, rows_in_place=in_place, split="balanced")
    e1.record(stream)
    e1.synchronize()
    res, _, ans = measure(ib.query)
    info = ib.info()
    res.update({"build_ms": e0.elapsed_time(e1), "leaves": info["leaves"], "max_leaf": info["max_leaf"]})
    res["same_answers"] = all(np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
                              for x, y in zip(answers["messi"], ans))
    out["messi_balanced_split"] = res
    ib.close()
    return out


# ------------------------------------------------------------------ rows copied by the build
def copy_leg(a, X, Qd, pkg, torch, stream):
    """The step with the other rows mode (by default: every build also copies
    the rows into leaf order), timed the same way: one warm-up step, then
    `steps` steps, CUDA events around the build and around the whole step, a
    host synchronisation after every query as in the main loop."""
    sp = stream.cuda_stream
    other = "copy" if a.rows == "in-place" else "in-place"
    build, total = [], []
    for it in range(a.steps + 1):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        ix = pkg.Index(X, cardinality=256, leaf_size=a.leaf, stream=sp, rows_in_place=other == "in-place")
        e1.record(stream)
        for b in range(len(Qd)):
            ix.query(Qd[b], a.k, stream=sp)
            stream.synchronize()
        e2.record(stream)
        e2.synchronize()
        ix.close()
        if it > 0:
            build.append(e0.elapsed_time(e1))
            total.append(e0.elapsed_time(e2))
    ms = sum(total) / len(total)
    return {"rows": other, "ms_per_step": ms, "value": len(Qd) / (ms / 1e3), "unit": "queries/s",
            "build_ms": sum(build) / len(build), "steps": a.steps, "warmup": 1}


# ------------------------------------------------------------------ rows in host memory
def host_rows_leg(a, X, Qd, pkg, torch, stream):
    """The step's queries on an index whose leaf-ordered rows live in pinned
    host memory (ISAX_BUILD_ROWS_HOST): bounds from the SAX words in HBM, rows
    refined over the CPU-GPU link.  Same answers as with the rows in HBM."""
    import numpy as np
    sp = stream.cuda_stream
    ref = pkg.Index(X, cardinality=256, leaf_size=a.leaf, stream=sp)
    want = [ref.query(Qd[b], a.k, stream=sp) for b in range(len(Qd))]
    ref.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ix = pkg.Index(X, cardinality=256, leaf_size=a.leaf, stream=sp, rows_on_host=True)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    ix.query(Qd[0], a.k, stream=sp)
    lat, rows_read, same = [], [], True
    for b in range(len(Qd)):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        i, d, st = ix.query(Qd[b], a.k, stats=True, stream=sp)
        e1.record(stream)
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))
        rows_read.append(st["series_refined"])
        same &= bool(torch.equal(i, want[b][0]) and torch.equal(d, want[b][1]))
    info = ix.info()
    ix.close()
    return {"build_s_incl_pinning": build_s, "device_bytes": info["device_bytes"],
            "host_bytes": a.N * a.n * 4,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "queries_per_s": len(lat) / (sum(lat) / 1e3),
            "rows_refined_per_query": float(np.mean(rows_read)),
            "same_answers_as_rows_in_hbm": same}


# ------------------------------------------------------------------ batched leg
def bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def batch_leg(a, X, pkg, torch, stream, rank):
    """Batches of B queries drawn like the single-query workload (90% fresh
    walks, 10% noisy members; seed 4), answered by the plain FP32 batch path
    (the single-query kernels launched once per chunk of queries, grid.y =
    query) and by the tensor-core filtered batch path, on the same index; both
    must return identical answers.  Device buffers in and out; times are CUDA
    events around whole batch calls; one more traced call of each gives the
    per-kernel times and the batched lower-bound scan's HBM fraction."""
    import datagen
    import numpy as np
    sp = stream.cuda_stream
    N, n = a.N, a.n
    ix = pkg.Index(X, cardinality=256, leaf_size=a.leaf, stream=sp, rows_in_place=a.rows == "in-place")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ix.prepare_bf16(stream=sp)
    prep_ms = (time.perf_counter() - t0) * 1e3
    tflops_peak, tsrc = bf16_peak()
    hbm, _ = peaks()
    runs = []

    def timed(fn, reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    for B in (a.batch, 4 * a.batch):
        Qh, _ = datagen.queries("walk", rank, N, n, 4 + 1000 * rank + B, B - B // 10, B // 10, 0.01)
        Q = torch.from_numpy(Qh).cuda()
        for k in (1, 10):
            i_p, d_p, st_p = ix.query_batch(Q, k, stats=True, stream=sp)
            i_b, d_b, st = ix.query_batch_bf16(Q, k, stats=True, stream=sp)
            identical = bool(torch.equal(i_p, i_b) and torch.equal(d_p, d_b))
            plain_ms = timed(lambda: ix.query_batch(Q, k, stream=sp), 2)
            bf16_ms = timed(lambda: ix.query_batch_bf16(Q, k, stream=sp), 3)
            pkg.isax_profile(1)
            ix.query_batch(Q, k, stream=sp)
            torch.cuda.synchronize()
            pkg.isax_profile(0)
            pprof = pkg.isax_profile_report()
            pkern = {nm: round(v[1], 4) for nm, v in sorted(pprof.items(), key=lambda kv: -kv[1][1])}
            scan = None
            if "bq_series_lb" in pprof:
                lb_ms = pprof["bq_series_lb"][1]
                lb_bytes = 16.0 * sum(s["series_lb"] for s in st_p)
                scan = {"kernel": "bq_series_lb", "bound": "hbm", "launches": pprof["bq_series_lb"][0],
                        "algorithmic_bytes": lb_bytes, "ms": lb_ms,
                        "achieved": lb_bytes / (lb_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": lb_bytes / (lb_ms / 1e3) / 1e9 / hbm}
            pkg.isax_profile(1)
            ix.query_batch_bf16(Q, k, stream=sp)
            torch.cuda.synchronize()
            pkg.isax_profile(0)
            prof = pkg.isax_profile_report()
            rows = sum(s["series_lb"] for s in st)
            kern = {nm: round(v[1], 4) for nm, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
            tf_ms = prof.get("tc_filter", (1, None))[1]
            flops = 2.0 * n * rows
            achieved = flops / (tf_ms / 1e3) / 1e12 if tf_ms else None
            runs.append({
                "B": B, "k": k, "identical_answers": identical,
                "plain_ms_per_batch": round(plain_ms, 3),
                "plain_queries_per_s": round(B / (plain_ms / 1e3), 1),
                "bf16_ms_per_batch": round(bf16_ms, 3),
                "bf16_queries_per_s": round(B / (bf16_ms / 1e3), 1),
                "speedup": round(plain_ms / bf16_ms, 2),
                "per_query": {
                    "leaves_contracted": float(np.mean([s["leaves_queued"] for s in st])),
                    "rows_contracted": rows / B,
                    "rows_rechecked_fp32": float(np.mean([s["series_refined"] - s["approx_series"]
                                                         for s in st])),
                    "reruns": int(sum(s["reruns"] for s in st)),
                },
                "plain_reruns": int(sum(s["reruns"] for s in st_p)),
                "plain_kernels_ms": pkern,
                "plain_scan_roofline": scan,
                "kernels_ms": kern,
                "tc_filter_roofline": {
                    "bound": "tensor", "unit": "TFLOP/s",
                    "achieved": achieved, "peak": tflops_peak,
                    "frac": achieved / tflops_peak if achieved else None,
                    "flops": "2 n x rows contracted (useful work; padding of tiles excluded)",
                    "bf16_copy_GB_per_s_if_read_once": (N * n * 2 / 1e9) / (tf_ms / 1e3) if tf_ms else None,
                    "hbm_peak": hbm,
                    "peak_source": "%s: MEASURED_PEAKS.json bf16_tflops (burst)" % tsrc,
                },
            })
        del Q
    ix.close()
    torch.cuda.synchronize()
    return {"prepare_bf16_ms": prep_ms, "bf16_copy_GB": N * n * 2 / 1e9,
            "queries": "config-0 style: 90% fresh walks, 10% members + N(0, 0.01) noise, seed 4",
            "runs": runs}


# ------------------------------------------------------------------ serving workload
def serving(a):
    """The serving workload alone (see serving_leg).  One JSON line."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2009_01614_gb300 as pkg
    torch.cuda.set_device(0)
    out = serving_leg(a, pkg, torch)
    out.update({"metric": "exact k-NN queries/s served (continuous batching) + p50/p99 latency",
                "unit": "queries/s", "dtype": "f32", "data": "synthetic"})
    print(json.dumps(out), flush=True)
    return 0


def serving_leg(a, pkg, torch):
    """Three resident collections (40M x 256, 80M x 128, 10M x 1024 z-normalised
    random walks, seeds 10-12, w 16, leaf 2000) behind one query server (16
    slots, 256 MiB candidate budget).  Requests arrive as a Poisson process
    (seed 20) at 200, 1000 and 5000 per second, each routed uniformly to a
    collection with k uniform in {1, 10, 100}, half fresh walks and half members
    with noise sigma ~ U[0.01, 0.5].  Latency = answer back on the host minus the
    scheduled arrival (queueing included)."""
    import numpy as np
    import datagen
    st = torch.cuda.current_stream().cuda_stream
    specs = [(10, int(40_000_000 * a.serve_scale), 256), (11, int(80_000_000 * a.serve_scale), 128),
             (12, int(10_000_000 * a.serve_scale), 1024)]
    indexes = []
    build_ms = []
    for seed, N, n in specs:
        X = torch.empty((N, n), dtype=torch.float32, device="cuda")
        datagen.rows_device("walk", seed, 0, N, n, X.data_ptr(), st)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        indexes.append(pkg.Index(X, leaf_size=a.leaf))
        torch.cuda.synchronize()
        build_ms.append((time.perf_counter() - t0) * 1e3)
        del X
        torch.cuda.empty_cache()
    rng = np.random.default_rng(20)
    R = a.serve_requests

    def requests(count, salt):
        out = []
        for t in range(count):
            c = int(rng.integers(3))
            seed, N, n = specs[c]
            k = int(rng.choice([1, 10, 100]))
            if rng.random() < 0.5:
                q = datagen.rows("walk", 100 + seed + salt, t, 1, n)[0]
            else:
                q = datagen.queries("walk", seed, N, n, 200 + seed + 1000 * salt + t, 0, 1,
                                    float(rng.uniform(0.01, 0.5)))[0][0]
            out.append((c, k, q))
        return out

    def run_rate(rate, reqs, srv):
        gaps = rng.exponential(1.0 / rate, size=len(reqs))
        sched = np.cumsum(gaps)
        got = {}
        t0 = srv.clock() + 0.05
        arrival = t0 + sched
        for i, (c, k, q) in enumerate(reqs):
            while srv.clock() < arrival[i]:
                for r in srv.poll(64, 0):
                    got[r["tag"]] = r
            srv.submit(c, q, k, i)
        while len(got) < len(reqs):
            for r in srv.poll(256, 20):
                got[r["tag"]] = r
        lat = np.array([got[i]["done_s"] - arrival[i] for i in range(len(reqs))]) * 1e3
        svc = np.array([got[i]["done_s"] - got[i]["start_s"] for i in range(len(reqs))]) * 1e3
        wall = max(r["done_s"] for r in got.values()) - arrival[0]
        assert all(r["status"] == 0 for r in got.values())
        return got, {"offered_per_s": rate, "requests": len(reqs),
                     "queries_per_s": len(reqs) / wall,
                     "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                    "mean": float(lat.mean())},
                     "in_slot_ms": {"p50": float(np.percentile(svc, 50)), "p99": float(np.percentile(svc, 99))},
                     "max_in_flight": srv.info()["max_in_flight"],
                     "reruns": int(sum(r["reruns"] for r in got.values()))}

    results = []
    identical = None
    for rate in (200, 1000, 5000):
        srv = pkg.Server(slots=16, candidate_budget=256 << 20)
        for ix in indexes:
            srv.add(ix)
        reqs = requests(min(R, int(rate * 4) + 200), rate)
        run_rate(rate, reqs[:64], srv)  # warm up: graphs captured per (slot, collection, k)
        got, res = run_rate(rate, reqs, srv)
        results.append(res)
        if rate == 5000:
            # the same requests one at a time give the same answers
            alone = pkg.Server(slots=16, candidate_budget=256 << 20)
            for ix in indexes:
                alone.add(ix)
            same = True
            for i, (c, k, q) in enumerate(reqs[:200]):
                alone.submit(c, q, k, i)
                r = alone.poll(1, 10_000)[0]
                same &= bool(np.array_equal(r["idx"], got[i]["idx"]) and
                             np.array_equal(r["dist"], got[i]["dist"]))
            identical = same
            alone.close()
        srv.close()
    out = {"workload": "3 resident collections %s (w 16, leaf %d); Poisson arrivals, collection uniform, "
                       "k in {1,10,100}, 50%% fresh / 50%% noisy members sigma U[0.01,0.5]" % (
                           ", ".join("%dx%d" % (N, n) for _, N, n in specs), a.leaf),
           "server": {"slots": 16, "candidate_budget_bytes": 256 << 20},
           "build_ms": build_ms, "rates": results,
           "mixed_equals_alone_first_200_at_5000_per_s": identical}
    for ix in indexes:
        ix.close()
    torch.cuda.synchronize()
    return out


# ------------------------------------------------------------------ CPU baseline
def cpu_baseline(a, sample_rows, n_queries=10):
    import numpy as np
    import datagen
    import oracle
    cores = len(os.sched_getaffinity(0))
    X = datagen.rows("walk", 0, 0, sample_rows, a.n)
    Q, _ = datagen.queries("walk", 0, sample_rows, a.n, 1, n_queries, 0, 0.01)
    t0 = time.perf_counter()
    oracle.bruteforce_knn(X, Q, a.k, nthreads=cores)
    t = time.perf_counter() - t0
    qps_full = n_queries / t * (sample_rows / a.N)
    return {"value": qps_full, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "FP64 brute-force k-NN (all host cores) of %d fresh random-walk queries over "
                      "the first %d rows of the collection: %.2f s; scaled to N=%d by rows"
                      % (n_queries, sample_rows, t, a.N)}


def reference_arm(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import datagen
    import oracle
    cores = len(os.sched_getaffinity(0))
    S = min(a.N, 1_000_000)
    X = datagen.rows("walk", 0, 0, S, a.n)
    Q, _ = datagen.queries("walk", 0, S, a.n, 1, a.queries - a.queries // 10, a.queries // 10, 0.01)
    for _ in range(a.warmup):
        oracle.bruteforce_knn(X, Q, a.k, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        oracle.bruteforce_knn(X, Q, a.k, nthreads=cores)
    t = time.perf_counter() - t0
    step_full = t / a.steps * (a.N / S)
    value = a.queries / step_full
    sample = ("CPU oracle (FP64 brute-force exact %d-NN, %d host cores) of the step's %d queries "
              "over a %d-row sample of the collection, %.3f s per sample step, scaled to N=%d by rows"
              % (a.k, cores, a.queries, S, t / a.steps, a.N))
    # a step is the bounded sample actually timed (so steps x ms_per_step is the
    # timed region); the value is the metric at the full N (the sample's time
    # scaled by rows)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": t / a.steps * 1e3,
            "sample_rows": S, "ms_per_step_scaled_to_N": step_full * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(a),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ query hardness
def hardness_leg(a, pkg, torch, datagen, queries_per_level=50):
    """Query hardness (the sum-of-3-sinusoids collection, 50M x 256 unless --N
    says otherwise): member queries with noise sigma in {0.01, 0.1, 0.5, 1.0},
    each answered for k in {1, 10, 100}; per (sigma, k): leaf and series
    pruning, series refined, row floats actually read by the refinement (early
    abandoning stops a row early), latency."""
    import numpy as np
    N = a.N if a.N != 100_000_000 else 50_000_000
    n = a.n
    stream = torch.cuda.current_stream()
    X = torch.empty((N, n), dtype=torch.float32, device="cuda")
    datagen.rows_device("sine", 0, 0, N, n, X.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ix = pkg.Index(X, cardinality=256, leaf_size=a.leaf)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    del X
    torch.cuda.empty_cache()
    info = ix.info()
    rows = []
    for si, sigma in enumerate([0.01, 0.1, 0.5, 1.0]):
        Q, _ = datagen.queries("sine", 0, N, n, 3 + si, 0, queries_per_level, sigma)
        Qd = torch.from_numpy(Q).cuda()
        for k in [1, 10, 100]:
            ix.query(Qd[0], k)  # its query graph
            lat, st_all = [], []
            for b in range(len(Q)):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                _, _, st = ix.query(Qd[b], k, stats=True)
                e1.record(stream)
                e1.synchronize()
                lat.append(e0.elapsed_time(e1))
                st_all.append(st)
            mean = lambda key: float(np.mean([x[key] for x in st_all]))
            rows.append({
                "sigma": sigma, "k": k,
                "leaf_pruning": 1.0 - mean("leaves_scanned") / info["leaves"],
                "series_lb_per_query": mean("series_lb"),
                "series_pruning_by_lb": 1.0 - (mean("series_refined") - mean("approx_series"))
                / max(1.0, mean("series_lb")),
                "series_refined_per_query": mean("series_refined"),
                "ed_floats_read_per_query": mean("ed_floats"),
                "ed_floats_if_rows_read_whole": mean("series_refined") * n,
                "latency_ms_p50": float(np.percentile(lat, 50)),
                "latency_ms_p99": float(np.percentile(lat, 99)),
            })
    ix.close()
    torch.cuda.synchronize()
    return {"workload": "query hardness: %d sum-of-3-sinusoid series x %d fp32, leaf %d; %d member "
                        "queries per noise level" % (N, n, a.leaf, queries_per_level),
            "build_s": build_s, "leaves": info["leaves"], "rows": rows}


def hardness(a):
    """The hardness leg alone, as one JSON line (--workload hardness)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import datagen
    import paper_2009_01614_gb300 as pkg
    torch.cuda.set_device(0)
    print(json.dumps(hardness_leg(a, pkg, torch, datagen)), flush=True)
    return 0


# ------------------------------------------------------------------ host round trip, floors
def host_latency_leg(a, X, Qh, pkg, torch, stream):
    """Single queries through the C ABI with HOST buffers: every call copies its
    1 KB query to the device and its k results back, and returns when they are
    in host memory; per-query wall-clock latency (the caller's view)."""
    import numpy as np
    sp = stream.cuda_stream
    ix = pkg.Index(X, cardinality=256, leaf_size=a.leaf, stream=sp, rows_in_place=a.rows == "in-place")
    Qp = torch.from_numpy(Qh).pin_memory().numpy()
    for b in range(3):
        ix.query(Qp[b], a.k, stream=sp)
    lat = []
    for b in range(len(Qp)):
        t0 = time.perf_counter()
        ix.query(Qp[b], a.k, stream=sp)
        lat.append((time.perf_counter() - t0) * 1e3)
    ix.close()
    return {"latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(np.mean(lat))},
            "queries_per_s": len(lat) / (sum(lat) / 1e3),
            "h2d_bytes_per_query": a.n * 4, "d2h_bytes_per_query": a.k * (8 + 4),
            "how": "wall clock around isax_query_knn with pinned host query and host outputs"}


def bruteforce_floor(a, X, Qd, torch, stream, queries=5):
    """The GPU brute-force floor, measured: every query reads the whole
    collection once (cuBLAS GEMV X q, then the smallest ||x||^2 - 2 x.q): the
    bytes a scan without an index must move.  A floor, not an exact answer."""
    norms = (X * X).sum(dim=1)
    torch.cuda.synchronize()
    times = []
    for b in range(queries + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d = norms - 2.0 * torch.mv(X, Qd[b])
        torch.argmin(d)
        e1.record(stream)
        e1.synchronize()
        if b > 0:
            times.append(e0.elapsed_time(e1))
    del norms, d
    ms = sum(times) / len(times)
    return {"ms_per_query": ms, "queries_per_s": 1e3 / ms, "bytes_per_query": a.N * a.n * 4,
            "GB_per_s": a.N * a.n * 4 / (ms / 1e3) / 1e9, "queries": queries,
            "how": "torch.mv (cuBLAS) over the resident collection + argmin, CUDA events"}


def isax_oracle_baseline(a, sample_rows=1_000_000, n_queries=10):
    """The CPU oracle's single-threaded iSAX index (ADS+ tree, MESSI-style exact
    search, FP64) on a bounded sample of the collection: seconds per exact query."""
    import datagen
    import oracle
    X = datagen.rows("walk", 0, 0, sample_rows, a.n)
    Q, _ = datagen.queries("walk", 0, sample_rows, a.n, 1, n_queries - n_queries // 10, n_queries // 10, 0.01)
    t0 = time.perf_counter()
    ix = oracle.ISAXIndex(X, 16, 256, a.leaf)
    build_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    for q in Q:
        ix.query(q, a.k)
    per_q = (time.perf_counter() - t0) / len(Q)
    return {"value": 1.0 / per_q, "unit": UNIT, "cores": 1, "kind": "oracle",
            "seconds_per_query": per_q, "build_s": build_s,
            "sample": "single-threaded FP64 iSAX index (oracle) over the first %d rows of the collection, %d "
                      "queries (not scaled: its query time grows with N)" % (sample_rows, len(Q))}


# ------------------------------------------------------------------ GPU arm
def main():
    a = parse()
    if a.impl == "reference":
        return reference_arm(a)
    if a.workload == "hardness":
        return hardness(a)
    if a.workload == "serving":
        return serving(a)

    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import datagen
    import paper_2009_01614_gb300 as pkg

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v):
        if dist is None:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    N, n, k = a.N, a.n, a.k

    # inputs: collection generated on the device (bit-identical to the host generator)
    X = torch.empty((N, n), dtype=torch.float32, device="cuda")
    # this rank's rows of the collection (all of it on one GPU)
    datagen.rows_device("walk", 0, rank * N, N, n, X.data_ptr(), sp)
    Qh, src = make_queries(a, world)
    Qd = torch.from_numpy(Qh).cuda()
    torch.cuda.synchronize()
    # the end-to-end leg's page-locked host copy of the collection (made after the
    # timed steps, before the host-rows leg page-locks 102 GB of its own: made after
    # that, it copied to the device measurably slower).  Every rank on this host
    # holds one: the leg runs only if they all fit, decided alike on every rank.
    Xh = None
    e2e_skip = None
    if not a.no_e2e:
        local_world = int(os.environ.get("LOCAL_WORLD_SIZE", "1"))
        avail = host_available_bytes()
        fits = avail is None or avail >= local_world * N * n * 4 * 1.15
        if dist is not None:
            t = torch.tensor([1.0 if fits else 0.0], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MIN)
            fits = bool(t.item() > 0)
        if not fits:
            e2e_skip = ("host memory available %.0f GB < %d ranks x %.0f GB of page-locked collection"
                        % ((avail or 0) / 1e9, local_world, N * n * 4 * 1.15 / 1e9))

    lat_ms = []
    stats_acc = {"series_lb": 0, "series_refined": 0, "approx_series": 0, "leaves_queued": 0,
                 "leaves_scanned": 0, "candidates": 0, "window": 0, "ed_floats": 0, "leaves_total": 0}

    from paper_2009_01614_gb300 import shard

    # every query goes through the C entry point with device buffers made once
    # (the per-call tensor allocations of the Python wrapper are not the query's cost)
    out_i = torch.empty((a.queries, k), dtype=torch.int64, device="cuda")
    out_d = torch.empty((a.queries, k), dtype=torch.float32, device="cuda")
    qstats = (pkg.QueryStats * a.queries)()
    dev_flags = pkg.MEM_INPUT_DEVICE | pkg.MEM_OUTPUT_DEVICE
    q_ptr = [Qd[b].data_ptr() for b in range(a.queries)]
    i_ptr = [out_i[b].data_ptr() for b in range(a.queries)]
    d_ptr = [out_d[b].data_ptr() for b in range(a.queries)]
    events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(a.queries)]

    def step(record, rows=a.rows):
        ix = pkg.Index(X, cardinality=256, leaf_size=a.leaf, stream=sp, rows_in_place=rows == "in-place")
        h = ix.handle
        for b in range(a.queries):
            e0, e1 = events[b]
            e0.record(stream)
            pkg.isax_query_knn(h, q_ptr[b], k, dev_flags, i_ptr[b], d_ptr[b], qstats[b], sp)
            e1.record(stream)
        if record:
            torch.cuda.synchronize()
            for b in range(a.queries):
                lat_ms.append(events[b][0].elapsed_time(events[b][1]))
                st = qstats[b].as_dict()
                for key in stats_acc:
                    stats_acc[key] += st[key]
        last = (out_i[-1], out_d[-1])
        if dist is not None:
            # row shards: the FP64 squared distances of this shard's answers, one
            # all-gather of every query's k triples, the exact merge
            I, D = out_i, out_d
            D2 = ix.exact_d2(Qd, I, stream=sp)
            gi, gd, _ = shard.gather_merge(I.cpu().numpy(), D.cpu().numpy(), D2.cpu().numpy(), k, rank * N,
                                           world, device=torch.device("cuda", local))
            last = (gi[-1], gd[-1])
        info = ix.info()
        ix.close()
        return info, last

    for _ in range(a.warmup):
        step(False)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = pkg.isax_launch_count()
    pkg.isax_profile(2)  # build kernels timed live; queries replay their CUDA graphs
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(a.steps):
        info, last = step(True)
    t_end.record(stream)
    torch.cuda.synchronize()
    pkg.isax_profile(False)
    clock_info = clocks.stop()
    launches = pkg.isax_launch_count() - launches0
    elapsed_ms = max_over_ranks(t_start.elapsed_time(t_end))
    barrier()
    prof = pkg.isax_profile_report()
    # one more step with every kernel timed (queries launched kernel by kernel),
    # outside the timed region, for the per-kernel table of the query path
    pkg.isax_profile(1)
    step(False)
    torch.cuda.synchronize()
    pkg.isax_profile(0)
    qprof = {nm: v for nm, v in pkg.isax_profile_report().items() if nm.startswith("q_")}

    # each query is answered once over the whole collection (its shards
    # together on N > 1 GPUs)
    total_queries = a.queries * a.steps
    value = total_queries / (elapsed_ms / 1e3)
    q_time_ms = sum(lat_ms)
    build_ms = (elapsed_ms - q_time_ms) / a.steps

    # roofline of the dominant kernel (largest share of the timed kernel time)
    hbm, peak_kind = peaks()
    dom_name, (dom_launches, dom_ms) = max(prof.items(), key=lambda kv: kv[1][1])
    algo_total = kernel_bytes(dom_name, a, dom_launches, stats_acc)
    avg_ms = dom_ms / dom_launches
    per_launch_bytes = algo_total / dom_launches if algo_total is not None else None
    achieved = per_launch_bytes / (avg_ms / 1e3) / 1e9 if per_launch_bytes else None
    tr = traffic_from_profile(dom_name)
    roof = {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": hbm,
            "unit": "GB/s", "frac": (achieved / hbm) if achieved else None,
            "traffic": tr[0] if tr else None, "traffic_source": tr[1] if tr else None,
            "algorithmic_bytes_per_launch": per_launch_bytes, "avg_launch_ms": avg_ms,
            "peak_source": "%s: MEASURED_PEAKS.json hbm_gbs (copy bandwidth)" % peak_kind
            if peak_kind == "measured" else "fallback 6800 GB/s"}
    kernels = {}
    total_kernel_ms = sum(v[1] for v in prof.values())
    # query kernels: from the extra traced step, scaled to the timed steps' launches
    qscale = a.steps
    allk = dict(prof)
    for nm, (cnt, ms) in qprof.items():
        allk[nm] = (cnt * qscale, ms * qscale)
    total_kernel_ms = sum(v[1] for v in allk.values())
    for nm, (cnt, ms) in sorted(allk.items(), key=lambda kv: -kv[1][1]):
        entry = {"launches": cnt, "total_ms": round(ms, 3), "avg_ms": round(ms / cnt, 5),
                 "share": round(ms / total_kernel_ms, 4)}
        b = kernel_bytes(nm, a, cnt, stats_acc)
        if b is not None and ms > 0:
            entry["GB_per_s"] = round(b / (ms / 1e3) / 1e9, 1)
        kernels[nm] = entry

    # the same step with the other rows mode
    rows_other = copy_leg(a, X, Qd, pkg, torch, stream)

    # the ParIS flat scan against MESSI's pruned, ordered search, same queries and index
    ablation = ablation_leg(a, X, Qd, pkg, torch, stream)


    # batched queries: the plain FP32 path against the tensor-core (BF16) filter
    batch_info = batch_leg(a, X, pkg, torch, stream, rank) if a.batch > 0 else None

    # the caller's view of a single query (host buffers: 1 KB in, k results out)
    # and the brute-force floor, measured on the resident collection
    host_rt = floor = None
    if not a.no_floor:
        host_rt = host_latency_leg(a, X, Qh, pkg, torch, stream)
        floor = bruteforce_floor(a, X, Qd, torch, stream)

    lat_sorted = sorted(lat_ms)

    def pct(p):
        if not lat_sorted:
            return None
        i = min(len(lat_sorted) - 1, int(math.ceil(p / 100.0 * len(lat_sorted))) - 1)
        return lat_sorted[max(i, 0)]

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": elapsed_ms / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(a, world),
        "roofline": roof,
        "latency_ms": {"p50": pct(50), "p99": pct(99), "mean": statistics.mean(lat_ms)},
        "query_qps": len(lat_ms) / (q_time_ms / 1e3) if q_time_ms else None,
        "latency_host_round_trip": host_rt,
        "bruteforce_floor": floor,
        "build_ms": build_ms, "build_input_GB_per_s": N * n * 4 / 1e9 / (build_ms / 1e3),
        "index": {"leaves": info["leaves"], "max_leaf": info["max_leaf"]},
        "pruning": {key + "_per_query": stats_acc[key] / max(1, len(lat_ms)) for key in stats_acc},
        "batch": batch_info,
        "rows_copied" if a.rows == "in-place" else "rows_in_place": rows_other,
        "ablation_flat_scan": ablation,
        "rows_in_host_memory": None,
        "kernels": kernels,
        "scan_roofline": scan_roofline(qprof, stats_acc["series_lb"] / a.steps,
                                       (stats_acc["ed_floats"] - n * stats_acc["approx_series"]) / a.steps, hbm,
                                       "messi_%dMx%d" % (a.N // 1000000, a.n)),
        "query_roofline": query_roofline(stats_acc, len(lat_ms), info["leaves"], n, q_time_ms, hbm),
        "gpu_launches": launches,
        "clocks": clock_info,
    }

    # ---------------------------------------------------------- end to end (host buffers)
    if e2e_skip is not None:
        out["e2e"] = {"skipped": e2e_skip}
    if not a.no_e2e and e2e_skip is None:
        # the page-locked host copy of the collection is made only now: made
        # before the timed steps, a build right after its fill once took 95 ms
        # instead of 31
        Xh = torch.empty((N, n), dtype=torch.float32, pin_memory=True)
        for r0 in range(0, N, 1 << 22):
            c = min(1 << 22, N - r0)
            Xh[r0:r0 + c].copy_(X[r0:r0 + c])
        torch.cuda.synchronize()
        del Qd
        del X
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        # the earlier legs' freed indexes and scratch stay cached in the library's pool;
        # hand them back so the collection's device copy is mapped in one piece
        pkg.isax_trim_memory(local)
        Qp = torch.from_numpy(Qh).pin_memory()
        Xh_np = Xh.numpy()
        Qp_np = Qp.numpy()

        def step_e2e():
            ix = pkg.Index(Xh_np, cardinality=256, leaf_size=a.leaf, stream=sp)
            for b in range(a.queries):
                ix.query(Qp_np[b], k, stream=sp)
            ix.close()

        for _ in range(max(1, min(a.warmup, 2))):
            step_e2e()
        # the CPU-GPU link's copy rate from this page-locked buffer (a slice of
        # up to 4 GiB, three copies timed with CUDA events), untimed, to read the
        # step time against
        rows_probe = min(N, (1 << 30) // n)
        dst = torch.empty((rows_probe, n), dtype=torch.float32, device="cuda")
        dst.copy_(Xh[:rows_probe], non_blocking=True)
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record()
        for _ in range(3):
            dst.copy_(Xh[:rows_probe], non_blocking=True)
        h1.record()
        torch.cuda.synchronize()
        h2d_gbs = 3 * rows_probe * n * 4 / (h0.elapsed_time(h1) * 1e-3) / 1e9
        del dst
        torch.cuda.empty_cache()
        barrier()
        t0 = time.perf_counter()
        marks = []
        for _ in range(a.steps):
            step_e2e()
            marks.append(time.perf_counter())
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0)
        step_ms = [round((b - a_) * 1e3, 1) for a_, b in zip([t0] + marks[:-1], marks)]
        out["e2e"] = {"value": total_queries / e2e_s, "unit": UNIT,
                      "h2d_bytes_per_step": N * n * 4 + a.queries * n * 4,
                      "d2h_bytes_per_step": a.queries * k * (8 + 4),
                      "ms_per_step": e2e_s / a.steps * 1e3, "step_ms": step_ms,
                      "h2d_GB_per_s": round(h2d_gbs, 1),
                      "h2d_ms_per_step_at_that_rate": round((N * n * 4 + a.queries * n * 4) / h2d_gbs / 1e6, 1)}
        del Xh, Qp, Qp_np, Xh_np
    else:
        del X, Qd
    # torch keeps freed page-locked blocks cached; hand them back to the system before
    # the host-rows leg page-locks 102 GB of its own (host memory holds one such copy)
    empty_host = getattr(torch._C, "_host_emptyCache", None)
    if empty_host is not None:
        torch.cuda.synchronize()
        empty_host()

    # rows in host memory, read over the CPU-GPU link by the refinement.  Run after
    # the end-to-end leg: run before it, its 102 GB of page-locked rows, once freed,
    # left the end-to-end leg's page-locked input slower to copy (a step took ~680
    # instead of ~520 ms).  The collection is generated on the device again.
    need = N * n * 4 * 1.1
    avail = host_available_bytes()
    if world > 1 and not a.no_host_rows:
        out["rows_in_host_memory"] = {"skipped": "one rank only (102 GB of page-locked rows per process)"}
    elif not a.no_host_rows and avail is not None and avail < need:
        out["rows_in_host_memory"] = {"skipped": "host memory available %.0f GB < %.0f GB needed"
                                                 % (avail / 1e9, need / 1e9)}
    elif not a.no_host_rows and (a.no_e2e or e2e_skip is not None or empty_host is not None):
        torch.cuda.synchronize()
        X = torch.empty((N, n), dtype=torch.float32, device="cuda")
        datagen.rows_device("walk", 0, rank * N, N, n, X.data_ptr(), sp)
        Qd = torch.from_numpy(Qh).cuda()
        out["rows_in_host_memory"] = host_rows_leg(a, X, Qd, pkg, torch, stream)
        del X, Qd
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    elif not a.no_host_rows:
        out["rows_in_host_memory"] = {"skipped": "this PyTorch cannot release its cached page-locked "
                                                 "memory, and host memory holds one 102 GB copy"}

    if rank == 0 and not a.no_serving and world == 1:
        # the served path (config 4): its own collections, after the main job's are freed
        torch.cuda.empty_cache()
        out["serving"] = serving_leg(a, pkg, torch)

    if rank == 0 and not a.no_hardness and world == 1:
        # query hardness (config 2): its own 50M-row collection, after the others are freed
        torch.cuda.empty_cache()
        out["hardness"] = hardness_leg(a, pkg, torch, datagen)

    if rank == 0 and not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(a, min(a.cpu_sample_rows, N))
        out["cpu_baseline_isax_index"] = isax_oracle_baseline(a)

    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
