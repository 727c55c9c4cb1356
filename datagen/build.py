"""Build the seeded input generator: a host shared library (gcc, FP64 with no
contraction) and a device shared library (nvcc, sm_103a)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "_build")
HOST_LIB = os.path.join(OUT, "libdghost.so")
CUDA_LIB = os.path.join(OUT, "libdgcuda.so")

GENCODE = "-gencode=arch=compute_103a,code=sm_103a"


def _stale(target, sources):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def host_cmd():
    src = os.path.join(HERE, "dg_host.c")
    return [
        "gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
        "-pthread", "-o", HOST_LIB, src, "-lm",
    ], [src, os.path.join(HERE, "dg_core.h")]


def cuda_cmd():
    src = os.path.join(HERE, "dg_cuda.cu")
    return [
        "nvcc", GENCODE, "-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC",
        "-shared", "-o", CUDA_LIB, src,
    ], [src, os.path.join(HERE, "dg_core.h")]


def build(cuda=True):
    os.makedirs(OUT, exist_ok=True)
    jobs = [(HOST_LIB,) + host_cmd()]
    if cuda:
        jobs.append((CUDA_LIB,) + cuda_cmd())
    procs = []
    for target, cmd, srcs in jobs:
        if _stale(target, srcs):
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("datagen build failed: %s\n%s" % (" ".join(cmd), out.decode()))


if __name__ == "__main__":
    build()
