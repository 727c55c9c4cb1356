"""Compile the sm_103a CUDA library libisaxgpu.so in-tree (nvcc, one gencode,
translation units in parallel)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libisaxgpu.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["isax_api.cu", "isax_build.cu", "isax_query.cu", "isax_profile.cu", "isax_noalloc.cu",
           "isax_tc.cu", "isax_serve.cu", "isax_selftest.cu"]
HEADERS = ["isax_common.cuh", "isax_kernels_util.cuh", "isax_tc.cuh"]
GENCODE = "-gencode=arch=compute_103a,code=sm_103a"
NVCC_FLAGS = [GENCODE, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-Xptxas", "-warn-spills", "--expt-relaxed-constexpr"]


def _deps():
    return ([os.path.join(CSRC, s) for s in SOURCES + HEADERS] +
            [os.path.join(INCLUDE, "isax.h")])


# the bounds-checked variant (-DISAX_CHECKS), built on demand by the tests that use it
OUT_CHECKS = os.path.join(HERE, "_build_checks")
LIB_CHECKS = os.path.join(OUT_CHECKS, "libisaxgpu.so")


def stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def build_checked(verbose=False):
    """The library with bounds-checked kernels (isax_check_word reports)."""
    return build(verbose, ("-DISAX_CHECKS",), out=OUT_CHECKS, lib=LIB_CHECKS)


def build(verbose=False, extra_flags=(), out=OUT, lib=LIB):
    if not stale(lib) and (not extra_flags or lib != LIB):
        return lib
    os.makedirs(out, exist_ok=True)
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(out, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = ["nvcc"] + NVCC_FLAGS + list(extra_flags) + ["-I", INCLUDE, "-c",
                                                            os.path.join(CSRC, src), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    logs = []
    for cmd, p in procs:
        out, _ = p.communicate()
        logs.append(out.decode())
        if p.returncode != 0:
            raise RuntimeError("nvcc failed: %s\n%s" % (" ".join(cmd), out.decode()))
    link = ["nvcc", GENCODE, "-shared", "-o", lib] + objs + ["-lcudart"]
    p = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if p.returncode != 0:
        raise RuntimeError("link failed:\n" + p.stdout.decode())
    if verbose:
        print("".join(logs))
    return lib


if __name__ == "__main__":
    import sys
    build(verbose=True, extra_flags=sys.argv[1:])
