"""Build libzxp.so in-tree: host C++ with g++, CUDA with nvcc for sm_103a.

The translation units compile in parallel; the library links the CUDA
runtime statically so that it loads on machines without a GPU driver (the
C ABI's host-only entry points, such as compilation, then still work).
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libzxp.so")
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
HOST_SRC = ["ps.cpp", "compile.cpp", "param.cpp", "plan.cpp", "sample.cpp", "split.cpp", "checkpoint.cpp",
            "reorder.cpp"]
CUDA_SRC = ["kernel.cu", "kernel_count.cu", "kernel_wide.cu", "batch.cu", "batch_count.cu", "api.cu", "serve.cu",
            "inner.cu", "peak.cu"]


def _nvcc() -> str:
    for c in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        p = os.path.join(c, "bin", "nvcc") if c else ""
        if p and os.path.exists(p):
            return p
    p = shutil.which("nvcc")
    if not p:
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libzxp")
    return p


def _sources_newer_than(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(ROOT, "include", "zxp.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _sources_newer_than(LIB):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    jobs = []
    for f in HOST_SRC:
        obj = os.path.join(BUILD, f + ".o")
        jobs.append(["g++", "-std=c++17", "-O2", "-fPIC", "-ffp-contract=off", "-Wall", "-Wno-unused-function", *inc,
                     "-c", os.path.join(CSRC, f), "-o", obj])
    for f in CUDA_SRC:
        obj = os.path.join(BUILD, f + ".o")
        jobs.append([nvcc, "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC",
                     "-Xptxas", "-v" if verbose else "-O3", *inc,
                     "-c", os.path.join(CSRC, f), "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(run, jobs))
    if verbose:
        for lg in logs:
            if lg.strip():
                print(lg)
    objs = [os.path.join(BUILD, f + ".o") for f in HOST_SRC + CUDA_SRC]
    tmp = LIB + f".tmp{os.getpid()}"
    run([nvcc, "-shared", *ARCH, "-cudart", "static", "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
