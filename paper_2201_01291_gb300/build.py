"""Build the in-tree C-ABI library `libavip.so` for GB300 (sm_103a).

Every translation unit is compiled in parallel (nvcc for .cu, g++ for the host .cpp) into
`_build/`, then linked with the shared CUDA runtime.  Run `python -m
paper_2201_01291_gb300.build` or call `build()`.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libavip.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-v"] + ARCH
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-Wall", "-pthread"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    return cu, cpp


def _run(cmd):
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    return p.returncode, " ".join(cmd), p.stdout


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile and link; returns the path of the shared library."""
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    cu, cpp = _sources()
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "avip.h")]
    newest = max(os.path.getmtime(d) for d in deps)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    jobs = []
    objs = []
    for f in cu:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        jobs.append([nvcc, *NVCC_FLAGS, "-I", INCLUDE, "-c", os.path.join(CSRC, f), "-o", o])
    for f in cpp:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        cuda_inc = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
        jobs.append(["g++", *CXX_FLAGS, "-I", INCLUDE, "-I", cuda_inc, "-c", os.path.join(CSRC, f), "-o", o])
    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        results = list(ex.map(_run, jobs))
    for rc, cmd, out in results:
        if verbose or rc != 0:
            sys.stdout.write(f"$ {cmd}\n{out}\n")
        if rc != 0:
            raise RuntimeError(f"compile failed: {cmd}\n{out}")
    tmp = LIB + ".tmp"
    rc, cmd, out = _run([nvcc, "-shared", *ARCH, "-cudart", "shared", "-o", tmp, *objs, "-lpthread", "-ldl"])
    if rc != 0:
        raise RuntimeError(f"link failed: {cmd}\n{out}")
    os.replace(tmp, LIB)
    with open(os.path.join(BUILD, "ptxas.log"), "w") as fh:
        for _, cmd, out in results:
            fh.write(f"$ {cmd}\n{out}\n")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
