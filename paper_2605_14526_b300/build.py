"""Build the C-ABI library libpd_b300.so in-tree with nvcc for sm_103a."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpd_b300.so")
SOURCES = ["factor.cpp", "tsolve.cpp", "lbfgs.cpp", "pd_api.cpp", "pd_batch.cpp", "pd_kernels.cu", "pd_backward.cu", "pd_noalloc.cu", "pd_persistent.cu", "pd_mlp.cu"]
# every header of csrc/ (a header edit makes the library stale)
HEADERS = sorted(f for f in os.listdir(CSRC) if f.endswith((".h", ".cuh")))
ROOT_INCLUDE = os.path.join(os.path.dirname(HERE), "include", "pd_b300.h")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [ROOT_INCLUDE, __file__]
    return any(os.path.getmtime(p) > t for p in deps if os.path.exists(p))


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every source into libpd_b300.so (skips when up to date)."""
    if not force and not _stale():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    objs = []
    procs = []
    for src in SOURCES:
        obj = os.path.join(CSRC, src + ".o")
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj, "-O3", "-std=c++17", "-lineinfo",
               "-Xcompiler", "-fPIC,-fopenmp,-O3", *ARCH]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
        objs.append(obj)
    failed = False
    for src, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stderr.write(f"--- {src}\n{out}\n")
        failed |= p.returncode != 0
    if failed:
        raise RuntimeError("nvcc failed")
    cmd = [nvcc, "-shared", "-o", LIB, *objs, *ARCH, "-Xcompiler", "-fopenmp", "-lcudart", "-lgomp"]
    subprocess.run(cmd, check=True)
    for o in objs:
        os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
