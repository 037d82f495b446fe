"""Builds libfgt.so in-tree with nvcc for sm_103a (GB300), and libfgt_checked.so (the same
library with bounds-checked kernels).

Five translation units (the kernels twice) are compiled in parallel, then linked with the CUDA
runtime.  Used by ``__graft_entry__.build()`` and on first import of the
package when the library is missing or older than its sources.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libfgt.so")
CHECKED_LIB = os.path.join(HERE, "libfgt_checked.so")  # kernels built with -DFGT_CHECKED
OBJDIR = os.path.join(HERE, "_build")
SOURCES = ["fgt_kernels.cu", "fgt_plan.cpp", "fgt_tables.cpp", "fgt_ozaki.cu"]
HEADERS = ["fgt_internal.h", "fgt_exec.h", "fgt_tables.h", "fgt_tc.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfgt.so")


def _stale() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(CHECKED_LIB):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(CHECKED_LIB))
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(INCLUDE, "fgt.h")]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    nvcc = _nvcc()
    os.makedirs(OBJDIR, exist_ok=True)
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", f"-I{INCLUDE}"]

    def compile_one(job):
        src, defs = job
        obj = os.path.join(OBJDIR, src + ("_checked" if defs else "") + ".o")
        cmd = [nvcc] + common + defs + ARCH + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc] + common + ["-x", "c++", "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    # the kernels once more with the bounds checks for libfgt_checked.so (same host objects)
    jobs = [(src, []) for src in SOURCES] + [("fgt_kernels.cu", ["-DFGT_CHECKED"])]
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        objs = list(ex.map(compile_one, jobs))
    plain, checked = objs[: len(SOURCES)], [objs[-1]] + objs[1: len(SOURCES)]
    for out, parts in ((LIB, plain), (CHECKED_LIB, checked)):
        tmp = out + f".tmp{os.getpid()}"
        r = subprocess.run([nvcc, "-shared"] + ARCH + parts + ["-o", tmp, "-lcudart"], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, out)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
