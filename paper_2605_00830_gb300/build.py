"""In-tree build of libfastged (sm_103a) with nvcc.

Translation units are compiled in parallel to objects under ``_build/`` and linked into one
shared library with the CUDA runtime linked statically, so nothing outside the tree is
needed at run time. Rebuilds only when a source or header is newer than the library.

build(checked=True) makes the bounds-checked library (``-DFASTGED_BOUNDS_CHECK``): every
index of the K-Best kernels is checked against its array, a violation is reported through
the batch's status word (the access goes to the array's first element instead) and the
call fails with FASTGED_ERR_CUDA. It is a debugging build; the binding loads it when the
environment variable FASTGED_LIBRARY names it.
"""
from __future__ import annotations

import os
import platform
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["kbest_kernels.cu", "kbest_b0.cu", "kbest_b2.cu", "kbest_b8.cu", "fastged_runtime.cu",
           "probe_kernels.cu", "noalloc.cu", "serve.cu", "paths.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def lib_path(checked: bool = False) -> str:
    tag = "_checked" if checked else ""
    return os.path.join(BUILD, f"libfastged{tag}_{platform.machine()}.so")


def _deps():
    out = [os.path.join(CSRC, s) for s in SOURCES]
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            if f.endswith((".h", ".cuh")):
                out.append(os.path.join(d, f))
    return out


def _stale(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in _deps())


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    out = lib_path(checked)
    if not force and not _stale(out):
        return out
    os.makedirs(BUILD, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                    "-I", INCLUDE, "-I", CSRC]
    if verbose:
        flags += ["-Xptxas", "-v"]
    if checked:
        flags += ["-DFASTGED_BOUNDS_CHECK"]
    tag = "_checked" if checked else ""

    def one(src):
        obj = os.path.join(BUILD, src.replace(".cu", f"{tag}_{platform.machine()}.o"))
        cmd = [NVCC] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        res = list(ex.map(one, SOURCES))
    objs = [o for o, _ in res]
    tmp = out + f".tmp{os.getpid()}"
    cmd = [NVCC] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs + ["-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    if verbose:
        for _, log in res:
            print(log)
    return out


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                checked="--checked" in sys.argv))
