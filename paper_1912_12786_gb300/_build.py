"""Build the GPU library ``libvsr.so`` in-tree for sm_103a.

Translation units are compiled in parallel with nvcc (device code) and g++
(the host BVH builder) and linked with nvcc into ``_build/libvsr.so``.  The
device code is compiled with ``-fmad=false`` and without fast-math so that the
FP32 tests keep the rounding order written in the source.
"""
from __future__ import annotations

import os
import subprocess
import sys
import threading
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libvsr.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["api.cu", "trace_static.cu", "trace_k0.cu", "trace_k1.cu", "trace_k2.cu",
              "trace_k4.cu", "trace_k8.cu", "trace_oct.cu", "trace_caps.cu", "trace_dynamic.cu", "trace_multi.cu",
              "trace_instances.cu", "render.cu", "batch.cu", "sort.cu", "path.cu", "measure.cu"]
CPP_SOURCES = [os.path.join(PKG, "inputs", "bvh_build.cpp")]
_lock = threading.Lock()


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def nvcc_flags(extra=()) -> list:
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler",
                   "-fPIC,-ffp-contract=off", "-I", INCLUDE, "-I", CSRC, *extra]


def _deps() -> list:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return files + CPP_SOURCES + [os.path.abspath(__file__)]


def _stale(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(f) > t for f in _deps())


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        print(r.stdout + r.stderr, file=sys.stderr)
    return r


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    """Compile libvsr.so if any source changed; returns its path."""
    with _lock:
        if not force and not _stale(LIB):
            return LIB
        os.makedirs(BUILD, exist_ok=True)
        nvcc = _nvcc()
        jobs = []
        for src in CU_SOURCES:
            obj = os.path.join(BUILD, src.replace(".cu", ".o"))
            extra = ["-Xptxas", "-v"] if ptxas_verbose else []
            jobs.append(([nvcc, *nvcc_flags(extra), "-c", os.path.join(CSRC, src), "-o", obj], obj))
        for src in CPP_SOURCES:
            obj = os.path.join(BUILD, os.path.basename(src).replace(".cpp", ".o"))
            jobs.append((["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-I",
                          INCLUDE, "-c", src, "-o", obj], obj))
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            list(ex.map(lambda j: _run(j[0], verbose or ptxas_verbose), jobs))
        tmp = LIB + f".tmp{os.getpid()}"
        _run([nvcc, *ARCH, "-shared", "-o", tmp, *[o for _, o in jobs]], verbose)
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_verbose="-v" in sys.argv))
