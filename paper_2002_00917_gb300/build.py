"""Compile libpslr.so in-tree for sm_103a (GB300).

The translation units are compiled in parallel with nvcc (one -gencode,
compute_103a -> sm_103a, -lineinfo) and linked into
``paper_2002_00917_gb300/libpslr.so``; objects go to ``_build/`` next to this
file.  No CMake, no host-specific flags, so the same command works on x86 and
on the Arm GPU hosts.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpslr.so")
SOURCES = ["pslr_apply.cu", "pslr_apply_ml.cu", "pslr_apply_unit.cu", "pslr_krylov.cu", "pslr_host.cpp", "pslr_noalloc.cu", "pslr_batch_f64.cu",
           "pslr_batch_f32.cu", "pslr_batch_f32d.cu", "pslr_bkrylov.cu", "pslr_batch_host.cpp",
           "pslr_partition.cpp", "pslr_ilu0.cu"]
HEADERS = [os.path.join(CSRC, "pslr_internal.h"), os.path.join(CSRC, "pslr_device.cuh"),
           os.path.join(CSRC, "pslr_kernels.cuh"),
           os.path.join(CSRC, "pslr_sys.h"), os.path.join(CSRC, "pslr_batch.cuh"),
           os.path.join(CSRC, "pslr_reduce.cuh"), os.path.join(CSRC, "pslr_trace.h"),
           os.path.join(ROOT, "include", "pslr.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpslr")
    return exe


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src):
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    if not _stale(obj, [src] + HEADERS):
        return obj
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-pthread",
           "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj + ".tmp"]
    if src.endswith(".cpp"):
        cmd[1:1] = ["-x", "cu"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj


def build(force=False, verbose=False):
    """Build libpslr.so if any source or header is newer; return its path."""
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    if not force and not _stale(LIB, srcs + HEADERS):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for f in os.listdir(BUILD):
            os.remove(os.path.join(BUILD, f))
    with cf.ThreadPoolExecutor(len(srcs)) as ex:
        objs = list(ex.map(_compile, srcs))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-Xcompiler", "-fPIC,-pthread", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB}", file=sys.stderr)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
