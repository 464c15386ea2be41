"""Builds the in-tree shared library ``paper_0910_5435_gb300/lib/libsht.so``.

The CUDA sources are compiled for sm_103a only
(``-gencode arch=compute_103a,code=sm_103a``); host C++ is compiled with g++.
Translation units are compiled in parallel and the link is skipped when a
stamp of the sources and flags is unchanged.  Run as ``python -m
paper_0910_5435_gb300.build`` or through ``__graft_entry__.build()``.
"""

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libsht.so")
ROOT = os.path.dirname(PKG)

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Host code is compiled without floating-point contraction: gcc fuses a * b + c
# on aarch64 but not on x86-64 without -march flags, and the precomputation
# must give the same bits on both.  (Device code keeps nvcc's own rules.)
CXXFLAGS = ["-O3", "-std=c++17", "-ffp-contract=off", "-fPIC", "-pthread", "-Wall", "-Wno-unused-function"]
NVFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
           "--expt-relaxed-constexpr"] + ARCH

CPP_SOURCES = ["plan_build.cpp", "unit_stats.cpp", "plan_io.cpp"]
CU_SOURCES = ["capi.cu", "sweep.cu", "direct.cu", "phi.cu", "noalloc.cu", "batch.cu", "plan_device.cu", "peak.cu"]
HEADERS = ["sht_stream.h", "plan_host.h", "kernels.h", "plan_access.h", "recurrence.h"]


def _stamp():
    h = hashlib.sha256()
    for name in CPP_SOURCES + CU_SOURCES + HEADERS:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    with open(os.path.join(ROOT, "include", "sht.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(CXXFLAGS + NVFLAGS).encode())
    return h.hexdigest()


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def build(force=False, verbose=False, extra_nvflags=()):
    """Compiles the library if needed; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    stamp = _stamp() + "|" + " ".join(extra_nvflags)
    stamp_file = os.path.join(BUILD, "stamp.txt")
    if not force and os.path.exists(LIB) and os.path.exists(stamp_file):
        with open(stamp_file) as f:
            if f.read() == stamp:
                return LIB
    if not os.path.exists(NVCC):
        raise RuntimeError("nvcc not found at " + NVCC)
    cxx = shutil.which("g++") or "g++"
    jobs = []
    for name in CPP_SOURCES:
        obj = os.path.join(BUILD, name + ".o")
        jobs.append([cxx] + CXXFLAGS + ["-I" + os.path.join(CUDA_HOME, "include"), "-c",
                                        os.path.join(CSRC, name), "-o", obj])
    for name in CU_SOURCES:
        obj = os.path.join(BUILD, name + ".o")
        jobs.append([NVCC] + NVFLAGS + list(extra_nvflags) + ["-c", os.path.join(CSRC, name), "-o", obj])
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    objs = [os.path.join(BUILD, n + ".o") for n in CPP_SOURCES + CU_SOURCES]
    tmp = LIB + ".tmp"
    _run([NVCC, "-shared", "-o", tmp] + objs + ARCH + [
        "-cudart", "shared", "-lcufft", "-lpthread",
        "-Xlinker", "-rpath," + os.path.join(CUDA_HOME, "lib64")])
    os.replace(tmp, LIB)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
