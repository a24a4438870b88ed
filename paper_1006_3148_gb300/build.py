"""Builds libjacobi.so in-tree from csrc/*.cu for sm_103a (nvcc, no cmake).

Each translation unit is compiled in parallel to _build/*.o, then linked
into paper_1006_3148_gb300/libjacobi.so (static CUDA runtime); a build tag
(JACOBI_BUILD_TAG) selects another object folder and library name.  Rebuilds only
when a source or header is newer than the library, or when the extra nvcc
flags differ from the last build's.  Extra flags come from the environment
variable JACOBI_NVCC_FLAGS (space separated), e.g.
JACOBI_NVCC_FLAGS=-DJACOBI_INT_ADDS=0x00 for the build with every FP64
addition on the FP64 pipe.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
# JACOBI_BUILD_TAG names a separate build (objects in _build_<tag>/, library
# libjacobi_<tag>.so), e.g. "checked" with JACOBI_NVCC_FLAGS=-DJACOBI_CHECKED
# for the bounds-checked library beside the normal one.
TAG = os.environ.get("JACOBI_BUILD_TAG", "")
BUILD = os.path.join(HERE, "_build" + ("_" + TAG if TAG else ""))
LIB = os.path.join(HERE, "libjacobi" + ("_" + TAG if TAG else "") + ".so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I" + INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libjacobi.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]


STAMP = os.path.join(BUILD, "flags.txt")


def extra_flags() -> list:
    return os.environ.get("JACOBI_NVCC_FLAGS", "").split()


def _stamped_flags() -> str:
    try:
        with open(STAMP) as fh:
            return fh.read()
    except OSError:
        return ""


def up_to_date() -> bool:
    if not os.path.exists(LIB) or _stamped_flags() != " ".join(extra_flags()):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    extra = extra_flags() + (["-Xptxas", "-v"] if ptxas_info else [])

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose or ptxas_info:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    with open(STAMP, "w") as fh:
        fh.write(" ".join(extra_flags()))
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
