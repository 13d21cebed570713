"""Build ``libbdfb.so`` in-tree with nvcc for sm_103a (B300).

    python -m paper_2011_12984_b300.build [--force] [--verbose] [--phases]

``--phases`` builds ``libbdfb_phases.so`` instead: the same library with the
per-cell kernels' phase timers compiled in (``bdfb_phase_cycles``), for
profiling; its objects go to ``_build/phases``.

The library is plain CUDA C++ behind a C ABI (``include/bdfb.h``); it links
the CUDA runtime statically and does not depend on PyTorch.  Each source is
compiled to an object under ``_build/`` (in parallel; an object is rebuilt
when its source or any header is newer), then the objects are linked.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libbdfb.so")
LIB_PHASES = os.path.join(PKG, "libbdfb_phases.so")
OBJDIR = os.path.join(ROOT, "_build")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(INCLUDE, "bdfb.h")]


def deps():
    return sources() + headers()


def _newest(paths):
    return max(os.path.getmtime(p) for p in paths)


def up_to_date(lib=LIB) -> bool:
    return os.path.exists(lib) and os.path.getmtime(lib) >= _newest(deps() + [__file__])


def _obj(src, objdir=OBJDIR):
    return os.path.join(objdir, os.path.basename(src)[:-3] + ".o")


def _compile(src, force, verbose, phases=False):
    obj = _obj(src, os.path.join(OBJDIR, "phases") if phases else OBJDIR)
    hdr = _newest(headers() + [__file__])
    if not force and os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr):
        return obj
    tmp = obj + ".%d.tmp" % os.getpid()
    cmd = [NVCC, *FLAGS, "-I", INCLUDE, "-c", "-o", tmp, src]
    if phases:
        cmd[1:1] = ["-DBDFB_PHASES"]
    if verbose:
        cmd[1:1] = ["-Xptxas", "-v"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, obj)
    return obj


def build(force: bool = False, verbose: bool = False, phases: bool = False) -> str:
    lib = LIB_PHASES if phases else LIB
    if not force and not verbose and up_to_date(lib):
        return lib
    os.makedirs(os.path.join(OBJDIR, "phases") if phases else OBJDIR, exist_ok=True)
    srcs = sources()
    with ThreadPoolExecutor(max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(lambda s: _compile(s, force, verbose, phases), srcs))
    tmp = lib + ".%d.tmp" % os.getpid()
    subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv, phases="--phases" in sys.argv))
