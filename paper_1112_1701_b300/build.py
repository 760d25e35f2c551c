"""In-tree build of ``libbls.so`` (CUDA kernels for sm_103a plus the C++ host runtime).

    python -m paper_1112_1701_b300.build [--force]

nvcc compiles the kernels with ``-gencode arch=compute_103a,code=sm_103a -lineinfo``;
g++ compiles the host runtime; nvcc links a shared library with the CUDA runtime
linked statically, so the library loads without any search path set.  The same kernels
compiled with -DBLS_DEBUG (device-side index checks) are linked with the same host
objects into ``libbls_debug.so``, which the binding loads when BLS_DEBUG=1.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJDIR = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libbls.so")
DEBUG_LIB = os.path.join(PKG, "libbls_debug.so")
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["bls_kernels.cu", "bls_static.cu", "bls_window.cu", "bls_shape.cu",
              "bls_variability.cu", "bls_unbinned.cu"]
CPP_SOURCES = ["bls_api.cpp", "bls_server.cpp"]
PROBES_SRC = "probes.cu"
PROBES = os.path.join(PKG, "bls_probes")


def _headers():
    hs = [os.path.join(INCLUDE, "bls.h")]
    hs += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")]
    return hs


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, debug=False):
    path = os.path.join(CSRC, src)
    obj = os.path.join(OBJDIR, src + (".debug.o" if debug else ".o"))
    if not _stale(obj, [path] + _headers()):
        return obj
    if src.endswith(".cu"):
        cmd = [NVCC, *ARCH, *(["-DBLS_DEBUG"] if debug else []), "-O3", "-lineinfo",
               "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-c", path, "-o", obj]
    else:
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall",
               "-Wno-unused-function",
               "-I", INCLUDE, "-I", os.path.join(CUDA_HOME, "include"), "-c", path, "-o", obj]
    subprocess.run(cmd, check=True)
    return obj


def _link(lib, objs, force):
    if force or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [NVCC, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)


def build(force: bool = False) -> str:
    """Compile every source that changed and relink ``libbls.so`` and ``libbls_debug.so``;
    returns the path of the former."""
    os.makedirs(OBJDIR, exist_ok=True)
    srcs = CU_SOURCES + CPP_SOURCES
    jobs = [(s, False) for s in srcs] + [(s, True) for s in CU_SOURCES]
    if force:
        for s, dbg in jobs:
            o = os.path.join(OBJDIR, s + (".debug.o" if dbg else ".o"))
            if os.path.exists(o):
                os.remove(o)
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        objs = list(ex.map(lambda j: _compile(*j), jobs))
    regular = objs[:len(srcs)]
    debug = objs[len(srcs):] + objs[len(CU_SOURCES):len(srcs)]
    _link(LIB, regular, force)
    _link(DEBUG_LIB, debug, force)
    src = os.path.join(CSRC, PROBES_SRC)
    if force or _stale(PROBES, [src]):
        tmp = PROBES + f".tmp{os.getpid()}"
        subprocess.run([NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-o", tmp, src],
                       check=True)
        os.replace(tmp, PROBES)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
