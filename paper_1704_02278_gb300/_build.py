"""Build the native libraries in-tree.

* ``libglop.so``           -- the CUDA library behind include/glop.h (nvcc,
  sm_103a only).
* ``libglop_hostcheck.so`` -- test-only host check of the compiler's tables
  (g++, no CUDA).

Translation units compile in parallel; nothing is compiled when every output
is newer than its sources (pass ``force=True`` to rebuild).
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libglop.so")
HOSTCHECK = os.path.join(PKG, "libglop_hostcheck.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v", *ARCH,
              "-I" + INCLUDE, "-I" + CSRC]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-Wall", "-I" + INCLUDE, "-I" + CSRC]

CUDA_SOURCES = ["scan.cu", "scan_f0.cu", "scan_f4.cu", "scan_f8.cu", "noalloc.cu", "split.cu", "words.cu"]
HOST_SOURCES = ["compile.cpp", "api.cpp", "ingest.cpp", "server.cpp"]
HEADERS = ["glop_layout.h", "glop_hash.h", "compile.h", "scan.h", "scan_kernel.cuh"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def cuda_home() -> str:
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc())))


def _newer(out: str, srcs) -> bool:
    if not os.path.exists(out):
        return False
    t = os.path.getmtime(out)
    return all(os.path.getmtime(s) <= t for s in srcs if os.path.exists(s))


def _deps(extra=()):
    return [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "glop.h"), __file__, *extra]


def _run(cmd, log):
    r = subprocess.run(cmd, capture_output=True, text=True)
    with open(log, "w") as f:
        f.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError("build failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r


def build_lib(force: bool = False) -> str:
    """Compile libglop.so for sm_103a."""
    os.makedirs(BUILD, exist_ok=True)
    deps = _deps()
    jobs = []
    objs = []
    for s in CUDA_SOURCES + HOST_SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s + ".o")
        objs.append(obj)
        if force or not _newer(obj, [src, *deps]):
            if s.endswith(".cu"):
                cmd = [nvcc(), *NVCC_FLAGS, "-c", src, "-o", obj]
            else:
                cmd = [nvcc(), "-O2", "-std=c++17", "-Xcompiler", "-fPIC,-Wall", "-I" + INCLUDE, "-I" + CSRC,
                       "-c", src, "-o", obj]
            jobs.append((cmd, obj + ".log"))
    if jobs:
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            list(ex.map(lambda j: _run(*j), jobs))
    if force or jobs or not _newer(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        _run([nvcc(), "-shared", *ARCH, "-o", tmp, *objs, "-lcudart_static", "-ldl", "-lrt", "-lpthread"],
             os.path.join(BUILD, "link.log"))
        os.replace(tmp, LIB)
    return LIB


def build_checked_lib(out_path: str) -> str:
    """A debug build of libglop.so with every global index bounds-checked (-DGLOP_BOUNDS_CHECK)."""
    objs = []
    jobs = []
    for src_name in CUDA_SOURCES + HOST_SOURCES:
        src = os.path.join(CSRC, src_name)
        obj = out_path + "." + src_name + ".o"
        objs.append(obj)
        flags = NVCC_FLAGS + ["-DGLOP_BOUNDS_CHECK"] if src_name.endswith(".cu") else \
            ["-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]
        jobs.append(([nvcc(), *flags, "-c", src, "-o", obj], obj + ".log"))
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        list(ex.map(lambda j: _run(*j), jobs))
    _run([nvcc(), "-shared", *ARCH, "-o", out_path, *objs, "-lcudart_static", "-ldl", "-lrt", "-lpthread"],
         out_path + ".link.log")
    return out_path


def build_hostcheck(force: bool = False) -> str:
    """Compile the test-only host check (g++, no CUDA)."""
    srcs = [os.path.join(CSRC, "compile.cpp"), os.path.join(CSRC, "hostcheck.cpp")]
    if not force and _newer(HOSTCHECK, srcs + _deps()):
        return HOSTCHECK
    tmp = HOSTCHECK + ".tmp%d" % os.getpid()
    subprocess.run(["g++", *CXX_FLAGS, "-shared", *srcs, "-o", tmp], check=True)
    os.replace(tmp, HOSTCHECK)
    return HOSTCHECK


def ptxas_report() -> str:
    """The -Xptxas -v lines (registers, spills, shared memory) of the last build."""
    out = []
    for s in CUDA_SOURCES:
        log = os.path.join(BUILD, s + ".o.log")
        if os.path.exists(log):
            out.append(open(log).read())
    return "\n".join(out)
