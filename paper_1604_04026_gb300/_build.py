"""In-tree build of the native libraries (no cmake; one nvcc / gcc call each).

* ``lib/libnmfkl.so``       -- the CUDA sweep library behind ``include/nmfkl.h``,
  compiled for sm_103a only.
* ``lib/libnmfkl_synth.so`` -- the host-side synthetic input generator.

Outputs go to ``paper_1604_04026_gb300/lib/`` (git-ignored). Builds are
skipped when the output is newer than every source.
"""
from __future__ import annotations

import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "lib")
INCLUDE = os.path.join(ROOT, "include")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def library_path() -> str:
    return os.path.join(LIBDIR, "libnmfkl.so")


def synth_library_path() -> str:
    return os.path.join(LIBDIR, "libnmfkl_synth.so")


def _stale(out: str, srcs) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(s) > t for s in srcs)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r


def build_synth(force: bool = False) -> str:
    os.makedirs(LIBDIR, exist_ok=True)
    src = os.path.join(CSRC, "synth_gen.c")
    out = synth_library_path()
    if force or _stale(out, [src]):
        tmp = out + ".tmp%d" % os.getpid()
        _run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", src, "-o", tmp, "-lm"])
        os.replace(tmp, out)
    return out


def _cuda_sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _cuda_headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")))


def build_cuda(force: bool = False, extra_flags=None, verbose_ptxas: bool = False) -> str:
    """Compiles every .cu in csrc/ (in parallel) and links libnmfkl.so."""
    os.makedirs(LIBDIR, exist_ok=True)
    out = library_path()
    srcs = _cuda_sources()
    if not srcs:
        raise RuntimeError("no CUDA sources found in %s" % CSRC)
    if not (force or _stale(out, srcs + _cuda_headers())):
        return out
    objdir = os.path.join(LIBDIR, "obj")
    os.makedirs(objdir, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    if verbose_ptxas:
        flags += ["-Xptxas", "-v"]
    flags += list(extra_flags or [])

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        r = _run([NVCC] + flags + ["-c", src, "-o", obj])
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(compile_one, srcs))
    objs = [o for o, _ in results]
    tmp = out + ".tmp%d" % os.getpid()
    _run([NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcuda"])
    os.replace(tmp, out)
    if verbose_ptxas:
        for _, err in results:
            print(err)
    return out


def build_all(force: bool = False) -> None:
    build_synth(force)
    build_cuda(force)
