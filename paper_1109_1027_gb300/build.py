"""Builds libnlse.so, the sm_103a CUDA library behind include/nlse.h.

Each translation unit under ``csrc/`` is compiled by nvcc in parallel and the
objects are linked into ``paper_1109_1027_gb300/lib/libnlse.so`` (static CUDA
runtime, so the library needs nothing beyond the driver at load time).  A
stamp of the sources and flags skips the build when nothing changed.

``build(checked=True)`` builds the bounds-check variant ``libnlse_checked.so``
from the same sources with -DNLSE_BOUNDS_CHECK: every kernel tests its
indices before the access and reports NLSE_EBOUNDS instead of accessing out
of range.  Loaded in place of the library through the NLSE_LIBRARY
environment variable (tests run it in a child process).
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libnlse.so")
CHECKED_LIB = os.path.join(LIBDIR, "libnlse_checked.so")
OBJDIR = os.path.join(PKG, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
                     "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnlse")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stamp(flags) -> str:
    h = hashlib.sha1()
    files = sources() + sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                               if f.endswith((".h", ".cuh")))
    files.append(os.path.join(INCLUDE, "nlse.h"))
    for f in files:
        h.update(f.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(flags).encode())
    return h.hexdigest()


def build(verbose: bool = False, force: bool = False, checked: bool = False) -> str:
    """Compile (if needed) and return the path of libnlse.so, or with checked
    of the bounds-check variant libnlse_checked.so."""
    lib = CHECKED_LIB if checked else LIB
    objdir = OBJDIR + ("_checked" if checked else "")
    flags = NVCC_FLAGS + (["-DNLSE_BOUNDS_CHECK"] if checked else [])
    stamp = _stamp(flags)
    stamp_file = lib + ".stamp"
    if not force and os.path.exists(lib) and os.path.exists(stamp_file):
        with open(stamp_file) as f:
            if f.read().strip() == stamp:
                return lib
    os.makedirs(objdir, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        cmd = [cc] + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    srcs = sources()
    with ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return lib


if __name__ == "__main__":
    print(build(verbose=True, force=True))
