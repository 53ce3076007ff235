"""Build libpic.so (the C ABI of include/pic.h) for sm_103a with nvcc, in-tree.

Each translation unit compiles to its own object in parallel (no relocatable
device code: every kernel is launched from the file that defines it), then
one host link makes the shared library.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libpic.so")
OBJDIR = os.path.join(HERE, "_build")
SOURCES = sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))
HEADERS = glob.glob(os.path.join(HERE, "csrc", "*.cuh")) + [os.path.join(ROOT, "include", "pic.h")]
DEPS = SOURCES + HEADERS
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", *ARCH, "-Xcompiler", "-fPIC"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _obj(src: str) -> str:
    return os.path.join(OBJDIR, os.path.basename(src)[:-3] + ".o")


def _compile(src: str, verbose: bool) -> str:
    obj = _obj(src)
    tmp = obj + f".tmp{os.getpid()}"
    cmd = [nvcc(), *FLAGS, "-I", os.path.join(ROOT, "include"), "-c", src, "-o", tmp]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, obj)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    newest_header = max(os.path.getmtime(p) for p in HEADERS)
    if not force and os.path.exists(LIB):
        lm = os.path.getmtime(LIB)
        if all(os.path.getmtime(p) <= lm for p in DEPS):
            return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    stale = [s for s in SOURCES
             if force or not os.path.exists(_obj(s))
             or os.path.getmtime(_obj(s)) < max(os.path.getmtime(s), newest_header)]
    workers = max(1, min(len(stale), os.cpu_count() or 1))
    if stale:
        with concurrent.futures.ThreadPoolExecutor(workers) as ex:
            list(ex.map(lambda s: _compile(s, verbose), stale))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc(), *ARCH, "-shared", *[_obj(s) for s in SOURCES], "-o", tmp,
                           "-lcudart"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="-f" in sys.argv or "-v" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
