"""Build the CUDA library libbd.so in-tree (sm_103a only).

Each translation unit is compiled by nvcc in parallel into ``_build/`` and
linked into ``_lib/libbd.so``.  Sources newer than their object are rebuilt;
``force=True`` rebuilds everything.
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
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libbd.so")

SOURCES = ["bd.cu", "ionic.cu", "pcg.cu", "amg.cu", "mixed.cu", "stream.cu", "stream2.cu", "assemble.cpp", "amg.cpp"]
HEADERS = ["bd_internal.h", "models.cuh", "sd.cuh", "sparse.cuh", "vcycle.cuh", "segment.cuh", "stream_rows.cuh"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
NVCC_FLAGS = ["-O3", "-std=c++20", ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O3",
              "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found")
    return path


def _obj(src: str) -> str:
    return os.path.join(BUILD, src.replace(".", "_") + ".o")


def _stale(src: str) -> bool:
    o = _obj(src)
    if not os.path.exists(o):
        return True
    t = os.path.getmtime(o)
    deps = [os.path.join(CSRC, src)] + [os.path.join(CSRC, h) for h in HEADERS] + \
           [os.path.join(ROOT, "include", "bd.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, extra) -> str:
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", _obj(src)] + NVCC_FLAGS + list(extra)
    if src.endswith(".cpp"):
        cmd = [nvcc(), "-x", "c++", "-c", os.path.join(CSRC, src), "-o", _obj(src),
               "-O3", "-std=c++20", "-Xcompiler", "-fPIC,-O3,-pthread",
               "-I" + os.path.join(ROOT, "include")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return r.stderr


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    todo = [s for s in SOURCES if force or _stale(s)]
    if todo:
        with cf.ThreadPoolExecutor(max_workers=len(todo)) as ex:
            logs = list(ex.map(lambda s: _compile(s, extra), todo))
        if verbose:
            for s, l in zip(todo, logs):
                if l.strip():
                    print(f"[{s}]\n{l}", file=sys.stderr)
    if todo or not os.path.exists(LIB):
        tmp = LIB + ".tmp"
        cmd = [nvcc(), "-shared", ARCH, "-o", tmp] + [_obj(s) for s in SOURCES] + \
              ["-Xcompiler", "-pthread", "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    force = "--force" in sys.argv
    print(build(force=force, verbose=True, extra=["-Xptxas", "-v"] if "-v" in sys.argv else []))
