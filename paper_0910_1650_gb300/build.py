"""Builds libapgb.so in-tree from csrc/*.cu for sm_103a with nvcc.

Each translation unit is compiled in parallel into ``_build/`` and the
objects are linked into ``paper_0910_1650_gb300/libapgb.so`` (cudart linked
statically, so the library only needs the driver at run time).  A unit is
recompiled when it, a header, or the flags changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libapgb.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-fvisibility=hidden", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libapgb.so")


def _headers_digest() -> str:
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(CSRC, "*.cuh")) +
                    glob.glob(os.path.join(ROOT, "include", "*.h"))):
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


def _unit_digest(src: str, hdr: str) -> str:
    with open(src, "rb") as f:
        return hashlib.sha256(f.read() + hdr.encode()).hexdigest()


def _compile(nvcc, src, obj, digest):
    cmd = [nvcc, *ARCH, *FLAGS, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stderr}")
    with open(obj + ".sha", "w") as f:
        f.write(digest)
    return obj


def build(verbose: bool = False, jobs: int | None = None) -> str:
    """Compile what changed and (re)link libapgb.so; returns its path."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    hdr = _headers_digest()
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    todo, objs = [], []
    for src in srcs:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        dig = _unit_digest(src, hdr)
        try:
            with open(obj + ".sha") as f:
                fresh = f.read() == dig and os.path.exists(obj)
        except OSError:
            fresh = False
        if not fresh:
            todo.append((src, obj, dig))
    if todo:
        n = jobs or min(len(todo), os.cpu_count() or 4)
        with cf.ThreadPoolExecutor(max_workers=n) as ex:
            futs = [ex.submit(_compile, nvcc, *t) for t in todo]
            for fu in cf.as_completed(futs):
                o = fu.result()
                if verbose:
                    print("compiled", os.path.basename(o), file=sys.stderr)
    if todo or not os.path.exists(LIB):
        tmp = LIB + ".tmp"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
