"""Build libflusi.so in-tree with nvcc for sm_103a (GB300).

Each CUDA translation unit is compiled in parallel, then linked into one
shared library next to this file.  The library carries the SHA-256 of the
sources and flags it was built from (``flusi_build_id()``), and the build is
redone whenever that differs from the sources present, so a library left over
from other sources is never reused, whatever the file times say.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libflusi.so")
BUILD = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-strict-aliasing",
         "--expt-relaxed-constexpr", "-I", INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libflusi")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def source_hash(extra=()) -> str:
    """SHA-256 (hex, 32 digits) of every source, header and flag of the library."""
    deps = sorted(sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")))
    h = hashlib.sha256()
    for p in deps:
        h.update(os.path.relpath(p, os.path.dirname(HERE)).encode())
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join([*ARCH, *FLAGS[:-1], *extra]).encode())
    return h.hexdigest()[:32]


def built_hash():
    """The source hash a built library reports, or None."""
    stamp = LIB + ".stamp"
    if not (os.path.exists(LIB) and os.path.exists(stamp)):
        return None
    with open(stamp) as f:
        return f.read().strip()


def _stale(extra=()) -> bool:
    return built_hash() != source_hash(extra)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and not _stale(extra):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    digest = source_hash(extra)

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra, f'-DFLUSI_SOURCE_HASH="{digest}"', "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = LIB + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(LIB + ".stamp", "w") as f:
        f.write(digest + "\n")
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
