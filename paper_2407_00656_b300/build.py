"""Build libhgks.so in-tree with nvcc for sm_103a (B300).

    python -m paper_2407_00656_b300.build [--force] [-v]

Each source compiles to its own object in parallel (the kernel translation
units take minutes each), then nvcc links the shared library.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libhgks.so")
OBJ = os.path.join(HERE, "_build")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")) + glob.glob(os.path.join(HERE, "csrc", "*.cpp")))


def headers():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.h")) + glob.glob(os.path.join(HERE, "csrc", "*.cuh")) +
                  [os.path.join(ROOT, "include", "hgks.h")])


def _newest_header() -> float:
    return max(os.path.getmtime(p) for p in headers())


def _obj(src: str) -> str:
    return os.path.join(OBJ, os.path.basename(src) + ".o")


def _stale_obj(src: str) -> bool:
    o = _obj(src)
    return not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(src), _newest_header())


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in sources() + headers())


def _compile(src: str, nvcc: str, verbose: bool) -> None:
    tmp = _obj(src) + f".{os.getpid()}.tmp"
    cmd = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp,-O2",
           "-I", os.path.join(ROOT, "include"), "-c", src, "-o", tmp]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    os.replace(tmp, _obj(src))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    os.makedirs(OBJ, exist_ok=True)
    todo = [s for s in sources() if force or _stale_obj(s)]
    with ThreadPoolExecutor(max_workers=max(1, min(len(todo), os.cpu_count() or 1))) as ex:
        for f in [ex.submit(_compile, s, nvcc, verbose) for s in todo]:
            f.result()
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.run([nvcc, ARCH, "-shared", "-o", tmp] + [_obj(s) for s in sources()] + ["-lgomp"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
