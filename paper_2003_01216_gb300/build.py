"""Build the native libraries in-tree with nvcc for sm_103a (GB300).

    libhsort.so  the sort (C ABI of include/hsort.h)
    libhsgen.so  the device twin of inputs.py (test and benchmark inputs)

Translation units compile in parallel; the device code is whole-program (no
relocatable device code), one -gencode, so a full build takes about a minute.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include")]

LIBS = {
    "libhsort.so": ["hsort_abi.cu", "hsort_noalloc.cu", "sort_i32.cu", "sort_u32.cu", "sort_u64.cu"],
    "libhsgen.so": ["gen.cu"],
}
HEADERS = ["common.cuh", "async.cuh", "scan.cuh", "partition.cuh", "blockmerge.cuh", "tilesort.cuh", "merge.cuh", "merge4.cuh",
           "driver.cuh", "runtime.h"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def _newer(out: str, deps: list[str]) -> bool:
    return os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(d) for d in deps)


def _compile(src: str, verbose: bool, extra: list[str]) -> str:
    obj = os.path.join(BUILD, os.path.basename(src).replace(".cu", ".o"))
    deps = [src] + [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "hsort.h")]
    if _newer(obj, deps) and not extra:
        return obj
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    return obj


def build(verbose: bool = False, extra: list[str] | None = None) -> dict[str, str]:
    """Compile every library; returns {name: path}."""
    extra = list(extra or [])
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted({s for v in LIBS.values() for s in v})
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = dict(zip(srcs, ex.map(lambda s: _compile(os.path.join(CSRC, s), verbose, extra), srcs)))
    out = {}
    for lib, parts in LIBS.items():
        path = os.path.join(PKG, lib)
        ol = [objs[p] for p in parts]
        if not _newer(path, ol) or extra:
            cmd = [nvcc(), *ARCH, "-shared", "-o", path, *ol]
            if verbose:
                print(" ".join(cmd), flush=True)
            subprocess.run(cmd, check=True)
        out[lib] = path
    return out


if __name__ == "__main__":
    import sys
    build(verbose=True, extra=sys.argv[1:])
