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

# (key type, tag, items per thread) of every tile shape built: sort_shape.cu
# is compiled once per shape (see driver.cuh for the shapes)
SHAPES = [("int32_t", "i32", t) for t in (11, 15, 23, 31)] + [("uint32_t", "u32", t) for t in (11, 15, 23, 31)] + \
    [("uint64_t", "u64", t) for t in (11, 15)]


def _shape_objs() -> list[tuple[str, str, list[str]]]:
    """(object name, source, defines) of the per-shape translation units."""
    return [(f"sort_{tag}_t{ipt}.o", "sort_shape.cu",
             [f"-DHS_SHAPE_KEY={key}", f"-DHS_SHAPE_IPT={ipt}", f"-DHS_SHAPE_FN=run_sort_{tag}_t{ipt}"])
            for key, tag, ipt in SHAPES]


# library -> [(object, source, defines)]
LIBS = {
    "libhsort.so": [("hsort_abi.o", "hsort_abi.cu", []), ("hsort_noalloc.o", "hsort_noalloc.cu", [])] + _shape_objs(),
    "libhsgen.so": [("gen.o", "gen.cu", [])],
}
HEADERS = ["common.cuh", "async.cuh", "scan.cuh", "partition.cuh", "blockmerge.cuh", "tilesort.cuh", "merge.cuh", "merge4.cuh",
           "sched.cuh", "driver.cuh", "runtime.h"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def _newer(out: str, deps: list[str]) -> bool:
    return os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(d) for d in deps)


def _compile(obj_name: str, src: str, defines: list[str], verbose: bool, extra: list[str]) -> str:
    obj = os.path.join(BUILD, obj_name)
    deps = [src] + [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "hsort.h")]
    if _newer(obj, deps) and not extra:
        return obj
    cmd = [nvcc(), *ARCH, *FLAGS, *defines, *extra, "-c", src, "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    return obj


def build(verbose: bool = False, extra: list[str] | None = None) -> dict[str, str]:
    """Compile every library; returns {name: path}."""
    extra = list(extra or [])
    os.makedirs(BUILD, exist_ok=True)
    units = {o: (s, d) for parts in LIBS.values() for o, s, d in parts}
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        objs = dict(zip(units, ex.map(
            lambda o: _compile(o, os.path.join(CSRC, units[o][0]), units[o][1], verbose, extra), units)))
    out = {}
    for lib, parts in LIBS.items():
        path = os.path.join(PKG, lib)
        ol = [objs[o] for o, _, _ in parts]
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
