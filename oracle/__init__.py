"""ctypes wrapper around the CPU oracle (``hsort_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the oracle restates the hybrid sort of Alghamdi &
Alaghband (arXiv 2003.01216) as a plain single-threaded CPU program, to check
the GPU library against.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the GPU library never
does, and this package imports nothing from it.

dtype codes: 0 = int32, 1 = uint32, 2 = uint64.  ``nbuckets`` is 10 (MSD
decimal digit, Sec. 2.1 / Sec. 3.4) or 256 (top-8-bit ablation).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hsort_oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")

DTYPES = {np.dtype(np.int32): 0, np.dtype(np.uint32): 1, np.dtype(np.uint64): 2}


def build(src: str = SRC, out: str = LIB) -> str:
    """Compile the oracle with g++ (plain C++17, no GPU code)."""
    cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", src, "-o", out]
    subprocess.run(cmd, check=True)
    return out


class Oracle:
    """One loaded copy of the oracle library (tests may load mutated copies)."""

    def __init__(self, path: str = LIB):
        if path == LIB and (not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC)):
            build()
        self.lib = ctypes.CDLL(path)
        u64, p = ctypes.c_uint64, ctypes.c_void_p
        L = self.lib
        L.hso_digit_info.argtypes = [ctypes.c_int, p, u64, ctypes.c_int, p, p]
        L.hso_partition.argtypes = [ctypes.c_int, p, p, u64, ctypes.c_int, p, p, p]
        L.hso_sort.argtypes = [ctypes.c_int, p, p, u64, ctypes.c_int, ctypes.c_uint32, ctypes.c_int, p]
        L.hso_sort_batch.argtypes = [ctypes.c_int, p, p, p, u64, ctypes.c_int, ctypes.c_uint32, ctypes.c_int]
        L.hso_tile_sort.argtypes = [ctypes.c_int, p, p, p, u64, u64]
        for f in (L.hso_digit_info, L.hso_partition, L.hso_sort, L.hso_sort_batch, L.hso_tile_sort):
            f.restype = ctypes.c_int

    @staticmethod
    def _code(keys: np.ndarray) -> int:
        if keys.dtype not in DTYPES:
            raise TypeError(f"unsupported key dtype {keys.dtype}")
        return DTYPES[keys.dtype]

    @staticmethod
    def _ptr(a):
        return None if a is None else a.ctypes.data

    def digit_info(self, keys: np.ndarray, nbuckets: int = 10):
        """(width, flip): D (or bit length) of the largest key image, sign flip used."""
        keys = np.ascontiguousarray(keys)
        w, f = ctypes.c_uint32(), ctypes.c_int()
        rc = self.lib.hso_digit_info(self._code(keys), self._ptr(keys), keys.size, nbuckets,
                                     ctypes.addressof(w), ctypes.addressof(f))
        if rc:
            raise ValueError("hso_digit_info: invalid argument")
        return w.value, bool(f.value)

    def partition(self, keys: np.ndarray, vals: np.ndarray | None = None, nbuckets: int = 10):
        """The MSD step alone: (packet layout of keys, of vals, offsets[nbuckets+1])."""
        keys = np.ascontiguousarray(keys)
        kout = np.empty_like(keys)
        vout = None
        if vals is not None:
            vals = np.ascontiguousarray(vals, dtype=np.uint32)
            vout = np.empty_like(vals)
        off = np.zeros(nbuckets + 1, dtype=np.uint64)
        rc = self.lib.hso_partition(self._code(keys), self._ptr(keys), self._ptr(vals), keys.size,
                                    nbuckets, self._ptr(kout), self._ptr(vout), self._ptr(off))
        if rc:
            raise ValueError("hso_partition: invalid argument")
        return kout, vout, off

    def sort(self, keys: np.ndarray, vals: np.ndarray | None = None, nbuckets: int = 10,
             T: int = 16, chunk_sort: int = 0):
        """The whole method on a copy: (sorted keys, values in stable order, offsets)."""
        keys = np.array(keys, copy=True, order="C")
        if vals is not None:
            vals = np.array(vals, dtype=np.uint32, copy=True, order="C")
        off = np.zeros(nbuckets + 1, dtype=np.uint64)
        rc = self.lib.hso_sort(self._code(keys), self._ptr(keys), self._ptr(vals), keys.size,
                               nbuckets, T, chunk_sort, self._ptr(off))
        if rc:
            raise ValueError("hso_sort: invalid argument")
        return keys, vals, off

    def sort_batch(self, keys: np.ndarray, offsets: np.ndarray, vals: np.ndarray | None = None,
                   nbuckets: int = 10, T: int = 16, chunk_sort: int = 0):
        keys = np.array(keys, copy=True, order="C")
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        if vals is not None:
            vals = np.array(vals, dtype=np.uint32, copy=True, order="C")
        rc = self.lib.hso_sort_batch(self._code(keys), self._ptr(keys), self._ptr(vals),
                                     self._ptr(offsets), offsets.size - 1, nbuckets, T, chunk_sort)
        if rc:
            raise ValueError("hso_sort_batch: invalid argument")
        return keys, vals

    def tile_sort(self, keys: np.ndarray, offsets: np.ndarray, tile: int,
                  vals: np.ndarray | None = None):
        """Sort every tile-long run of every packet (runs start at packet starts)."""
        keys = np.array(keys, copy=True, order="C")
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        if vals is not None:
            vals = np.array(vals, dtype=np.uint32, copy=True, order="C")
        rc = self.lib.hso_tile_sort(self._code(keys), self._ptr(keys), self._ptr(vals),
                                    self._ptr(offsets), offsets.size - 1, tile)
        if rc:
            raise ValueError("hso_tile_sort: invalid argument")
        return keys, vals


_default: Oracle | None = None


def get() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default
