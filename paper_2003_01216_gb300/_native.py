"""ctypes binding of libhsort.so (the C ABI of include/hsort.h).

Argument marshalling only: every step of the sort runs in the library's CUDA
kernels.  There is no fallback: if the library is missing or cannot load,
every call raises.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libhsort.so")

HS_OK, HS_ERR_INVALID, HS_ERR_NOMEM, HS_ERR_CUDA, HS_ERR_TIMEOUT, HS_ERR_UNSUPPORTED, HS_ERR_DEVICE = range(7)
HS_INT32, HS_UINT32, HS_UINT64 = 0, 1, 2

# every symbol include/hsort.h declares
EXPORTS = [
    "hs_sort_keys", "hs_sort_pairs", "hs_sort_batch", "hs_sort_keys_host", "hs_workspace_size",
    "hs_workspace_reserve", "hs_workspace_release", "hs_stream_error", "hs_plan_describe",
    "hs_timing_enable", "hs_timing_read", "hs_timing_read_launches", "hs_kernel_launches", "hs_status_string", "hs_last_error",
    "hs_sort_keys_noalloc", "hs_graph_cache_clear", "hs_tune_set", "hs_tune_get", "hs_tune_clear",
    "hs_tune_set_shape", "hs_tune_get_shape", "hs_tiles",
]


class HsOpts(ctypes.Structure):
    _fields_ = [
        ("partition", ctypes.c_int),
        ("tile", ctypes.c_int),
        ("fan_in", ctypes.c_int),
        ("stop_after", ctypes.c_int),
        ("d_packet_offsets_out", ctypes.c_void_p),
        ("d_workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_size_t),
        ("debug_flags", ctypes.c_int),
        ("graph", ctypes.c_int),
        ("merge", ctypes.c_int),
    ]


class HsPlan(ctypes.Structure):
    _fields_ = [
        ("tile", ctypes.c_int),
        ("part_tile", ctypes.c_int),
        ("merge_passes", ctypes.c_int),
        ("launches", ctypes.c_int),
        ("fan_in", ctypes.c_int),
    ]


class HsKernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int), ("total_ms", ctypes.c_double)]


class HsError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {status_string(status)} (status {status})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


_lib: ctypes.CDLL | None = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        p, sz, i = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
        L.hs_sort_keys.argtypes = [i, p, sz, p, p]
        L.hs_sort_pairs.argtypes = [i, p, p, sz, i, p, p]
        L.hs_sort_batch.argtypes = [i, p, p, p, sz, sz, p, p]
        L.hs_sort_keys_host.argtypes = [i, p, sz, p, p]
        L.hs_sort_keys_noalloc.argtypes = [i, p, sz, i, p]
        L.hs_workspace_size.argtypes = [i, sz, i, sz, p, p]
        L.hs_workspace_reserve.argtypes = [sz, p]
        L.hs_workspace_release.argtypes = []
        L.hs_graph_cache_clear.argtypes = []
        L.hs_tune_set.argtypes = [i, i, i, i, i]
        L.hs_tune_get.argtypes = [i, i, i, sz, p]
        L.hs_tune_clear.argtypes = []
        L.hs_tune_set_shape.argtypes = [i, i, i, i, i, i, i]
        L.hs_tune_get_shape.argtypes = [i, i, i, sz, p, p, p]
        L.hs_tiles.argtypes = [i, i, p, i, p]
        L.hs_stream_error.argtypes = [p]
        L.hs_plan_describe.argtypes = [i, sz, i, sz, p, p]
        L.hs_timing_enable.argtypes = [i]
        L.hs_timing_read.argtypes = [p, i, p]
        L.hs_timing_read_launches.argtypes = [p, i, p]
        L.hs_kernel_launches.argtypes = []
        L.hs_kernel_launches.restype = ctypes.c_ulonglong
        L.hs_status_string.argtypes = [i]
        L.hs_status_string.restype = ctypes.c_char_p
        L.hs_last_error.argtypes = []
        L.hs_last_error.restype = ctypes.c_char_p
        for name in EXPORTS:
            f = getattr(L, name)
            if name not in ("hs_kernel_launches", "hs_status_string", "hs_last_error"):
                f.restype = ctypes.c_int
        _lib = L
    return _lib


def status_string(s: int) -> str:
    try:
        return lib().hs_status_string(s).decode()
    except Exception:  # noqa: BLE001 - message formatting only
        return "?"


def check(status: int, where: str) -> None:
    if status != HS_OK:
        detail = lib().hs_last_error().decode() if status == HS_ERR_CUDA else ""
        raise HsError(status, where, detail)


def make_opts(partition: int = 10, stop_after: int = 0, packet_offsets_ptr: int = 0, workspace_ptr: int = 0,
              workspace_bytes: int = 0, debug_flags: int = 0, tile: int = 0, fan_in: int = 0,
              graph: bool = False, merge: int = 0) -> HsOpts:
    return HsOpts(partition, tile, fan_in, stop_after, packet_offsets_ptr or None, workspace_ptr or None,
                  workspace_bytes, debug_flags, int(graph), merge)
