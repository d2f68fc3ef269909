"""GPU (sm_103a) hybrid sort of Alghamdi & Alaghband (arXiv 2003.01216).

One MSD-radix step into ten packets by most significant decimal digit
(Sec. 2.1, Sec. 3.4), a per-packet tile sort, and bottom-up merge passes
(Fig. 1(b), Sec. 3.2), all in the CUDA kernels of libhsort.so.  This module
is a thin PyTorch-facing wrapper of the C ABI (include/hsort.h): tensors give
device memory, torch streams give the CUDA stream.
"""
from __future__ import annotations

import ctypes

from . import _native as N

__all__ = [
    "sort_keys", "sort_pairs", "sort_batch", "sort_keys_host", "stream_error", "plan", "workspace_size",
    "workspace_reserve", "workspace_release", "graph_cache_clear", "timing_enable", "timing_read", "timing_read_launches", "kernel_launches", "HsError",
    "dtype_code",
]

HsError = N.HsError


def dtype_code(t) -> int:
    import torch
    m = {torch.int32: N.HS_INT32, torch.uint32: N.HS_UINT32, torch.uint64: N.HS_UINT64}
    if t.dtype not in m:
        raise TypeError(f"keys must be int32, uint32 or uint64, not {t.dtype}")
    return m[t.dtype]


def _stream(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _check_dev(*ts):
    for t in ts:
        if t is None:
            continue
        if not t.is_cuda:
            raise ValueError("tensor must be on a CUDA device")
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")


def _opts(partition, stop_after, packet_offsets, debug_flags, workspace, graph=False, fan_in=0, tile=0, merge=0):
    po = 0
    if packet_offsets is not None:
        _check_dev(packet_offsets)
        po = packet_offsets.data_ptr()
    wp, wb = 0, 0
    if workspace is not None:
        _check_dev(workspace)
        wp, wb = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    return N.make_opts(partition=partition, stop_after=stop_after, packet_offsets_ptr=po, workspace_ptr=wp,
                       workspace_bytes=wb, debug_flags=debug_flags, graph=graph, fan_in=fan_in, tile=tile,
                       merge=merge)


def sort_keys(keys, partition: int = 10, stop_after: int = 0, packet_offsets=None, stream=None,
              debug_flags: int = 0, workspace=None, graph: bool = False, fan_in: int = 0, tile: int = 0,
              merge: int = 0):
    """Sort a CUDA tensor of int32/uint32/uint64 keys in place (ascending).
    fan_in: runs merged per merge pass, 2 or 4; tile: keys per tile, one of
    tiles(dtype); merge: 1 = two-way passes in one persistent launch, 2 = a
    launch per pass (0 everywhere = the tuned or default shape)."""
    _check_dev(keys)
    o = _opts(partition, stop_after, packet_offsets, debug_flags, workspace, graph, fan_in, tile, merge)
    N.check(N.lib().hs_sort_keys(dtype_code(keys), keys.data_ptr(), keys.numel(), ctypes.byref(o), _stream(stream)),
            "hs_sort_keys")
    return keys


def sort_pairs(keys, vals, partition: int = 10, stop_after: int = 0, packet_offsets=None, stream=None,
               debug_flags: int = 0, workspace=None, graph: bool = False, fan_in: int = 0, tile: int = 0,
               merge: int = 0):
    """Stable in-place sort of (key, uint32 value) pairs by key."""
    import torch
    _check_dev(keys, vals)
    if vals.dtype not in (torch.uint32, torch.int32) or vals.numel() != keys.numel():
        raise ValueError("vals must be a uint32 (or int32) tensor as long as keys")
    o = _opts(partition, stop_after, packet_offsets, debug_flags, workspace, graph, fan_in, tile, merge)
    N.check(N.lib().hs_sort_pairs(dtype_code(keys), keys.data_ptr(), vals.data_ptr(), keys.numel(), 1,
                                  ctypes.byref(o), _stream(stream)), "hs_sort_pairs")
    return keys, vals


def sort_batch(keys, offsets, vals=None, partition: int = 10, stop_after: int = 0, packet_offsets=None,
               stream=None, workspace=None, graph: bool = False, fan_in: int = 0, tile: int = 0,
               debug_flags: int = 0, merge: int = 0):
    """Sort every segment [offsets[s], offsets[s+1]) of `keys` on its own.
    offsets: CUDA uint64 (or int64) tensor of nseg + 1 entries."""
    _check_dev(keys, offsets, vals)
    o = _opts(partition, stop_after, packet_offsets, debug_flags, workspace, graph, fan_in, tile, merge)
    nseg = offsets.numel() - 1
    vp = vals.data_ptr() if vals is not None else None
    N.check(N.lib().hs_sort_batch(dtype_code(keys), keys.data_ptr(), vp, offsets.data_ptr(), nseg, keys.numel(),
                                  ctypes.byref(o), _stream(stream)), "hs_sort_batch")
    return keys


def sort_keys_host(arr, partition: int = 10, stream=None, fan_in: int = 0, merge: int = 0, tile: int = 0):
    """Sort host keys (numpy array or CPU tensor, contiguous) in place through
    the device; returns after the result is back in host memory."""
    import numpy as np
    codes = {np.dtype(np.int32): N.HS_INT32, np.dtype(np.uint32): N.HS_UINT32, np.dtype(np.uint64): N.HS_UINT64}
    if hasattr(arr, "numpy") and not isinstance(arr, np.ndarray):
        ptr, n, code = arr.data_ptr(), arr.numel(), dtype_code(arr)
    else:
        if not arr.flags.c_contiguous:
            raise ValueError("array must be contiguous")
        ptr, n, code = arr.ctypes.data, arr.size, codes[arr.dtype]
    o = N.make_opts(partition=partition, fan_in=fan_in, merge=merge, tile=tile)
    N.check(N.lib().hs_sort_keys_host(code, ptr, n, ctypes.byref(o), _stream(stream)), "hs_sort_keys_host")
    return arr


def stream_error(stream=None) -> int:
    """Synchronise the stream; return (and clear) the device error status."""
    return N.lib().hs_stream_error(_stream(stream))


def tiles(dtype: int, has_vals: bool = False) -> list[int]:
    """The tile sizes (keys) built for a key type, ascending."""
    out = (ctypes.c_int * 8)()
    c = ctypes.c_int()
    N.check(N.lib().hs_tiles(dtype, int(has_vals), out, 8, ctypes.byref(c)), "hs_tiles")
    return [out[i] for i in range(c.value)]


def plan(dtype: int, n: int, has_vals: bool = False, nseg: int = 1, partition: int = 10, stop_after: int = 0,
         fan_in: int = 0, debug_flags: int = 0, tile: int = 0, merge: int = 0):
    p = N.HsPlan()
    o = N.make_opts(partition=partition, stop_after=stop_after, fan_in=fan_in, debug_flags=debug_flags, tile=tile,
                    merge=merge)
    N.check(N.lib().hs_plan_describe(dtype, n, int(has_vals), nseg, ctypes.byref(o), ctypes.byref(p)),
            "hs_plan_describe")
    return {"tile": p.tile, "part_tile": p.part_tile, "merge_passes": p.merge_passes, "launches": p.launches,
            "fan_in": p.fan_in}


def workspace_size(dtype: int, n: int, has_vals: bool = False, nseg: int = 1, partition: int = 10) -> int:
    b = ctypes.c_size_t()
    o = N.make_opts(partition=partition)
    N.check(N.lib().hs_workspace_size(dtype, n, int(has_vals), nseg, ctypes.byref(o), ctypes.byref(b)),
            "hs_workspace_size")
    return b.value


def workspace_reserve(nbytes: int, stream=None) -> None:
    N.check(N.lib().hs_workspace_reserve(nbytes, _stream(stream)), "hs_workspace_reserve")


def workspace_release() -> None:
    N.check(N.lib().hs_workspace_release(), "hs_workspace_release")


def graph_cache_clear() -> None:
    N.check(N.lib().hs_graph_cache_clear(), "hs_graph_cache_clear")


def timing_enable(on: bool = True) -> None:
    N.check(N.lib().hs_timing_enable(int(on)), "hs_timing_enable")


def timing_read() -> dict[str, tuple[int, float]]:
    """{kernel name: (launches, total ms)} since the last read (synchronises)."""
    arr = (N.HsKernelTime * 64)()
    c = ctypes.c_int()
    N.check(N.lib().hs_timing_read(arr, 64, ctypes.byref(c)), "hs_timing_read")
    return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(c.value)}


def timing_read_launches(max_launches: int = 4096) -> list[tuple[str, float]]:
    """[(kernel name, ms)] launch by launch, in launch order, since the last
    read (synchronises)."""
    arr = (N.HsKernelTime * max_launches)()
    c = ctypes.c_int()
    N.check(N.lib().hs_timing_read_launches(arr, max_launches, ctypes.byref(c)), "hs_timing_read_launches")
    return [(arr[i].name.decode(), arr[i].total_ms) for i in range(c.value)]


def kernel_launches() -> int:
    return int(N.lib().hs_kernel_launches())
