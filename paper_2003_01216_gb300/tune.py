"""Autotuner for the shape of a sort: merge fan-in and tile size.

The library chooses two shapes at run time, neither of which changes the
result (the sorted order of Sec. 3.4, bit for bit):
  * the tile: keys per tile of the per-packet sort, = 256 threads x items
    per thread (hs_tiles lists the built ones per key type).  A larger tile
    means fewer merge passes but a heavier tile sort and fewer CTAs busy on
    small inputs;
  * the merge fan-in: how many sorted runs a merge pass merges (2, as in
    Fig. 1(b), or 4).  Fan-in 4 halves the passes over memory but does two
    merge levels per pass in shared memory, so it wins while passes are short
    (launch- and latency-bound) and loses once they are long and HBM-bound.
Calls with ``fan_in=0`` / ``tile=0`` use the library's tuning table
(``hs_tune_set_shape``), else a built-in rule; this module fills the table by
timing every (fan-in, tile) candidate on the current GPU and keeps the results
in a JSON cache:

    {"version": 2, "device": "<GPU name>",
     "entries": [{"dtype": "int32", "has_vals": false, "partition": 10, "log2n": 20,
                  "fan_in": 4, "tile": 3840, "merge": 0,
                  "ms": {"2x3840q": 0.33, "2x3840p": 0.30, "4x3840": 0.27, ...}}, ...]}

Timing: CUDA events on the sorting stream around one sort, the input restored
from a pristine copy before every sort (outside the events), the median of
``reps`` sorts after ``warmup`` untimed ones.
"""
from __future__ import annotations

import json
import os
import statistics

from . import _native as N

DTYPE_NAMES = {N.HS_INT32: "int32", N.HS_UINT32: "uint32", N.HS_UINT64: "uint64"}
DTYPE_CODES = {v: k for k, v in DTYPE_NAMES.items()}
# the synthetic distribution timed for each key type (seeded generator)
TUNE_DIST = {N.HS_INT32: "uniform31", N.HS_UINT32: "uniform32", N.HS_UINT64: "uniform64"}
FANS = (2, 4)


def size_bucket(n: int) -> int:
    """ceil(log2(n)) (0 for n <= 1): the library's bucket of a size."""
    b = 0
    while (1 << b) < n:
        b += 1
    return b


MERGE_QUEUE, MERGE_PER_PASS = 1, 2


def candidates(dtype: int, has_vals: bool = False) -> list[tuple[int, int, int]]:
    """Every (fan-in, tile, merge launch) shape built for this key type (the
    launch style only matters for two-way passes)."""
    import paper_2003_01216_gb300 as hs
    out = []
    for t in hs.tiles(dtype, has_vals):
        out += [(2, t, MERGE_QUEUE), (2, t, MERGE_PER_PASS), (4, t, 0)]
    return out


def _key(fan: int, tile: int, merge: int = 0) -> str:
    return f"{fan}x{tile}" + {MERGE_QUEUE: "q", MERGE_PER_PASS: "p"}.get(merge, "")


def set_entry(dtype: int, has_vals: bool, partition: int, log2n: int, fan_in: int, tile: int = 0,
              merge: int = 0) -> None:
    N.check(N.lib().hs_tune_set_shape(dtype, int(has_vals), partition, log2n, fan_in, tile, merge),
            "hs_tune_set_shape")


def get_shape(dtype: int, n: int, has_vals: bool = False, partition: int = 10) -> tuple[int, int, int]:
    """The (fan-in, tile, merge launch) a call with all three 0 uses for n keys."""
    import ctypes
    f, t, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    N.check(N.lib().hs_tune_get_shape(dtype, int(has_vals), partition, n, ctypes.byref(f), ctypes.byref(t),
                                      ctypes.byref(m)), "hs_tune_get_shape")
    return f.value, t.value, m.value


def get(dtype: int, n: int, has_vals: bool = False, partition: int = 10) -> int:
    """The fan-in a call with fan_in=0 uses for n keys."""
    return get_shape(dtype, n, has_vals, partition)[0]


def clear() -> None:
    N.check(N.lib().hs_tune_clear(), "hs_tune_clear")


def measure(dtype: int, n: int, has_vals: bool = False, partition: int = 10, shapes=None,
            reps: int = 5, warmup: int = 2, seed: int = 0) -> dict[tuple[int, int, int], float]:
    """Median milliseconds of one sort of n synthetic keys per shape."""
    import torch

    import paper_2003_01216_gb300 as hs
    from . import inputs as I
    shapes = list(shapes) if shapes is not None else candidates(dtype, has_vals)
    pristine = I.device_generate(TUNE_DIST[dtype], n, seed=seed)
    work = torch.empty_like(pristine)
    vals0 = I.device_index_values(n) if has_vals else None
    vals = torch.empty_like(vals0) if has_vals else None
    st = torch.cuda.Stream()
    out = {}
    with torch.cuda.stream(st):
        for fan, tile, merge in shapes:
            ms = []
            for it in range(warmup + reps):
                work.copy_(pristine)
                if has_vals:
                    vals.copy_(vals0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(st)
                if has_vals:
                    hs.sort_pairs(work, vals, partition=partition, fan_in=fan, tile=tile, merge=merge, stream=st)
                else:
                    hs.sort_keys(work, partition=partition, fan_in=fan, tile=tile, merge=merge, stream=st)
                b.record(st)
                b.synchronize()
                if it >= warmup:
                    ms.append(a.elapsed_time(b))
            if hs.stream_error(st) != 0:
                raise RuntimeError(f"device error while timing shape {_key(fan, tile, merge)}")
            out[(fan, tile, merge)] = statistics.median(ms)
    return out


def autotune(dtype: int, sizes, has_vals: bool = False, partition: int = 10, reps: int = 5) -> list[dict]:
    """Time every candidate shape at every size, install the fastest in the
    library's table (one entry per size bucket) and return the entries."""
    entries = []
    for n in sizes:
        ms = measure(dtype, n, has_vals, partition, reps=reps)
        fan, tile, merge = min(ms, key=ms.get)
        e = {"dtype": DTYPE_NAMES[dtype], "has_vals": bool(has_vals), "partition": partition,
             "log2n": size_bucket(n), "fan_in": fan, "tile": tile, "merge": merge,
             "ms": {_key(*k): v for k, v in ms.items()}}
        set_entry(dtype, has_vals, partition, e["log2n"], fan, tile, merge)
        entries.append(e)
    return entries


def device_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name() if torch.cuda.is_available() else "none"
    except Exception:  # noqa: BLE001 - the name only labels the cache
        return "unknown"


def save(path: str, entries: list[dict], device: str | None = None) -> None:
    doc = {"version": 2, "device": device if device is not None else device_name(), "entries": entries}
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(doc, f, indent=1)
    os.replace(tmp, path)


def load(path: str, device: str | None = None, any_device: bool = False) -> int:
    """Install the entries of a cache file; entries measured on another GPU
    model are skipped unless any_device.  Returns the number installed."""
    with open(path) as f:
        doc = json.load(f)
    if doc.get("version") not in (1, 2):  # version 1: fan-in only
        raise ValueError(f"{path}: unknown tuning cache version {doc.get('version')}")
    dev = device if device is not None else device_name()
    if not any_device and doc.get("device") != dev:
        return 0
    k = 0
    for e in doc["entries"]:
        set_entry(DTYPE_CODES[e["dtype"]], bool(e["has_vals"]), int(e["partition"]), int(e["log2n"]), int(e["fan_in"]),
                  int(e.get("tile", 0)), int(e.get("merge", 0)))
        k += 1
    return k
