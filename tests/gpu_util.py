"""Helpers for the GPU parity tests: move numpy inputs to the device, run one
library call through the C ABI, bring the results back."""
from __future__ import annotations

import numpy as np

HS_INVALID, HS_TIMEOUT = 1, 4


def dev():
    import torch
    return torch.device("cuda", 0)


def to_dev(a: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def run(keys: np.ndarray, vals: np.ndarray | None = None, nb: int = 10, stop_after: int = 0, debug_flags: int = 0,
        fan_in: int = 0, tile: int = 0, merge: int = 0):
    """One hs_sort_keys / hs_sort_pairs call; returns (keys, vals, offsets, status)."""
    import torch

    import paper_2003_01216_gb300 as hs
    tk = to_dev(keys)
    tv = to_dev(vals) if vals is not None else None
    off = torch.zeros(nb + 1, dtype=torch.uint64, device=dev())
    if tv is None:
        hs.sort_keys(tk, partition=nb, stop_after=stop_after, packet_offsets=off, debug_flags=debug_flags,
                     fan_in=fan_in, tile=tile, merge=merge)
    else:
        hs.sort_pairs(tk, tv, partition=nb, stop_after=stop_after, packet_offsets=off, debug_flags=debug_flags,
                      fan_in=fan_in, tile=tile, merge=merge)
    st = hs.stream_error()
    return tk.cpu().numpy(), (tv.cpu().numpy() if tv is not None else None), off.cpu().numpy(), st


def assert_equal(got, exp, what=""):
    if not np.array_equal(got, exp):
        bad = np.flatnonzero(got != exp) if got.shape == exp.shape else None
        where = f" first mismatch at {bad[0]} of {got.size} ({bad.size} differ)" if bad is not None and bad.size else ""
        raise AssertionError(f"{what} differs from the oracle:{where}")
