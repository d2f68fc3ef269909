"""Reader for the hand-worked fixtures in tests/golden/ and definitions used to
pin the oracle.  The helpers here restate the paper's packet rule in the most
literal way (decimal strings), independent of the oracle's integer arithmetic.
"""
from __future__ import annotations

import glob
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NP_DTYPE = {"int32": np.int32, "uint32": np.uint32, "uint64": np.uint64}


def load(path: str) -> dict:
    out = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = (s.strip() for s in line.split("=", 1))
            out[k] = v
    dt = NP_DTYPE[out["dtype"]]
    fx = {"name": os.path.basename(path), "dtype": dt, "nbuckets": int(out["nbuckets"])}
    for k in ("keys", "layout", "sorted"):
        fx[k] = np.array([int(x) for x in out[k].split()], dtype=object).astype(dt)
    for k in ("vals", "layout_vals", "sorted_vals"):
        if k in out:
            fx[k] = np.array([int(x) for x in out[k].split()], dtype=np.uint32)
    fx["width"] = int(out["width"])
    fx["flip"] = bool(int(out["flip"]))
    nb = fx["nbuckets"]
    if "offsets" in out:
        fx["offsets"] = np.array([int(x) for x in out["offsets"].split()], dtype=np.uint64)
    else:
        counts = np.zeros(nb, dtype=np.uint64)
        for item in out["counts_sparse"].split():
            p, c = item.split(":")
            counts[int(p)] = int(c)
        off = np.zeros(nb + 1, dtype=np.uint64)
        off[1:] = np.cumsum(counts)
        fx["offsets"] = off
    return fx


def all_fixtures() -> list[dict]:
    return [load(p) for p in sorted(glob.glob(os.path.join(GOLDEN, "*.txt"))) if not p.endswith("README.txt")]


# --- literal restatement of the packet rule (Sec. 2.1 / Sec. 3.4) ----------

def image_literal(keys: np.ndarray) -> list[int]:
    """Python ints: key, or key + 2^31 for int32 arrays holding a negative key."""
    ks = [int(k) for k in keys]
    if keys.dtype == np.int32 and any(k < 0 for k in ks):
        return [k + 2**31 for k in ks]
    return ks


def packets_literal(keys: np.ndarray, nbuckets: int) -> list[int]:
    """Packet of each key: the leading digit of the key image written with as
    many digits as the largest image (decimal), or its top byte (256)."""
    u = image_literal(keys)
    if not u:
        return []
    m = max(u)
    if nbuckets == 10:
        D = len(str(m))
        return [int(str(x).zfill(D)[0]) for x in u]
    shift = max(0, m.bit_length() - 8)
    return [x >> shift for x in u]


def stable_layout_literal(keys: np.ndarray, nbuckets: int, vals=None):
    """Keys (and values) grouped by packet, input order inside each packet."""
    p = packets_literal(keys, nbuckets)
    order = sorted(range(len(p)), key=lambda i: p[i])  # Python's sort is stable
    lay = keys[np.array(order, dtype=np.int64)] if order else keys[:0]
    lv = None if vals is None else (vals[np.array(order, dtype=np.int64)] if order else vals[:0])
    counts = np.bincount(np.array(p, dtype=np.int64), minlength=nbuckets) if p else np.zeros(nbuckets, np.int64)
    off = np.zeros(nbuckets + 1, dtype=np.uint64)
    off[1:] = np.cumsum(counts)
    return lay, lv, off


def stable_sorted_literal(keys: np.ndarray, vals: np.ndarray):
    """Pairs in key order, ties in input order (Python's stable sort)."""
    order = sorted(range(len(keys)), key=lambda i: int(keys[i]))
    idx = np.array(order, dtype=np.int64)
    return keys[idx], vals[idx]
