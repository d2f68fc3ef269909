"""Seeded synthetic inputs (host side, numpy).

This module only makes inputs; it holds none of the sort's arithmetic.  Both
the CPU oracle (through the tests) and the GPU library are fed from it, and
the device-side generator in ``csrc/gen.cu`` implements the same definitions
bit for bit, so large inputs never have to cross PCIe.

Every value derives from one counter-based generator: the i-th output of a
SplitMix64 stream (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; output mixer constants of Vigna's splitmix64.c):

    mix64(z):  z ^= z >> 30; z *= 0xbf58476d1ce4e5b9;
               z ^= z >> 27; z *= 0x94d049bb133111eb;  z ^= z >> 31
    base(seed, stream) = mix64(seed * GAMMA + stream)
    h(seed, stream, i) = mix64(base + (i + 1) * GAMMA),   GAMMA = 0x9e3779b97f4a7c15

all arithmetic mod 2^64.  The paper itself sorts randomly generated
three-digit integers (Sec. 4.2); the larger workloads below keep that kind of
data (uniform random integers) and add the skewed shapes a packet partition
has to survive.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
MASK64 = (1 << 64) - 1

# distribution codes shared with the device generator (csrc/gen.cu)
DIST = {
    "uniform31": 0,      # int32  h & 0x7fffffff                  uniform [0, 2^31)
    "uniform1e9": 1,     # int32  h mod 10^9                      uniform [0, 10^9)
    "zipf": 2,           # int32  Zipf s=1.1 over 2^20 values, spread by a bijection, << 11
    "sorted": 3,         # int32  floor(i * 2^31 / n)
    "reverse": 4,        # int32  floor((n-1-i) * 2^31 / n)
    "equal": 5,          # int32  123456789
    "distinct16": 6,     # int32  (h & 15) * 2^27 + 12345
    "uniform64": 7,      # uint64 h
    "distinct2p24": 8,   # uint64 h'(h mod 2^24): 2^24 distinct 64-bit values
    "uniform32": 9,      # uint32 h & 0xffffffff
    "int32full": 10,     # int32  (int32)(h & 0xffffffff): negative keys too
    "three_digit": 11,   # int32  h mod 1000 (the paper's own data, Sec. 4.2)
}
DTYPE_OF = {
    "uniform31": np.int32, "uniform1e9": np.int32, "zipf": np.int32, "sorted": np.int32,
    "reverse": np.int32, "equal": np.int32, "distinct16": np.int32, "uniform64": np.uint64,
    "distinct2p24": np.uint64, "uniform32": np.uint32, "int32full": np.int32,
    "three_digit": np.int32,
}
PLAIN_AT_SCALE = ["uniform31", "zipf", "sorted", "reverse", "equal", "distinct16"]

ZIPF_S = 1.1
ZIPF_N = 1 << 20


def mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z ^ (z >> np.uint64(30))
        z = z * M1
        z = z ^ (z >> np.uint64(27))
        z = z * M2
        z = z ^ (z >> np.uint64(31))
    return z


def stream_base(seed: int, stream: int) -> np.uint64:
    v = (int(seed) * int(GAMMA) + int(stream)) & MASK64
    return mix64(np.array([v], dtype=np.uint64))[0]


def hashes(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """h(seed, stream, i) for i in [start, start + n)."""
    b = stream_base(seed, stream)
    i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(b + i * GAMMA)


def unit_double(h: np.ndarray) -> np.ndarray:
    """Uniform double in [0, 1) from the top 53 bits (exact)."""
    return (h >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


_zipf_cdf: np.ndarray | None = None


def zipf_cdf() -> np.ndarray:
    """Cumulative Zipf(s=1.1) weights over ranks 0..2^20-1, last entry exactly 1."""
    global _zipf_cdf
    if _zipf_cdf is None:
        w = np.arange(1, ZIPF_N + 1, dtype=np.float64) ** (-ZIPF_S)
        c = np.cumsum(w)
        _zipf_cdf = c / c[-1]
        _zipf_cdf[-1] = 1.0
    return _zipf_cdf


def perm20(x: np.ndarray) -> np.ndarray:
    """A fixed bijection on 20-bit integers: odd multiply mod 2^20, then xorshift."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        y = (x * np.uint64(0x9E3779B1)) & np.uint64(0xFFFFF)
    return y ^ (y >> np.uint64(10))


def generate(dist: str, n: int, seed: int = 0, stream: int = 0) -> np.ndarray:
    """n keys of the named distribution (see DIST), as numpy in its key dtype."""
    code = DIST[dist]
    dt = DTYPE_OF[dist]
    if n == 0:
        return np.zeros(0, dtype=dt)
    if dist in ("sorted", "reverse"):
        i = np.arange(n, dtype=np.uint64)
        if dist == "reverse":
            i = np.uint64(n - 1) - i
        return ((i << np.uint64(31)) // np.uint64(n)).astype(np.int32)
    if dist == "equal":
        return np.full(n, 123456789, dtype=np.int32)
    h = hashes(seed, stream, n)
    if code == 0:
        return (h & np.uint64(0x7FFFFFFF)).astype(np.int32)
    if code == 1:
        return (h % np.uint64(1_000_000_000)).astype(np.int32)
    if code == 2:
        r = np.searchsorted(zipf_cdf(), unit_double(h), side="right").astype(np.uint64)
        return (perm20(r) << np.uint64(11)).astype(np.int32)
    if code == 6:
        return ((h & np.uint64(15)) * np.uint64(1 << 27) + np.uint64(12345)).astype(np.int32)
    if code == 7:
        return h
    if code == 8:
        b2 = stream_base(seed, stream ^ 0xFFFF)
        with np.errstate(over="ignore"):
            return mix64(b2 + ((h & np.uint64((1 << 24) - 1)) + np.uint64(1)) * GAMMA)
    if code == 9:
        return (h & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    if code == 10:
        return (h & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.int32)
    if code == 11:
        return (h % np.uint64(1000)).astype(np.int32)
    raise ValueError(dist)


def index_values(n: int) -> np.ndarray:
    """Values of a key-value workload: the input index (a stability witness)."""
    return np.arange(n, dtype=np.uint32)


# --------------------------------------------------------------------------
# batched workload: segment lengths log-uniform in [lo, hi]
# --------------------------------------------------------------------------
SEGLEN_STREAM = 0x5E6
ARRIVAL_STREAM = 0xA77


def log_uniform_lengths(count: int, lo: int, hi: int, seed: int = 0, stream: int = SEGLEN_STREAM):
    """floor(exp(U[ln lo, ln(hi + 1)))), clipped to [lo, hi]."""
    u = unit_double(hashes(seed, stream, count))
    a, b = math.log(lo), math.log(hi + 1)
    ln = np.floor(np.exp(a + u * (b - a))).astype(np.int64)
    return np.clip(ln, lo, hi)


def batch_offsets(count: int, lo: int, hi: int, seed: int = 0) -> np.ndarray:
    lens = log_uniform_lengths(count, lo, hi, seed)
    off = np.zeros(count + 1, dtype=np.uint64)
    off[1:] = np.cumsum(lens, dtype=np.uint64)
    return off


def poisson_requests(rate: float, duration: float, lo: int, hi: int, seed: int = 0):
    """Serving workload: (arrival times s, dtype codes 0=int32/2=uint64, lengths)."""
    # draw enough exponential gaps to cover the duration
    m = int(rate * duration * 1.2) + 64
    h = hashes(seed, ARRIVAL_STREAM, 3 * m)
    gaps = -np.log1p(-unit_double(h[0::3])) / rate
    t = np.cumsum(gaps)
    keep = t < duration
    t = t[keep]
    k = t.size
    dtype_codes = np.where((h[1::3][:k] & np.uint64(1)) == 0, 0, 2).astype(np.int32)
    u = unit_double(h[2::3][:k])
    a, b = math.log(lo), math.log(hi + 1)
    lens = np.clip(np.floor(np.exp(a + u * (b - a))).astype(np.int64), lo, hi)
    return t, dtype_codes, lens


def request_dist(dtype_code: int) -> str:
    """Serving payloads: uniform values of the request's dtype."""
    return "uniform31" if dtype_code == 0 else "uniform64"


# --------------------------------------------------------------------------
# device twin (libhsgen.so): the same keys written straight into GPU memory
# --------------------------------------------------------------------------
_gen_lib = None
_cdf_dev: dict = {}


def _gen():
    global _gen_lib
    if _gen_lib is None:
        import ctypes
        import os
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libhsgen.so")
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is not built")
        L = ctypes.CDLL(path)
        u64, p = ctypes.c_uint64, ctypes.c_void_p
        L.hsg_fill.argtypes = [ctypes.c_int, u64, u64, u64, u64, p, ctypes.c_int, p, u64, p]
        L.hsg_fill.restype = ctypes.c_int
        L.hsg_iota.argtypes = [p, u64, p]
        L.hsg_iota.restype = ctypes.c_int
        _gen_lib = L
    return _gen_lib


def device_generate(dist: str, n: int, seed: int = 0, stream: int = 0, out=None, device=None):
    """The keys of generate(dist, n, seed, stream), produced on the GPU."""
    import torch
    tdt = {np.int32: torch.int32, np.uint32: torch.uint32, np.uint64: torch.uint64}[DTYPE_OF[dist]]
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    if out is None:
        out = torch.empty(n, dtype=tdt, device=dev)
    cdf_ptr, cdf_n = None, 0
    if dist == "zipf":
        key = out.device.index
        if key not in _cdf_dev:
            _cdf_dev[key] = torch.from_numpy(zipf_cdf()).to(out.device)
        cdf_ptr, cdf_n = _cdf_dev[key].data_ptr(), ZIPF_N
    s = torch.cuda.current_stream(out.device).cuda_stream
    rc = _gen().hsg_fill(DIST[dist], seed, stream, n, 0, out.data_ptr() if n else None, out.element_size(),
                         cdf_ptr, cdf_n, s)
    if rc:
        raise RuntimeError(f"hsg_fill failed ({rc})")
    return out


def device_index_values(n: int, out=None, device=None):
    import torch
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    if out is None:
        out = torch.empty(n, dtype=torch.uint32, device=dev)
    rc = _gen().hsg_iota(out.data_ptr() if n else None, n, torch.cuda.current_stream(out.device).cuda_stream)
    if rc:
        raise RuntimeError(f"hsg_iota failed ({rc})")
    return out
