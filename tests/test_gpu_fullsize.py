"""GPU parity at the full workload sizes, in the launch configuration the
benchmark times (one hs_sort_keys / hs_sort_pairs call on the whole array):

  * 268,435,456 int32 keys, six distributions, 10 packets (and 256 buckets
    for the uniform case): uniform [0, 2^31) and Zipf are compared element
    by element with the oracle's full sort; sorted, reverse, all-equal and
    16-distinct inputs against their closed-form sorted order; every packet
    offset against the oracle's packet step;
  * 134,217,728 stable uint64-key / uint32-value pairs (uniform 64-bit, and
    2^24 distinct keys): element by element against the oracle.

Inputs are made on the host by the seeded generator (never by the GPU)."""
import numpy as np
import pytest
import torch

import paper_2003_01216_gb300 as hs
from gpu_util import assert_equal, dev
from paper_2003_01216_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N_PLAIN = 268_435_456
N_PAIRS = 134_217_728
_cache = {}


def gpu_sort(keys, vals=None, nb=10, fan_in=0):
    tk = torch.from_numpy(keys).to(dev())
    tv = torch.from_numpy(vals).to(dev()) if vals is not None else None
    off = torch.zeros(nb + 1, dtype=torch.uint64, device=dev())
    if tv is None:
        hs.sort_keys(tk, partition=nb, packet_offsets=off, fan_in=fan_in)
    else:
        hs.sort_pairs(tk, tv, partition=nb, packet_offsets=off, fan_in=fan_in)
    assert hs.stream_error() == 0
    out = (tk.cpu().numpy(), tv.cpu().numpy() if tv is not None else None, off.cpu().numpy())
    del tk, tv
    torch.cuda.empty_cache()
    return out


def host_keys(dist):
    if dist not in _cache:
        _cache.clear()
        _cache[dist] = I.generate(dist, N_PLAIN, seed=0)
    return _cache[dist]


@pytest.mark.parametrize("dist", ["uniform31", "zipf"])
def test_fullsize_plain_vs_oracle(oracle, dist):
    keys = host_keys(dist)
    gk, _, goff = gpu_sort(keys)
    ek, _, eoff = oracle.sort(keys, None, 10)
    assert_equal(goff, eoff, f"{dist} packet offsets")
    assert_equal(gk, ek, f"{dist} sorted keys")
    # fan-in 4 merge passes: the same unique sorted output
    gk4, _, goff4 = gpu_sort(keys, fan_in=4)
    assert_equal(goff4, eoff, f"{dist} packet offsets (fan-in 4)")
    assert_equal(gk4, ek, f"{dist} sorted keys (fan-in 4)")
    # through pinned host memory, as the end-to-end benchmark sorts: read by
    # the histogram kernel, the last merge pass of every packet written back
    # to host memory by the merge queue
    pinned = torch.from_numpy(keys).pin_memory()
    hs.sort_keys_host(pinned)
    assert_equal(pinned.numpy(), ek, f"{dist} sorted keys through host memory")
    del pinned
    if dist == "uniform31":
        # 256-bucket ablation: same unique sorted output, its own offsets
        gk2, _, goff2 = gpu_sort(keys, nb=256)
        _, _, eoff2 = oracle.partition(keys, None, 256)
        assert_equal(goff2, eoff2, "256-bucket offsets")
        assert_equal(gk2, ek, "256-bucket sorted keys")


@pytest.mark.parametrize("dist", ["sorted", "reverse", "equal", "distinct16"])
@pytest.mark.parametrize("fan", [2, 4])
def test_fullsize_plain_closed_form(oracle, dist, fan):
    keys = host_keys(dist)
    gk, _, goff = gpu_sort(keys, fan_in=fan)
    _, _, eoff = oracle.partition(keys, None, 10)
    assert_equal(goff, eoff, f"{dist} packet offsets")
    if dist == "sorted" or dist == "equal":
        exp = keys
    elif dist == "reverse":
        exp = keys[::-1]
    else:  # 16 values c * 2^27 + 12345, in order, each repeated its count
        c = np.bincount((keys.astype(np.int64) - 12345) >> 27, minlength=16)
        exp = np.repeat((np.arange(16, dtype=np.int64) * (1 << 27) + 12345).astype(np.int32), c)
    assert_equal(gk, np.ascontiguousarray(exp), f"{dist} sorted keys")


@pytest.mark.parametrize("dist", ["uniform64", "distinct2p24"])
def test_fullsize_stable_pairs_vs_oracle(oracle, dist):
    _cache.clear()
    keys = I.generate(dist, N_PAIRS, seed=0)
    vals = I.index_values(N_PAIRS)
    gk, gv, goff = gpu_sort(keys, vals)
    ek, ev, eoff = oracle.sort(keys, vals, 10)
    assert_equal(goff, eoff, f"{dist} packet offsets")
    assert_equal(gk, ek, f"{dist} pair keys")
    assert_equal(gv, ev, f"{dist} pair values (stable order)")
    gk, gv, goff = gpu_sort(keys, vals, fan_in=4)
    assert_equal(goff, eoff, f"{dist} packet offsets (fan-in 4)")
    assert_equal(gk, ek, f"{dist} pair keys (fan-in 4)")
    assert_equal(gv, ev, f"{dist} pair values (stable order, fan-in 4)")
