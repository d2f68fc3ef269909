"""GPU: segments of at most one tile are sorted whole by one CTA (no packet
step, no merge passes) and must still give the oracle's keys, stable values
and packet offsets (the packet rule applied to the segment alone).  Covers
the tile boundary (tile - 1, tile, tile + 1 keys), one-key and all-equal
segments, negative int32 keys (sign-flipped image), keys at the type's
maximum, the 256-bucket and one-packet variants, and a plain call on one
short array."""
import numpy as np
import pytest
import torch

import paper_2003_01216_gb300 as hs
from gpu_util import assert_equal, dev, run, to_dev
from paper_2003_01216_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DTYPE_CODE = {np.dtype(np.int32): 0, np.dtype(np.uint32): 1, np.dtype(np.uint64): 2}


def edge_lengths(tile):
    return [1, 2, 3, 31, 32, 33, 1000, tile - 1, tile, tile + 1, 0, 5, tile, 2 * tile + 3, 17, tile - 31, 9]


def special_keys(dist, n, seed):
    keys = I.generate(dist, n, seed=seed)
    if keys.size > 40:
        keys[:8] = keys[8]                          # a run of equal keys
        keys[20] = np.iinfo(keys.dtype).max         # the largest key
        keys[21] = np.iinfo(keys.dtype).min
    return keys


def check_batch(oracle, keys, off, nb, with_vals):
    n = keys.size
    nseg = off.size - 1
    vals = I.index_values(n) if with_vals else None
    ek, ev = oracle.sort_batch(keys, off, vals, nbuckets=nb)
    tk, to = to_dev(keys), to_dev(off)
    tv = to_dev(vals) if with_vals else None
    poff = torch.zeros(nseg * nb + 1, dtype=torch.uint64, device=dev())
    hs.sort_batch(tk, to, tv, partition=nb, packet_offsets=poff)
    assert hs.stream_error() == 0
    assert_equal(tk.cpu().numpy(), ek, "keys")
    if with_vals:
        assert_equal(tv.cpu().numpy(), ev, "stable values")
    po = poff.cpu().numpy()
    for s in range(nseg):
        lo, hi = int(off[s]), int(off[s + 1])
        _, _, so = oracle.partition(keys[lo:hi], None, nb)
        assert_equal(po[s * nb:(s + 1) * nb + 1], so + np.uint64(lo), f"segment {s} (length {hi - lo}) packet offsets")


@pytest.mark.parametrize("with_vals", [False, True])
@pytest.mark.parametrize("nb", [1, 10, 256])
@pytest.mark.parametrize("dist", ["uniform1e9", "int32full", "uniform32", "uniform64", "distinct16"])
def test_short_segments_at_the_tile_boundary(oracle, dist, nb, with_vals):
    code = DTYPE_CODE[np.dtype(I.DTYPE_OF[dist])]
    tile = hs.plan(code, 1 << 20, with_vals)["tile"]
    lens = np.array(edge_lengths(tile) * 3, dtype=np.int64)
    off = np.zeros(lens.size + 1, dtype=np.uint64)
    off[1:] = np.cumsum(lens)
    keys = special_keys(dist, int(off[-1]), seed=31)
    check_batch(oracle, keys, off, nb, with_vals)


@pytest.mark.parametrize("dist", ["uniform31", "int32full", "uniform64"])
def test_many_short_segments_among_long_ones(oracle, dist):
    # 2000 segments, most of them short (lengths log-uniform in [1, 40000]),
    # so the tile sort launch holds thousands of whole-segment items beside
    # the tiles of the long segments' packets
    lens = I.log_uniform_lengths(2000, 1, 40_000, seed=3)
    lens[::11] = 0
    off = np.zeros(lens.size + 1, dtype=np.uint64)
    off[1:] = np.cumsum(lens)
    keys = I.generate(dist, int(off[-1]), seed=4)
    check_batch(oracle, keys, off, 10, True)


@pytest.mark.parametrize("nb", [1, 10, 256])
@pytest.mark.parametrize("dist", ["uniform1e9", "int32full", "uniform64", "equal"])
def test_plain_short_array(oracle, dist, nb):
    code = DTYPE_CODE[np.dtype(I.DTYPE_OF[dist])]
    tile = hs.plan(code, 1 << 20)["tile"]
    for n in (1, 2, 100, tile - 1, tile):
        keys = special_keys(dist, n, seed=n)
        launches0 = hs.kernel_launches()
        gk, _, go, st = run(keys, nb=nb)
        # a short array costs three launches: segment table, plan, tile sort
        assert hs.kernel_launches() - launches0 == 3 == hs.plan(code, n, partition=nb)["launches"]
        assert st == 0
        ek, _, eo = oracle.sort(keys, None, nb)
        assert_equal(gk, ek, f"n = {n} keys")
        assert_equal(go, eo, f"n = {n} packet offsets")
        vals = I.index_values(n)
        gk, gv, _, st = run(keys, vals, nb=nb)
        ek, ev, _ = oracle.sort(keys, vals, nb)
        assert st == 0
        assert_equal(gk, ek, f"n = {n} pair keys")
        assert_equal(gv, ev, f"n = {n} pair values")
