"""GPU: every built tile shape (items per thread of the tile sort and the
merge passes) gives the oracle's result, stage by stage: the tile sort's
state against the oracle's tile sort with that tile, the state after merge
passes against the oracle's tile sort with tile x fan_in^r, and the whole
sort (keys, stable values, packet offsets).  Sizes span several tiles with
ragged tails; a batch mixes short segments (sorted whole) and long ones."""
import numpy as np
import pytest
import torch

import paper_2003_01216_gb300 as hs
from gpu_util import assert_equal, dev, run, to_dev
from paper_2003_01216_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CASES = [(0, False, "uniform1e9"), (0, True, "zipf"), (1, False, "uniform32"), (1, True, "distinct16"),
         (2, False, "uniform64"), (2, True, "distinct2p24")]
SHAPES = [(code, hv, dist, tile) for code, hv, dist in CASES for tile in hs.tiles(code, hv)]


def test_built_tiles():
    assert hs.tiles(0) == [3840, 5888, 7936] == hs.tiles(1)
    assert hs.tiles(0, True) == [2816, 3840] == hs.tiles(2) == hs.tiles(2, True) == hs.tiles(1, True)


def _keys(dist, code, n, seed):
    k = I.generate(dist, n, seed=seed)
    if code == 1 and k.dtype != np.uint32:
        k = k.astype(np.uint32)
    return k


@pytest.mark.parametrize("code,hv,dist,tile", SHAPES)
def test_tile_shape_stages_and_whole_sort(oracle, code, hv, dist, tile):
    for n in (tile - 1, tile, 5 * tile + 77, 70_001):
        keys = _keys(dist, code, n, seed=n)
        vals = I.index_values(n) if hv else None
        lay, lv, off = oracle.partition(keys, vals, 10)
        # tile sort alone
        gk, gv, go, st = run(keys, vals, stop_after=2, tile=tile)
        assert st == 0
        ek, ev = oracle.tile_sort(lay, off, tile, lv)
        assert_equal(gk, ek, f"tile {tile} n {n}: tile-sort keys")
        if hv:
            assert_equal(gv, ev, f"tile {tile} n {n}: tile-sort values")
        # one merge pass, two-way and four-way
        for fan in (2, 4):
            gk, gv, _, st = run(keys, vals, stop_after=3, tile=tile, fan_in=fan)
            assert st == 0
            ek, ev = oracle.tile_sort(lay, off, tile * fan, lv)
            assert_equal(gk, ek, f"tile {tile} n {n} fan {fan}: state after pass 1")
            if hv:
                assert_equal(gv, ev, f"tile {tile} n {n} fan {fan}: values after pass 1")
        # the whole sort
        ek, ev, eo = oracle.sort(keys, vals)
        for fan in (2, 4):
            gk, gv, go, st = run(keys, vals, tile=tile, fan_in=fan)
            assert st == 0
            assert_equal(gk, ek, f"tile {tile} n {n} fan {fan}: keys")
            assert_equal(go, eo, f"tile {tile} n {n} fan {fan}: packet offsets")
            if hv:
                assert_equal(gv, ev, f"tile {tile} n {n} fan {fan}: values")
        p = hs.plan(code, n, hv, tile=tile, fan_in=2)
        assert p["tile"] == tile
        tiles_max = -(-n // tile)
        assert p["merge_passes"] == (0 if tiles_max <= 1 else int(tiles_max - 1).bit_length())


@pytest.mark.parametrize("code,hv,dist,tile", SHAPES)
def test_tile_shape_batch(oracle, code, hv, dist, tile):
    lens = I.log_uniform_lengths(120, 1, 6 * tile, seed=tile)
    lens[::9] = 0
    off = np.zeros(lens.size + 1, dtype=np.uint64)
    off[1:] = np.cumsum(lens)
    keys = _keys(dist, code, int(off[-1]), seed=3)
    vals = I.index_values(keys.size) if hv else None
    ek, ev = oracle.sort_batch(keys, off, vals)
    tk = to_dev(keys)
    tv = to_dev(vals) if hv else None
    hs.sort_batch(tk, to_dev(off), tv, tile=tile)
    assert hs.stream_error() == 0
    assert_equal(tk.cpu().numpy(), ek, f"batch tile {tile}: keys")
    if hv:
        assert_equal(tv.cpu().numpy(), ev, f"batch tile {tile}: values")


def test_unbuilt_tile_is_rejected():
    t = torch.zeros(100, dtype=torch.uint64, device=dev())
    with pytest.raises(hs.HsError):
        hs.sort_keys(t, tile=7936)  # 7936 is built for 4-byte keys without values only
    with pytest.raises(hs.HsError):
        hs.sort_keys(t, tile=1000)
