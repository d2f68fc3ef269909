"""GPU parity: every stage and the whole sort against the CPU oracle,
element by element, bit-exact (integer work).  Sizes span several tiles and
packet-step blocks (TILE keys each) with ragged tails, plus the edge cases:
one key, one tile exactly, tile +- 1, empty packets, all-equal, negative
int32 keys, the largest uint64 digit width."""
import numpy as np
import pytest

import paper_2003_01216_gb300 as hs
from gpu_util import assert_equal, run
from paper_2003_01216_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# merge shapes: two-way passes in one persistent launch (merge = 1), two-way
# passes with a launch each (merge = 2), four-way passes
SHAPES = [(2, 1), (2, 2), (4, 0)]
SHAPE_IDS = ["fan2-queue", "fan2-per-pass", "fan4"]

TILE = hs.plan(0, 1 << 20)["tile"]                    # int32 keys: keys per tile and merge block
TILE_PAIRS = hs.plan(0, 1 << 20, has_vals=True)["tile"]  # pairs (and 64-bit keys)
PART = hs.plan(0, 1 << 20)["part_tile"]                # keys per packet-step block
SIZES = sorted({1, 2, 100, TILE - 1, TILE, TILE + 1, PART - 1, PART, PART + 1, 3 * TILE + 123, 65536 + 17,
                300_001})


def tile_of(keys, has_vals):
    return hs.plan(hs.dtype_code(__import__("torch").from_numpy(keys[:1])), 1 << 20, has_vals=has_vals)["tile"]
DISTS = ["uniform31", "uniform1e9", "zipf", "sorted", "reverse", "equal", "distinct16", "int32full",
         "three_digit", "uniform32", "uniform64", "distinct2p24"]


@pytest.mark.parametrize("dist", DISTS)
def test_device_generator_matches_host(dist):
    for n in (1, 1000, 100_003):
        h = I.generate(dist, n, seed=9, stream=3)
        d = I.device_generate(dist, n, seed=9, stream=3)
        assert_equal(d.cpu().numpy(), h, f"device generator {dist} n={n}")


@pytest.mark.parametrize("nb", [1, 10, 256])
@pytest.mark.parametrize("dist", DISTS)
def test_partition_stage(oracle, dist, nb):
    # the packet step alone: stable layout and packet offsets, bit-exact
    for n in (1, TILE + 1, 65536 + 17, 300_001):
        keys = I.generate(dist, n, seed=1)
        vals = I.index_values(n)
        ek, ev, eoff = oracle.partition(keys, vals, nb)
        gk, _, goff, st = run(keys, None, nb, stop_after=1)
        assert st == 0
        assert_equal(goff, eoff, f"packet offsets {dist} n={n}")
        assert_equal(gk, ek, f"packet layout {dist} n={n}")
        gk, gv, _, st = run(keys, vals, nb, stop_after=1)
        assert st == 0
        assert_equal(gk, ek, f"packet layout (pairs) {dist} n={n}")
        assert_equal(gv, ev, f"packet layout values {dist} n={n}")


@pytest.mark.parametrize("nb", [1, 10, 256])
@pytest.mark.parametrize("dist", ["uniform1e9", "zipf", "reverse", "distinct16", "uniform64", "distinct2p24"])
def test_tilesort_stage(oracle, dist, nb):
    # packet step + tile sort: every tile of every packet sorted on its own
    for n in (TILE + 1, TILE_PAIRS + 1, 3 * TILE + 123, 300_001):
        keys = I.generate(dist, n, seed=2)
        vals = I.index_values(n)
        lk, lv, off = oracle.partition(keys, vals, nb)
        ek, ev = oracle.tile_sort(lk, off, tile_of(keys, True), lv)
        gk, gv, _, st = run(keys, vals, nb, stop_after=2)
        assert st == 0
        assert_equal(gk, ek, f"tile-sorted keys {dist} n={n}")
        assert_equal(gv, ev, f"tile-sorted values {dist} n={n}")
        ek, _ = oracle.tile_sort(lk, off, tile_of(keys, False))
        gk, _, _, st = run(keys, None, nb, stop_after=2)
        assert st == 0
        assert_equal(gk, ek, f"tile-sorted keys (keys only) {dist} n={n}")


@pytest.mark.parametrize("fan,merge", SHAPES, ids=SHAPE_IDS)
@pytest.mark.parametrize("nb", [1, 10, 256])
@pytest.mark.parametrize("dist", DISTS)
def test_sort_keys(oracle, dist, nb, fan, merge):
    for n in SIZES:
        keys = I.generate(dist, n, seed=3)
        ek, _, eoff = oracle.sort(keys, None, nb)
        gk, _, goff, st = run(keys, None, nb, fan_in=fan, merge=merge)
        assert st == 0
        assert_equal(gk, ek, f"sorted keys {dist} n={n}")
        assert_equal(goff, eoff, f"packet offsets {dist} n={n}")


@pytest.mark.parametrize("fan,merge", SHAPES, ids=SHAPE_IDS)
@pytest.mark.parametrize("nb", [1, 10, 256])
@pytest.mark.parametrize("dist", ["uniform31", "zipf", "equal", "distinct16", "int32full", "uniform32",
                                  "uniform64", "distinct2p24"])
def test_sort_pairs_stable(oracle, dist, nb, fan, merge):
    for n in SIZES:
        keys = I.generate(dist, n, seed=4)
        vals = I.index_values(n)
        ek, ev, _ = oracle.sort(keys, vals, nb)
        gk, gv, _, st = run(keys, vals, nb, fan_in=fan, merge=merge)
        assert st == 0
        assert_equal(gk, ek, f"pair keys {dist} n={n}")
        assert_equal(gv, ev, f"pair values (stable order) {dist} n={n}")


@pytest.mark.parametrize("dist", ["uniform31", "zipf", "sorted", "reverse", "equal", "distinct16", "uniform64"])
def test_fan4_group_shapes(oracle, dist):
    # one packet (no MSD step), so the run geometry is exact: groups of four
    # runs, ragged last groups of one, two and three runs, and packets needing
    # one to three passes of four-way merges; keys and stable pairs
    sizes = []
    for tiles in (2, 3, 4, 5, 7, 8, 9, 15, 16, 17, 33, 63, 64, 65):
        sizes += [tiles * TILE - 1, tiles * TILE + 1]
    for n in sizes:
        keys = I.generate(dist, n, seed=40)
        ek, _, _ = oracle.sort(keys, None, 1)
        gk, _, _, st = run(keys, None, 1, fan_in=4)
        assert st == 0
        assert_equal(gk, ek, f"fan-in 4 keys {dist} n={n}")
    for n in (2 * TILE_PAIRS + 7, 5 * TILE_PAIRS + 3, 17 * TILE_PAIRS + 1, 70 * TILE_PAIRS + 11):
        keys = I.generate(dist, n, seed=41)
        vals = I.index_values(n)
        ek, ev, _ = oracle.sort(keys, vals, 1)
        gk, gv, _, st = run(keys, vals, 1, fan_in=4)
        assert st == 0
        assert_equal(gk, ek, f"fan-in 4 pair keys {dist} n={n}")
        assert_equal(gv, ev, f"fan-in 4 pair values {dist} n={n}")


def test_fan4_large(oracle):
    # 2^22 keys in ten packets: up to five four-way passes with multi-chunk groups
    for dist in ("uniform1e9", "zipf"):
        keys = I.generate(dist, 1 << 22, seed=42)
        ek, _, eoff = oracle.sort(keys, None, 10)
        gk, _, goff, st = run(keys, None, 10, fan_in=4)
        assert st == 0
        assert_equal(gk, ek, f"fan-in 4 sorted keys {dist}")
        assert_equal(goff, eoff, f"fan-in 4 packet offsets {dist}")


def test_config1_plain_keys(oracle):
    # 1,048,576 int32 keys uniform in [0, 10^9) from seed 0: D = 9, packet = key / 10^8
    keys = I.generate("uniform1e9", 1 << 20, seed=0)
    ek, _, eoff = oracle.sort(keys, None, 10)
    gk, _, goff, st = run(keys)
    assert st == 0
    assert_equal(gk, ek, "config 1 sorted keys")
    assert_equal(goff, eoff, "config 1 packet offsets")
    counts = np.diff(goff.astype(np.int64))
    assert counts.size == 10 and np.all(np.abs(counts - (1 << 20) / 10) < 5 * 310)


def test_special_values(oracle):
    for dt in (np.int32, np.uint32, np.uint64):
        info = np.iinfo(dt)
        base = np.array([info.max, info.min, 0, 9, 10, 99, 100, info.max, 1], dtype=dt)
        keys = np.tile(base, 1000)
        for nb in (10, 256):
            ek, _, eoff = oracle.sort(keys, None, nb)
            gk, _, goff, st = run(keys, None, nb)
            assert st == 0
            assert_equal(gk, ek, f"special values {dt}")
            assert_equal(goff, eoff, f"special values offsets {dt}")


def test_empty_input():
    gk, _, goff, st = run(np.zeros(0, np.int32))
    assert gk.size == 0 and st == 0 and np.all(goff == 0)


@pytest.mark.parametrize("dist", ["reverse", "sorted", "equal", "distinct16", "uniform31", "int32full"])
def test_persistent_ctas_loop_over_many_blocks(oracle, dist):
    # 2^23 keys: every persistent CTA of the packet step and the tile sort
    # handles many blocks in turn (the sizes above give each at most one), and
    # sorted / reverse inputs make every block a single run of one packet
    n = (1 << 23) + 1234
    keys = I.generate(dist, n, seed=45)
    vals = I.index_values(n)
    lk, lv, loff = oracle.partition(keys, vals, 10)
    for rep in range(2):
        gk, gv, goff, st = run(keys, vals, 10, stop_after=1)
        assert st == 0
        assert_equal(goff, loff, f"{dist} packet offsets (pass {rep})")
        assert_equal(gk, lk, f"{dist} packet layout (pass {rep})")
        assert_equal(gv, lv, f"{dist} packet layout values (pass {rep})")
    ek, ev, _ = oracle.sort(keys, vals, 10)
    for fan, merge in SHAPES:
        gk, gv, _, st = run(keys, vals, 10, fan_in=fan, merge=merge)
        assert st == 0
        assert_equal(gk, ek, f"{dist} pair keys fan-in {fan}")
        assert_equal(gv, ev, f"{dist} pair values fan-in {fan}")
        gk, _, _, st = run(keys, None, 10, fan_in=fan, merge=merge)
        assert st == 0
        assert_equal(gk, ek, f"{dist} keys fan-in {fan}")


@pytest.mark.parametrize("fan,merge", SHAPES, ids=SHAPE_IDS)
@pytest.mark.parametrize("nb", [1, 10])
@pytest.mark.parametrize("dist", ["uniform1e9", "zipf", "uniform64", "distinct2p24"])
def test_merge_passes_one_by_one(oracle, dist, nb, fan, merge):
    # the state after every merge pass r: inside each packet every group of
    # fan^r tiles is sorted on its own (pairs stably), the rest untouched by
    # later passes -- the oracle's tile sort with tile * fan^r
    n = 40 * TILE + 123
    keys = I.generate(dist, n, seed=46)
    vals = I.index_values(n)
    lk, lv, off = oracle.partition(keys, vals, nb)
    for has_vals in (False, True):
        tile = tile_of(keys, has_vals)
        code = hs.dtype_code(__import__("torch").from_numpy(keys[:1]))
        passes = hs.plan(code, n, has_vals, partition=nb, fan_in=fan)["merge_passes"]
        assert passes >= 2
        for r in range(1, passes + 1):
            ek, ev = oracle.tile_sort(lk, off, tile * fan ** r, lv if has_vals else None)
            gk, gv, goff, st = run(keys, vals if has_vals else None, nb, stop_after=2 + r, fan_in=fan, merge=merge)
            assert st == 0
            assert_equal(goff, off, f"{dist} packet offsets after pass {r}")
            assert_equal(gk, ek, f"{dist} keys after merge pass {r} (fan-in {fan}, values {has_vals})")
            if has_vals:
                assert_equal(gv, ev, f"{dist} values after merge pass {r} (fan-in {fan})")


@pytest.mark.parametrize("case", ["g16_keys", "g4_keys", "g4_pairs"])
def test_corank_lane_groups(oracle, case):
    # two-way merge passes at sizes that take each co-rank shape: 16 lanes per
    # search (at most 4096 merge blocks), 4 lanes (at most 16384), keys and
    # stable pairs, ten packets and one packet, spread keys and heavy ties
    n = {"g16_keys": (1 << 22) + 77, "g4_keys": (1 << 25) + 999, "g4_pairs": 16_000_003}[case]
    has_vals = case.endswith("pairs")
    dists = ["uniform64", "distinct2p24"] if has_vals else ["uniform31", "distinct16"]
    for dist in dists:
        keys = I.generate(dist, n, seed=47)
        vals = I.index_values(n) if has_vals else None
        for nb in (10, 1):
            ek, ev, eoff = oracle.sort(keys, vals, nb)
            gk, gv, goff, st = run(keys, vals, nb, fan_in=2)
            assert st == 0
            assert_equal(goff, eoff, f"{case} {dist} nb={nb} packet offsets")
            assert_equal(gk, ek, f"{case} {dist} nb={nb} keys")
            if has_vals:
                assert_equal(gv, ev, f"{case} {dist} nb={nb} values (stable order)")
