"""The C-ABI library loads and exports every symbol include/hsort.h declares;
host-side argument checks and plan queries work without a GPU (no kernel is
launched by anything here)."""
import ctypes
import os
import re

import pytest

from paper_2003_01216_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "hsort.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hs_[a-z_0-9]+)\s*\(", src)))


def test_header_lists_the_abi():
    names = declared_functions()
    for want in ("hs_sort_keys", "hs_sort_pairs", "hs_sort_batch", "hs_stream_error", "hs_status_string"):
        assert want in names
    assert sorted(N.EXPORTS) == names


def test_library_exports_every_declared_symbol():
    lib = N.lib()
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_generator_library_exports():
    from paper_2003_01216_gb300 import inputs
    g = inputs._gen()
    assert hasattr(g, "hsg_fill") and hasattr(g, "hsg_iota")


def test_status_strings():
    lib = N.lib()
    for s in range(7):
        assert lib.hs_status_string(s)
    assert lib.hs_status_string(4).decode() == "bounded device wait expired"


def test_host_side_rejections():
    lib = N.lib()
    o = N.make_opts()
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: every call below fails its host checks first
    assert lib.hs_sort_keys(7, fake, 10, ctypes.byref(o), None) == N.HS_ERR_INVALID          # bad dtype
    assert lib.hs_sort_keys(0, None, 10, ctypes.byref(o), None) == N.HS_ERR_INVALID          # null keys
    assert lib.hs_sort_keys(0, fake, 1 << 32, ctypes.byref(o), None) == N.HS_ERR_INVALID     # n too large
    bad = N.make_opts(partition=7)
    assert lib.hs_sort_keys(0, fake, 10, ctypes.byref(bad), None) == N.HS_ERR_INVALID
    tile = N.make_opts(tile=1000)
    assert lib.hs_sort_keys(0, fake, 10, ctypes.byref(tile), None) == N.HS_ERR_UNSUPPORTED
    fan = N.make_opts(fan_in=3)
    assert lib.hs_sort_keys(0, fake, 10, ctypes.byref(fan), None) == N.HS_ERR_UNSUPPORTED
    assert lib.hs_sort_pairs(0, fake, None, 10, 1, ctypes.byref(o), None) == N.HS_ERR_INVALID  # null values
    assert lib.hs_sort_batch(0, fake, None, None, 3, 10, ctypes.byref(o), None) == N.HS_ERR_INVALID
    assert lib.hs_sort_batch(0, fake, None, fake, 0, 10, ctypes.byref(o), None) == N.HS_ERR_INVALID
    assert lib.hs_sort_keys(0, None, 0, ctypes.byref(o), None) == N.HS_OK                     # n = 0 no-op
    assert lib.hs_sort_keys_host(0, None, 5, None, None) == N.HS_ERR_INVALID
    # element alignment: keys to their size, values to 4, offsets to 8 (checked before any CUDA call)
    assert lib.hs_sort_keys(0, 0x1002, 10, ctypes.byref(o), None) == N.HS_ERR_INVALID
    assert lib.hs_sort_keys(2, 0x1004, 10, ctypes.byref(o), None) == N.HS_ERR_INVALID
    assert lib.hs_sort_pairs(0, 0x1000, 0x2002, 10, 1, ctypes.byref(o), None) == N.HS_ERR_INVALID
    assert lib.hs_sort_batch(0, 0x1000, None, 0x3004, 2, 10, ctypes.byref(o), None) == N.HS_ERR_INVALID
    assert lib.hs_sort_keys_host(2, 0x1004, 10, None, None) == N.HS_ERR_INVALID


@pytest.mark.parametrize("n", [1, 3839, 3840, 3841, 7935, 7936, 7937, 1 << 20, 1 << 28])
def test_plan_describe(n):
    import math

    import paper_2003_01216_gb300 as hs
    for dtype, has_vals, tile in [(N.HS_INT32, False, 256 * 31), (N.HS_UINT32, False, 256 * 31),
                                  (N.HS_INT32, True, 256 * 15), (N.HS_UINT64, False, 256 * 15),
                                  (N.HS_UINT64, True, 256 * 15)]:
        p = hs.plan(dtype, n, has_vals, fan_in=2)
        assert p["tile"] == tile and p["part_tile"] == 256 * 15
        tiles = -(-n // tile)
        passes = 0 if tiles <= 1 else math.ceil(math.log2(tiles))
        assert p["merge_passes"] == passes
        # seg_plan, histogram (+ flipped-image histogram for int32), finalize, fold, 3 scan
        # kernels, packet offsets, tile prefix, scatter, tile sort, 2 per merge pass; small
        # calls (<= 2^16 block x packet entries) run finalize .. tile prefix as one kernel
        blocks = -(-n // 3840) + 1
        small = blocks * 10 <= 1 << 16
        hist = 2 if dtype == N.HS_INT32 else 1
        # an array of at most one tile is sorted whole by the tile sort launch:
        # seg_plan, the one-CTA plan, tile sort
        short = n <= tile
        # fan-in 2: every merge pass in one persistent launch (merge = 1), or a
        # co-rank and a merge launch per pass (merge = 2); the default takes
        # the queue above 2^24 keys
        sched = 1 if passes else 0
        q = hs.plan(dtype, n, has_vals, fan_in=2, merge=1)
        assert q["launches"] == (3 if short else 1 + hist + (1 if small else 7) + 2 + sched)
        per_pass = hs.plan(dtype, n, has_vals, fan_in=2, merge=2)["launches"]
        assert per_pass == (3 if short else 1 + hist + (1 if small else 7) + 2 + 2 * passes)
        queue = not has_vals and n > 1 << (24 if dtype == N.HS_UINT64 else 26)
        assert p["launches"] == (q["launches"] if queue else per_pass)
        # without the MSD step: seg_plan, packet table, tile prefix, tile sort
        small1 = blocks <= 1 << 16
        assert hs.plan(dtype, n, has_vals, partition=1, fan_in=2, merge=1)["launches"] == (
            3 if short else (3 if small1 else 4) + sched)
        # the testing stop after the tile sort keeps the packet step
        assert hs.plan(dtype, n, has_vals, fan_in=2, stop_after=2)["launches"] == (
            1 + hist + (1 if small else 7) + 2)
        # fan-in 4: ceil(log4(tiles)) passes, still two launches each
        p4 = hs.plan(dtype, n, has_vals, fan_in=4)
        passes4 = 0 if tiles <= 1 else math.ceil(math.log(tiles, 4) - 1e-12)
        assert p4["fan_in"] == 4 and p4["merge_passes"] == passes4 == (passes + 1) // 2
        assert p4["launches"] == (3 if short else 1 + hist + (1 if small else 7) + 2 + 2 * passes4)
        assert p["fan_in"] == 2


def test_stop_after_merge_pass_plan():
    import paper_2003_01216_gb300 as hs
    full = hs.plan(N.HS_INT32, 1 << 24, fan_in=2)
    for r in (1, 3, full["merge_passes"], full["merge_passes"] + 5):
        p = hs.plan(N.HS_INT32, 1 << 24, fan_in=2, stop_after=2 + r, merge=1)
        # the passes up to r (one scheduler launch), then one copy-back kernel
        assert p["launches"] == hs.plan(N.HS_INT32, 1 << 24, fan_in=2, merge=1)["launches"] + 1
        q = hs.plan(N.HS_INT32, 1 << 24, fan_in=2, stop_after=2 + r, merge=2)
        assert q["launches"] == full["launches"] - 2 * full["merge_passes"] + 2 * min(r, full["merge_passes"]) + 1
    lib = N.lib()
    assert lib.hs_sort_keys(0, ctypes.c_void_p(0x1000), 10, ctypes.byref(N.make_opts(stop_after=67)), None) == \
        N.HS_ERR_INVALID


def test_workspace_size_grows_with_n():
    import paper_2003_01216_gb300 as hs
    a = hs.workspace_size(N.HS_INT32, 1 << 20)
    b = hs.workspace_size(N.HS_INT32, 1 << 21)
    assert b > a >= 4 << 20
    assert hs.workspace_size(N.HS_UINT64, 1 << 20, has_vals=True) >= 12 << 20


def test_tuning_table_and_default_rule():
    import ctypes

    import paper_2003_01216_gb300 as hs
    from paper_2003_01216_gb300 import tune
    lib = N.lib()
    tune.clear()
    try:
        # built-in rule: four-way passes up to 2^21 keys, two-way above
        assert tune.get(N.HS_INT32, 1 << 21) == 4 and tune.get(N.HS_INT32, (1 << 21) + 1) == 2
        assert hs.plan(N.HS_INT32, 1 << 20)["fan_in"] == 4 and hs.plan(N.HS_INT32, 1 << 28)["fan_in"] == 2
        # a table entry overrides the rule for its bucket only (bucket = ceil(log2 n))
        tune.set_entry(N.HS_INT32, False, 10, 28, 4)
        assert tune.get(N.HS_INT32, 1 << 28) == 4 and hs.plan(N.HS_INT32, 1 << 28)["fan_in"] == 4
        assert tune.get(N.HS_INT32, (1 << 27) + 1) == 4 and tune.get(N.HS_INT32, (1 << 28) + 1) == 2
        assert tune.get(N.HS_INT32, 1 << 28, has_vals=True) == 2 and tune.get(N.HS_UINT64, 1 << 28) == 2
        assert tune.get(N.HS_INT32, 1 << 28, partition=256) == 2
        # an explicit fan-in is never overridden
        assert hs.plan(N.HS_INT32, 1 << 28, fan_in=2)["fan_in"] == 2
        # invalid entries
        assert lib.hs_tune_set(N.HS_INT32, 0, 10, 20, 3) == N.HS_ERR_INVALID
        assert lib.hs_tune_set(N.HS_INT32, 0, 7, 20, 2) == N.HS_ERR_INVALID
        assert lib.hs_tune_set(N.HS_INT32, 0, 10, 33, 2) == N.HS_ERR_INVALID
        assert lib.hs_tune_set(5, 0, 10, 20, 2) == N.HS_ERR_INVALID
        assert lib.hs_tune_get(N.HS_INT32, 0, 10, 5, None) == N.HS_ERR_INVALID
        out = ctypes.c_int()
        assert lib.hs_tune_get(N.HS_INT32, 0, 0, 1 << 20, ctypes.byref(out)) == N.HS_OK and out.value == 4
        tune.clear()
        assert tune.get(N.HS_INT32, 1 << 28) == 2
    finally:
        tune.clear()


def test_tuning_cache_roundtrip(tmp_path):
    from paper_2003_01216_gb300 import tune
    tune.clear()
    try:
        entries = [{"dtype": "uint64", "has_vals": True, "partition": 10, "log2n": 20, "fan_in": 2,
                    "ms": {"2": 1.0, "4": 1.5}},
                   {"dtype": "int32", "has_vals": False, "partition": 256, "log2n": 30, "fan_in": 4,
                    "ms": {"2": 9.0, "4": 8.0}}]
        path = str(tmp_path / "tune.json")
        tune.save(path, entries, device="GPU A")
        assert tune.load(path, device="GPU B") == 0            # measured on another GPU: skipped
        assert tune.get(N.HS_UINT64, 1 << 20, has_vals=True) == 4  # rule still in force
        assert tune.load(path, device="GPU A") == 2
        assert tune.get(N.HS_UINT64, 1 << 20, has_vals=True) == 2
        assert tune.get(N.HS_INT32, 1 << 30, partition=256) == 4
        assert tune.size_bucket(1) == 0 and tune.size_bucket(1 << 20) == 20 and tune.size_bucket((1 << 20) + 1) == 21
    finally:
        tune.clear()


def test_tile_shapes_and_tuning_table():
    import paper_2003_01216_gb300 as hs
    assert hs.tiles(N.HS_INT32) == [3840, 5888, 7936]
    assert hs.tiles(N.HS_UINT64) == [2816, 3840] == hs.tiles(N.HS_INT32, True)
    # a call's plan follows the tile asked for; the default is the largest 4-byte tile
    for tile in hs.tiles(N.HS_INT32):
        p = hs.plan(N.HS_INT32, 1 << 22, tile=tile, fan_in=2)
        assert p["tile"] == tile
        assert p["merge_passes"] == int(-(-(1 << 22) // tile) - 1).bit_length()
    with pytest.raises(hs.HsError):
        hs.plan(N.HS_UINT64, 1 << 20, tile=7936)
    lib = N.lib()
    fan, tile, merge = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    shape = (ctypes.byref(fan), ctypes.byref(tile), ctypes.byref(merge))
    lib.hs_tune_clear()
    try:
        assert lib.hs_tune_get_shape(0, 0, 10, 1 << 20, *shape) == N.HS_OK
        assert (fan.value, tile.value, merge.value) == (4, 7936, 2)  # the built-in rule
        assert lib.hs_tune_get_shape(0, 0, 10, 1 << 28, *shape) == N.HS_OK
        assert (fan.value, tile.value, merge.value) == (2, 7936, 1)
        assert lib.hs_tune_set_shape(0, 0, 10, 20, 2, 3840, 1) == N.HS_OK
        assert lib.hs_tune_get_shape(0, 0, 10, 1 << 20, *shape) == N.HS_OK
        assert (fan.value, tile.value, merge.value) == (2, 3840, 1)
        assert hs.plan(N.HS_INT32, 1 << 20)["tile"] == 3840  # tile = 0 takes the table's
        assert hs.plan(N.HS_INT32, 1 << 21)["tile"] == 7936  # another size bucket
        # the fan-in alone keeps the tuned tile
        assert lib.hs_tune_set(0, 0, 10, 20, 4) == N.HS_OK
        assert lib.hs_tune_get_shape(0, 0, 10, 1 << 20, *shape) == N.HS_OK
        assert (fan.value, tile.value, merge.value) == (4, 3840, 1)
        # shapes not built for the key type are refused
        assert lib.hs_tune_set_shape(2, 0, 10, 20, 2, 7936, 0) == N.HS_ERR_INVALID
        assert lib.hs_tune_set_shape(0, 0, 10, 20, 3, 3840, 0) == N.HS_ERR_INVALID
        assert lib.hs_tune_set_shape(0, 0, 10, 20, 2, 3840, 3) == N.HS_ERR_INVALID
        with pytest.raises(hs.HsError):
            hs.plan(N.HS_INT32, 1 << 20, merge=5)
    finally:
        lib.hs_tune_clear()
