"""GPU: a seeded sweep of call shapes against the oracle.

Every case draws (key type, distribution, size, partition, merge fan-in, merge
launch style, tile, values or not, device or host buffers) from a fixed seed;
sizes are drawn near the edges the kernels care about (multiples of the
packet-step block of 3840 keys and of the tile, plus or minus a few keys, and
powers of two).  Each result is compared element by element with the
oracle's sort (keys, and the stable order of the values).

HS_SWEEP_CASES / HS_SWEEP_FIRST (environment) widen the sweep: that many
cases from that case index on (default 40 from 0)."""
import os

import numpy as np
import pytest
import torch

import paper_2003_01216_gb300 as hs
from gpu_util import assert_equal, run
from paper_2003_01216_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DISTS = {0: ["uniform1e9", "uniform31", "zipf", "sorted", "reverse", "equal", "distinct16", "int32full",
             "three_digit"],
         1: ["uniform32"],
         2: ["uniform64", "distinct2p24"]}
N_CASES = int(os.environ.get("HS_SWEEP_CASES", "40"))
FIRST = int(os.environ.get("HS_SWEEP_FIRST", "0"))


def _case(i):
    rng = np.random.default_rng(20261204 + i)
    code = int(rng.choice([0, 0, 0, 1, 2]))
    dist = str(rng.choice(DISTS[code]))
    with_vals = bool(rng.random() < 0.3)
    tiles = hs.tiles(code, with_vals)
    tile = int(rng.choice([0] + tiles))
    unit = int(rng.choice([3840, tile or tiles[-1], 1 << int(rng.integers(10, 21))]))
    n = max(0, unit * int(rng.integers(1, 400)) + int(rng.integers(-3, 4)))
    n = min(n, 3_000_000)
    nb = int(rng.choice([10, 10, 256, 1]))
    fan = int(rng.choice([0, 2, 4]))
    merge = int(rng.choice([0, 1, 2])) if fan != 4 else 0
    host = bool(rng.random() < 0.2) and not with_vals
    return code, dist, n, nb, fan, merge, tile, with_vals, host


CASES = [_case(i) for i in range(FIRST, FIRST + N_CASES)]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[1]}-{c[2]}-nb{c[3]}-f{c[4]}m{c[5]}t{c[6]}{'-v' if c[7] else ''}"
                                             f"{'-host' if c[8] else ''}" for c in CASES])
def test_random_shapes_vs_oracle(oracle, case):
    code, dist, n, nb, fan, merge, tile, with_vals, host = case
    keys = I.generate(dist, n, seed=n % 9973)
    vals = I.index_values(n) if with_vals else None
    ek, ev, eoff = oracle.sort(keys, vals, nbuckets=nb)
    if host:
        pinned = torch.from_numpy(keys.copy()).pin_memory()
        hs.sort_keys_host(pinned, partition=nb, fan_in=fan, merge=merge, tile=tile)
        assert hs.stream_error() == 0
        assert_equal(pinned.numpy(), ek, "host-buffer sort")
        return
    gk, gv, goff, st = run(keys, vals, nb=nb, fan_in=fan, merge=merge, tile=tile)
    assert st == 0
    assert_equal(goff, eoff, "packet offsets")
    assert_equal(gk, ek, "sorted keys")
    if with_vals:
        assert_equal(gv, ev, "values in stable order")
