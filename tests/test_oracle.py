"""Pins for the CPU oracle (no GPU).  The oracle is checked against things
other than itself: hand-worked fixtures (tests/golden), closed forms, a
literal decimal-string restatement of the packet rule, brute force over every
short sequence against Python's sorted(), invariants, and the independence of
the result from the thread count T and the per-part sort of Sec. 3.2."""
import itertools

import numpy as np
import pytest

import golden_io as G
from paper_2003_01216_gb300 import inputs as I

DTYPES = [np.int32, np.uint32, np.uint64]


# --------------------------------------------------------------------------
# hand-worked fixtures
# --------------------------------------------------------------------------
@pytest.mark.parametrize("fx", G.all_fixtures(), ids=lambda f: f["name"])
def test_golden_fixture(oracle, fx):
    keys, nb = fx["keys"], fx["nbuckets"]
    vals = fx.get("vals")
    w, flip = oracle.digit_info(keys, nb)
    assert (w, flip) == (fx["width"], fx["flip"])
    lay, lv, off = oracle.partition(keys, vals, nb)
    np.testing.assert_array_equal(off, fx["offsets"])
    np.testing.assert_array_equal(lay, fx["layout"])
    if vals is not None:
        np.testing.assert_array_equal(lv, fx["layout_vals"])
    for T in (1, 2, 4):
        for cs in (0, 1):
            sk, sv, soff = oracle.sort(keys, vals, nb, T=T, chunk_sort=cs)
            np.testing.assert_array_equal(sk, fx["sorted"])
            np.testing.assert_array_equal(soff, fx["offsets"])
            if vals is not None:
                np.testing.assert_array_equal(sv, fx["sorted_vals"])


def test_fixture_count():
    assert len(G.all_fixtures()) >= 9


# --------------------------------------------------------------------------
# brute force: every sequence of length <= 5 over small alphabets (this covers
# every permutation of every multiset drawn from them)
# --------------------------------------------------------------------------
ALPHABETS = {
    np.int32: [[0, 9, 10, 99], [-5, 0, 7, 100], [-2147483648, -1, 2147483647, 5], [3, 3, 30, 300]],
    np.uint32: [[0, 9, 10, 4294967295], [1, 2, 1000000000, 999999999]],
    np.uint64: [[0, 10, 18446744073709551615, 10000000000000000000], [5, 9999999999999999999, 7, 70]],
}


@pytest.mark.parametrize("dt", DTYPES, ids=lambda d: np.dtype(d).name)
@pytest.mark.parametrize("nb", [10, 256])
def test_bruteforce_short_sequences(oracle, dt, nb):
    for alpha in ALPHABETS[dt]:
        alpha = list(dict.fromkeys(alpha))
        for n in range(0, 6):
            for seq in itertools.product(alpha, repeat=n):
                keys = np.array(seq, dtype=object).astype(dt) if n else np.zeros(0, dt)
                vals = np.arange(n, dtype=np.uint32) * 7 + 3
                T = [1, 2, 4][n % 3]
                sk, _, off = oracle.sort(keys, None, nb, T=T, chunk_sort=n % 2)
                assert [int(x) for x in sk] == sorted(int(x) for x in keys)
                pk, pv, _ = oracle.sort(keys, vals, nb, T=T, chunk_sort=(n + 1) % 2)
                ek, ev = G.stable_sorted_literal(keys, vals)
                np.testing.assert_array_equal(pk, ek)
                np.testing.assert_array_equal(pv, ev)
                lay, lv, poff = oracle.partition(keys, vals, nb)
                el, elv, eoff = G.stable_layout_literal(keys, nb, vals)
                np.testing.assert_array_equal(lay, el)
                np.testing.assert_array_equal(lv, elv)
                np.testing.assert_array_equal(poff, eoff)
                np.testing.assert_array_equal(off, eoff)


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 9, 10, 11, 100, 1000, 1234, 99999, 100000, 654321])
def test_closed_form_identity_keys_decimal(oracle, n):
    # key_i = i: the largest key n-1 has D digits, P = 10^(D-1), and packet p
    # holds the keys p*P .. min(n, (p+1)*P) - 1.
    keys = np.arange(n, dtype=np.uint32)
    D = len(str(n - 1))
    P = 10 ** (D - 1)
    counts = [min(max(n - p * P, 0), P) for p in range(10)]
    _, _, off = oracle.partition(keys, None, 10)
    assert list(np.diff(off.astype(np.int64))) == counts
    assert oracle.digit_info(keys, 10) == (D, False)
    sk, _, _ = oracle.sort(keys[::-1].copy(), None, 10)
    np.testing.assert_array_equal(sk, keys)


@pytest.mark.parametrize("k", [0, 3, 8, 9, 12, 17])
def test_closed_form_identity_keys_256(oracle, k):
    # key_i = i for n = 2^k: the largest key has bit length k; bucket = i >> (k-8)
    # puts 2^(k-8) keys in each of 256 buckets (k >= 8), else one key per bucket.
    n = 1 << k
    keys = np.arange(n, dtype=np.uint32)
    _, _, off = oracle.partition(keys, None, 256)
    c = np.diff(off.astype(np.int64))
    if k >= 8:
        assert (c == (1 << (k - 8))).all()
    else:
        assert list(c[:n]) == [1] * n and c[n:].sum() == 0
    assert oracle.digit_info(keys, 256)[0] == (n - 1).bit_length()


def test_uniform_packet_fractions(oracle):
    # uniform [0, 10^9): D = 9 and each packet holds 10% of the keys; with
    # n = 10^6 every count lies within 5 binomial sigmas (sigma = 300).
    n = 1_000_000
    keys = I.generate("uniform1e9", n)
    _, _, off = oracle.partition(keys, None, 10)
    c = np.diff(off.astype(np.int64))
    assert np.all(np.abs(c - n // 10) < 5 * 300)
    assert oracle.digit_info(keys, 10) == (9, False)
    # uniform [0, 2^31): D = 10, packets 0 and 1 hold 10^9/2^31 each, packet 2
    # the rest (2^31 - 2*10^9)/2^31, packets 3..9 nothing.
    keys = I.generate("uniform31", n)
    _, _, off = oracle.partition(keys, None, 10)
    c = np.diff(off.astype(np.int64)) / n
    exp = [1e9 / 2**31, 1e9 / 2**31, (2**31 - 2e9) / 2**31] + [0.0] * 7
    assert np.all(np.abs(c - exp) < 5 * np.sqrt(0.25 / n))
    # uniform 64-bit: D = 20, packet 0 holds 10^19 / 2^64 of the keys.
    keys = I.generate("uniform64", n)
    _, _, off = oracle.partition(keys, None, 10)
    assert abs(int(off[1]) / n - 1e19 / 2**64) < 5 * np.sqrt(0.25 / n)
    assert int(off[2]) == n


# --------------------------------------------------------------------------
# invariants on random inputs
# --------------------------------------------------------------------------
def check_invariants(keys, sk, nb, off):
    n = keys.size
    assert sk.size == n and sk.dtype == keys.dtype
    if n:
        assert np.all(sk[1:] >= sk[:-1])                      # non-decreasing
    v1, c1 = np.unique(keys, return_counts=True)
    v2, c2 = np.unique(sk, return_counts=True)
    np.testing.assert_array_equal(v1, v2)                     # same multiset
    np.testing.assert_array_equal(c1, c2)
    assert int(off[-1]) == n and np.all(np.diff(off.astype(np.int64)) >= 0)
    # packets do not overlap: every key of packet p is below every key of p+1,
    # and carries digit p
    packets = np.array(G.packets_literal(sk, nb), dtype=np.int64)
    for p in range(nb):
        seg = packets[int(off[p]):int(off[p + 1])]
        assert np.all(seg == p)


@pytest.mark.parametrize("dist", ["uniform31", "zipf", "sorted", "reverse", "equal", "distinct16",
                                  "uniform1e9", "int32full", "three_digit", "uniform32", "uniform64",
                                  "distinct2p24"])
@pytest.mark.parametrize("nb", [10, 256])
def test_invariants_random(oracle, dist, nb):
    n = 60_000 if nb == 10 else 30_000
    keys = I.generate(dist, n, seed=3)
    sk, _, off = oracle.sort(keys, None, nb)
    check_invariants(keys, sk, nb, off)
    vals = I.index_values(n)
    pk, pv, _ = oracle.sort(keys, vals, nb)
    np.testing.assert_array_equal(pk, sk)
    assert np.array_equal(np.sort(pv), vals)                  # values are a permutation
    same = pk[1:] == pk[:-1]
    assert np.all(pv[1:][same] > pv[:-1][same])               # input order kept on ties
    np.testing.assert_array_equal(pk, np.sort(keys, kind="stable"))
    np.testing.assert_array_equal(pv, np.argsort(keys, kind="stable").astype(np.uint32))


def test_partition_matches_literal_on_random(oracle):
    for dist in ["uniform1e9", "int32full", "uniform64", "zipf", "three_digit"]:
        keys = I.generate(dist, 5000, seed=11)
        vals = I.index_values(5000)
        for nb in (10, 256):
            lay, lv, off = oracle.partition(keys, vals, nb)
            el, elv, eoff = G.stable_layout_literal(keys, nb, vals)
            np.testing.assert_array_equal(lay, el)
            np.testing.assert_array_equal(lv, elv)
            np.testing.assert_array_equal(off, eoff)


@pytest.mark.parametrize("dist", ["uniform31", "zipf", "distinct16", "uniform64"])
def test_thread_count_independence(oracle, dist):
    keys = I.generate(dist, 50_001, seed=5)
    vals = I.index_values(keys.size)
    ref = None
    for T in (1, 2, 4, 16, 64):
        for cs in (0, 1):
            sk, sv, _ = oracle.sort(keys, vals, 10, T=T, chunk_sort=cs)
            if ref is None:
                ref = (sk, sv)
            np.testing.assert_array_equal(sk, ref[0])
            np.testing.assert_array_equal(sv, ref[1])


@pytest.mark.parametrize("dt", DTYPES, ids=lambda d: np.dtype(d).name)
def test_special_inputs(oracle, dt):
    info = np.iinfo(dt)
    cases = [
        np.zeros(0, dt), np.array([5], dt), np.full(1000, 42, dt),
        np.arange(3000, dtype=dt), np.arange(3000, dtype=dt)[::-1].copy(),
        np.array([info.max, info.min, 0, info.max, 9, 10, 99], dt),
        np.array([info.max] * 5 + [info.min] * 5, dt),
    ]
    for keys in cases:
        for nb in (10, 256):
            sk, _, off = oracle.sort(keys, None, nb)
            np.testing.assert_array_equal(sk, np.sort(keys))
            check_invariants(keys, sk, nb, off)
    # maximum digit width: D = 10 for 32-bit images, 20 for 64-bit
    top = np.array([info.max], dt)
    assert oracle.digit_info(top, 10)[0] == (20 if dt == np.uint64 else 10)


def test_batch_segments(oracle):
    off = I.batch_offsets(40, 1, 3000, seed=2)
    n = int(off[-1])
    keys = I.generate("uniform31", n, seed=2)
    vals = I.index_values(n)
    bk, bv = oracle.sort_batch(keys, off, vals)
    for s in range(off.size - 1):
        lo, hi = int(off[s]), int(off[s + 1])
        ek, ev = oracle.sort(keys[lo:hi], vals[lo:hi])[:2]
        np.testing.assert_array_equal(bk[lo:hi], ek)
        np.testing.assert_array_equal(bv[lo:hi], ev)
        np.testing.assert_array_equal(bk[lo:hi], np.sort(keys[lo:hi]))


def test_tile_sort_intermediate(oracle):
    keys = I.generate("uniform1e9", 10_000, seed=4)
    lay, _, off = oracle.partition(keys, None, 10)
    ts, _ = oracle.tile_sort(lay, off, 512)
    for p in range(10):
        for lo in range(int(off[p]), int(off[p + 1]), 512):
            hi = min(lo + 512, int(off[p + 1]))
            np.testing.assert_array_equal(ts[lo:hi], np.sort(lay[lo:hi]))


TILE_PAIR_CASES = [
    # (distribution, n, reduce keys modulo, tile): ties-heavy keys, tiles that
    # do not divide the packets (a ragged last tile in every packet)
    ("distinct16", 9_001, None, 512),
    ("distinct16", 9_001, None, 3840),
    ("distinct2p24", 7_777, 997, 700),
    ("distinct2p24", 7_777, 5, 64),
    ("uniform1e9", 6_000, 50, 1000),
    ("int32full", 5_003, 7, 333),
]


@pytest.mark.parametrize("dist,n,mod,tile", TILE_PAIR_CASES)
def test_tile_sort_pairs_is_stable_per_tile(oracle, dist, n, mod, tile):
    # The key-value tile sort (Sec. 3.2 with the stable reading for pairs):
    # every tile of every packet, on its own, in the order of a stable sort by
    # key, equal keys in their packet-layout order.  numpy's stable argsort of
    # each tile is the independent statement of that order.
    keys = I.generate(dist, n, seed=11)
    if mod is not None:
        keys = keys % keys.dtype.type(mod)
    vals = I.index_values(n)
    lay, lv, off = oracle.partition(keys, vals, 10)
    tk, tv = oracle.tile_sort(lay, off, tile, lv)
    ntiles = 0
    for p in range(off.size - 1):
        for lo in range(int(off[p]), int(off[p + 1]), tile):
            hi = min(lo + tile, int(off[p + 1]))
            order = np.argsort(lay[lo:hi], kind="stable")
            np.testing.assert_array_equal(tk[lo:hi], lay[lo:hi][order])
            np.testing.assert_array_equal(tv[lo:hi], lv[lo:hi][order])
            ntiles += 1
    nonempty = int(np.count_nonzero(np.diff(off.astype(np.int64))))
    assert ntiles > nonempty  # some packet has several tiles and a ragged last one
    # ties are really present inside tiles (the case stability decides)
    assert np.unique(lay).size < n // 2


@pytest.mark.parametrize("dist", ["uniform31", "int32full", "uniform64", "distinct16"])
def test_one_packet_is_the_plain_hybrid(oracle, dist):
    # nbuckets = 1: no MSD step, the whole array is one packet (Sec. 3.2 alone);
    # the sorted result is the same as with the MSD step
    keys = I.generate(dist, 20_000, seed=8)
    vals = I.index_values(keys.size)
    lay, lv, off = oracle.partition(keys, vals, 1)
    np.testing.assert_array_equal(lay, keys)
    np.testing.assert_array_equal(lv, vals)
    assert list(off) == [0, keys.size]
    k1, v1, _ = oracle.sort(keys, vals, 1)
    k10, v10, _ = oracle.sort(keys, vals, 10)
    np.testing.assert_array_equal(k1, k10)
    np.testing.assert_array_equal(v1, v10)


def test_invalid_arguments(oracle):
    keys = np.arange(10, dtype=np.int32)
    with pytest.raises(ValueError):
        oracle.sort(keys, None, 7)          # neither 1, 10 nor 256 packets
    with pytest.raises(ValueError):
        oracle.sort(keys, None, 10, T=3)    # T must be a power of two (Sec. 3.2)


# --------------------------------------------------------------------------
# the input generator: published SplitMix64 outputs for seed 0
# --------------------------------------------------------------------------
def test_splitmix64_published_vector():
    z = I.mix64(np.array([0x9E3779B97F4A7C15, (2 * 0x9E3779B97F4A7C15) % 2**64], dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF
    assert int(z[1]) == 0x6E789E6AA1B965F4


def test_generators_shapes():
    assert I.generate("sorted", 1 << 20)[-1] == ((1 << 20) - 1) * 2048
    assert I.generate("reverse", 8)[0] == (7 << 31) // 8
    z = I.generate("zipf", 200_000)
    top = np.bincount(np.unique(z, return_inverse=True)[1]).max() / z.size
    assert 0.10 < top < 0.15          # Zipf s=1.1 over 2^20: the top value holds ~12.4%
    d = I.generate("distinct16", 10_000)
    assert np.unique(d).size == 16
    off = I.batch_offsets(10_000, 16, 1 << 20)
    lens = np.diff(off.astype(np.int64))
    assert lens.min() >= 16 and lens.max() <= 1 << 20
