"""Plant plausible mistakes in copies of the oracle (on the CPU only) and check
that the pins catch every one of them: a dropped term, a wrong sign or index,
a lost tie-break.  Each mutant is a one-line textual edit of the source.

(Swapping the two lists of a merge, or sending merge ties to the right list,
are equivalent mutants here and are not listed: pair records compare by
(key, input index), which is unique, so neither changes any result.)"""
import os
import subprocess
import sys

import numpy as np
import pytest

import golden_io as G
import oracle as orc
import test_oracle as T
from paper_2003_01216_gb300 import inputs as I

MUTANTS = {
    # the input-index tie-break dropped from the pair order: stability lost
    "no_index_tiebreak": ("return a.idx < b.idx;", "return false;"),
    # merge forgets the rest of the right list
    "merge_drops_tail": ("while (j < nb) out[o++] = b[j++];", ";"),
    # divisor 10^D instead of 10^(D-1): every key lands in packet 0
    "divisor_off_by_one": ("d.divisor = pow10u(d.width - 1);", "d.divisor = pow10u(d.width);"),
    # negative int32 keys not mapped to an order-preserving image
    "no_sign_flip": ("if (is_negative(keys[i])) d.flip = true;", ";"),
    # three-way partition skips the element swapped in from the right
    "quicksort_skip": ("std::swap(s[i], s[g]);", "std::swap(s[i], s[g]); ++i;"),
    # last part loses the remainder when T does not divide the packet
    "tree_drops_remainder": ("b[T] = len;", "b[T] = T * part;"),
    # 256-bucket shift off by one
    "shift_off_by_one": ("d.shift = d.width > 8 ? d.width - 8 : 0;", "d.shift = d.width > 7 ? d.width - 7 : 0;"),
    # scatter visits the input backwards: packet layout no longer stable
    "scatter_reversed": ("out[next[p]++] = in[i];", "out[next[p]++] = in[n - 1 - i]; (void)i;"),
    # digit count off by one
    "digits_off_by_one": ("while (v >= 10) {", "while (v > 10) {"),
    # tree merge reads the neighbour's list from the wrong part
    "tree_wrong_neighbour": ("uint64_t lo = b[m], mid = b[m + w],", "uint64_t lo = b[m], mid = b[m + w / 2 + (w == 1)],"),
    # key-value tile sort loses its tile-local index tie-break: equal keys of a
    # tile no longer keep their packet-layout order
    "tile_sort_no_tiebreak": ("r[i - lo] = Rec<K>{keys[i], vals[i], static_cast<uint32_t>(i - lo)};",
                              "r[i - lo] = Rec<K>{keys[i], vals[i], 0u};"),
}


def battery(o) -> list[str]:
    """Run the pins against oracle ``o``; return the names of those that fail."""
    failed = []

    def run(name, fn, *args):
        try:
            fn(o, *args)
        except (AssertionError, ValueError):
            failed.append(name)

    for fx in G.all_fixtures():
        run("golden:" + fx["name"], T.test_golden_fixture, fx)
    for dt in T.DTYPES:
        run("brute", T.test_bruteforce_short_sequences, dt, 10)
    run("closed_form", T.test_closed_form_identity_keys_decimal, 1234)
    run("closed_form_256", T.test_closed_form_identity_keys_256, 12)
    for dist in ("uniform31", "int32full", "uniform64"):
        run("invariants:" + dist, T.test_invariants_random, dist, 10)
    run("thread_count", T.test_thread_count_independence, "distinct16")
    for case in T.TILE_PAIR_CASES:
        run("tile_sort_pairs", T.test_tile_sort_pairs_is_stable_per_tile, *case)
    return failed


@pytest.fixture(scope="module")
def source():
    with open(orc.SRC) as f:
        return f.read()


def test_unmutated_battery_passes(oracle):
    assert battery(oracle) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, source, name):
    old, new = MUTANTS[name]
    assert source.count(old) == 1, f"mutation site for {name} not unique"
    src = tmp_path / f"{name}.cpp"
    src.write_text(source.replace(old, new))
    lib = str(tmp_path / f"lib{name}.so")
    orc.build(str(src), lib)
    # A mutant may crash (an out-of-range packet index); run it in a child so a
    # crash counts as caught instead of taking the test session down.
    here = os.path.dirname(os.path.abspath(__file__))
    code = ("import sys; sys.path[:0] = [%r, %r]; import oracle, test_oracle_mutants as M; "
            "f = M.battery(oracle.Oracle(%r)); print(f); sys.exit(1 if f else 0)"
            % (here, os.path.dirname(here), lib))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived every pin"
