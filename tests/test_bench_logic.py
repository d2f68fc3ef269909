"""The benchmark's host-side logic on the CPU: the byte model of the merge
passes, the clock samples it keeps, and the traffic record it scales."""
import datetime
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_merge_active_keys_two_way():
    # packets of 3 tiles, empty, 2 tiles (one key over), 1 short tile:
    # passes ceil(log2(tiles)) = 2, 0, 1, 0
    t = 7936
    lens = [3 * t, 0, t + 1, 5]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    assert bench.merge_active_keys(off, t, 2) == [3 * t + t + 1, 3 * t]


def test_merge_active_keys_four_way():
    # ceil(log4(tiles)): 17 tiles -> 3 passes, 4 tiles -> 1, 5 tiles -> 2, 1 tile -> 0
    t = 3840
    lens = [17 * t, 4 * t, 4 * t + 1, t]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    assert bench.merge_active_keys(off, t, 4) == [17 * t + 4 * t + 4 * t + 1, 17 * t + 4 * t + 1, 17 * t]


def test_merge_active_keys_nothing_to_merge():
    off = np.array([0, 10, 10, 20], dtype=np.uint64)
    assert bench.merge_active_keys(off, 7936, 2) == []


def _write_samples(path, t0, rows):
    with open(path, "w") as f:
        for dt, mhz, cap in rows:
            ts = datetime.datetime.fromtimestamp(t0 + dt).strftime("%Y/%m/%d %H:%M:%S.%f")
            f.write(f"{ts}, 0, {mhz}, 2070, 610.5, 0x0, Not Active, Not Active, Not Active, "
                    f"{'Active' if cap else 'Not Active'}\n")


def test_clock_summary_keeps_samples_inside_the_region():
    c = bench.ClockSampler(0)
    c.proc = object()  # a sampler that "ran"
    t0 = time.time()
    # samples 0.1 s before, inside, and after the region [t0, t0 + 0.1]
    _write_samples(c.path, t0, [(-0.1, 900, False), (0.02, 2070, False), (0.06, 2040, True), (0.5, 1000, False)])
    try:
        c.t0, c.t1 = t0, t0 + 0.1
        s = c.summary()
        assert s["samples"] == 2 and s["samples_where"] == "inside the timed region"
        assert s["sm_mhz"] == (2070 + 2040) / 2 and s["reasons"] == ["sw_power_cap"]
        # a region between samples: the two nearest are kept and said to be so
        c.t0, c.t1 = t0 + 0.2, t0 + 0.21
        s = c.summary()
        assert s["samples"] == 2 and s["samples_where"].startswith("nearest")
    finally:
        os.remove(c.path)


def test_clock_summary_without_nvidia_smi():
    c = bench.ClockSampler(0)
    assert c.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_traffic_record_scales_and_expires():
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        rec = json.load(f)["merge"]
    got = bench.ncu_traffic("merge", 1000.0)
    if rec["source_sha"] == bench.source_sha(*rec["sources"]):
        assert got == rec["dram_bytes_per_key"] * 1000.0
    else:  # sources changed since the capture: no traffic figure
        assert got is None
    assert bench.ncu_traffic("no_such_kernel", 1000.0) is None


def test_per_kernel_roofline_fractions():
    # 2^28 int32 keys: hist reads 1 GiB, scatter and tile sort move 2 GiB each,
    # 14 merge passes over 2^28 active keys move 28 GiB; two steps were timed
    n = 1 << 28
    per_kernel = {"hist": (2, 0.8), "scatter": (2, 1.0), "tilesort": (2, 4.0), "merge": (28, 9.0),
                  "corank": (28, 0.9)}
    r = bench.per_kernel_roofline(per_kernel, 2, 4 * n, 4 * n, 14 * n, 4, "merge", 6800.0)
    assert set(r) == {"hist", "scatter", "tilesort", "merge"}
    assert r["hist"]["bytes_per_step"] == 4 * n
    assert abs(r["hist"]["achieved_gbs"] - 4 * n / 0.4e-3 / 1e9) < 1e-6
    assert abs(r["merge"]["frac"] - (2 * 4 * 14 * n / 4.5e-3 / 1e9) / 6800.0) < 1e-9
    assert abs(r["scatter"]["frac_vs_nominal"] - (8 * n / 0.5e-3 / 1e9) / bench.NOMINAL_HBM_GBS) < 1e-9
    assert r["merge"]["launches_per_step"] == 14
    # a kernel that was not timed is left out
    assert "tilesort" not in bench.per_kernel_roofline({"merge": (1, 1.0)}, 1, 1, 1, 1, 4, "merge", 1.0)


def test_merge_pass_roofline():
    # three passes with active keys; launches in launch order, other kernels mixed in,
    # and one extra enqueued pass that does no work
    n = 1 << 20
    active = [n, n, n // 2]
    launches = [("hist", 0.1), ("corank", 0.01), ("merge", 0.5), ("corank", 0.01), ("merge", 0.25),
                ("corank", 0.01), ("merge", 0.125), ("corank", 0.0), ("merge", 0.002)]
    r = bench.merge_pass_roofline(launches, "merge", active, 4, 6800.0)
    assert [p["pass"] for p in r["passes"]] == [1, 2, 3]
    assert abs(r["passes"][0]["achieved_gbs"] - round(2 * 4 * n / 0.5e-3 / 1e9, 1)) < 1e-9
    assert abs(r["passes"][2]["achieved_gbs"] - round(2 * 4 * (n // 2) / 0.125e-3 / 1e9, 1)) < 1e-9
    assert abs(r["search_ms"] - 0.03) < 1e-9
    # a missing launch ends the list
    assert bench.merge_pass_roofline(launches[:3], "merge", active, 4, 6800.0)["passes"][-1]["pass"] == 1
