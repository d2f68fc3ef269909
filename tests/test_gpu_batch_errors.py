"""GPU: segmented sort against the oracle segment by segment, and the
device-detected error paths (malformed batch offsets; a bounded wait that is
made to expire).  Failures are made on the host side or by a flag that nothing
sets; no test faults or hangs the GPU."""
import numpy as np
import pytest
import torch

import paper_2003_01216_gb300 as hs
from gpu_util import HS_INVALID, HS_TIMEOUT, assert_equal, dev, run, to_dev
from paper_2003_01216_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# merge shapes: two-way passes in one persistent launch (merge = 1), two-way
# passes with a launch each (merge = 2), four-way passes
SHAPES = [(2, 1), (2, 2), (4, 0)]
SHAPE_IDS = ["fan2-queue", "fan2-per-pass", "fan4"]


def make_batch(count, lo, hi, seed, empties=True):
    lens = I.log_uniform_lengths(count, lo, hi, seed=seed)
    if empties:
        lens[::7] = 0
    off = np.zeros(count + 1, dtype=np.uint64)
    off[1:] = np.cumsum(lens)
    return off


@pytest.mark.parametrize("fan,merge", SHAPES, ids=SHAPE_IDS)
@pytest.mark.parametrize("nb", [1, 10, 256])
@pytest.mark.parametrize("dist", ["uniform31", "zipf", "int32full", "uniform32", "uniform64", "distinct2p24"])
def test_sort_batch(oracle, dist, nb, fan, merge):
    off = make_batch(300, 1, 20_000, seed=5)
    n = int(off[-1])
    keys = I.generate(dist, n, seed=6)
    vals = I.index_values(n)
    ek, ev = oracle.sort_batch(keys, off, vals, nbuckets=nb)
    tk, tv, to = to_dev(keys), to_dev(vals), to_dev(off)
    poff = torch.zeros(300 * nb + 1, dtype=torch.uint64, device=dev())
    hs.sort_batch(tk, to, tv, partition=nb, packet_offsets=poff, fan_in=fan, merge=merge)
    assert hs.stream_error() == 0
    assert_equal(tk.cpu().numpy(), ek, f"batch keys {dist}")
    assert_equal(tv.cpu().numpy(), ev, f"batch values {dist}")
    tk = to_dev(keys)
    hs.sort_batch(tk, to, None, partition=nb, fan_in=fan, merge=merge)
    assert hs.stream_error() == 0
    assert_equal(tk.cpu().numpy(), ek, f"batch keys only {dist}")
    # packet offsets of every segment equal the oracle's, shifted by the segment start
    po = poff.cpu().numpy()
    for s in range(0, 300, 13):
        lo, hi = int(off[s]), int(off[s + 1])
        _, _, so = oracle.partition(keys[lo:hi], None, nb)
        assert_equal(po[s * nb:(s + 1) * nb + 1], so + np.uint64(lo), f"segment {s} packet offsets")


def test_batch_single_segment_equals_plain(oracle):
    keys = I.generate("uniform31", 100_000, seed=8)
    off = np.array([0, keys.size], dtype=np.uint64)
    tk = to_dev(keys)
    hs.sort_batch(tk, to_dev(off))
    assert hs.stream_error() == 0
    gk, _, _, _ = run(keys)
    assert_equal(tk.cpu().numpy(), gk, "one-segment batch vs plain sort")


def test_batch_bad_offsets_leave_keys_untouched():
    keys = I.generate("uniform31", 10_000, seed=9)
    for bad in ([0, 6000, 5000, 10_000], [0, 5000, 9999], [1, 5000, 10_000]):
        tk = to_dev(keys)
        hs.sort_batch(tk, to_dev(np.array(bad, dtype=np.uint64)))
        assert hs.stream_error() == HS_INVALID
        assert_equal(tk.cpu().numpy(), keys, "keys after rejected offsets")
    assert hs.stream_error() == 0  # the word was cleared


def test_bounded_wait_expires_and_context_survives(oracle):
    # one bulk copy of the tile sort announces bytes that never arrive (debug
    # flag) and the wait limit is 2 ms: the waiting CTA gives up, the call
    # reports HS_ERR_TIMEOUT
    keys = I.generate("uniform31", 5 * 4096, seed=10)
    _, _, _, st = run(keys, debug_flags=1)
    assert st == HS_TIMEOUT
    # the context stays usable and the next call is correct
    gk, _, _, st = run(keys)
    assert st == 0
    assert_equal(gk, oracle.sort(keys)[0], "sort after an expired wait")


def test_scatter_wait_expires_and_context_survives(oracle):
    # the same for the packet step's scatter (two input stages): CTA 0's first
    # block never completes its copy, its bounded wait gives up, and the copy
    # of the next block was never issued, so nothing is left in flight
    # (64-bit keys with values take the one-stage layout)
    for dist, n, with_vals in (("uniform31", 1_000_000, False), ("uniform64", 300_000, False),
                               ("uniform64", 300_000, True)):
        keys = I.generate(dist, n, seed=10)
        vals = I.index_values(n) if with_vals else None
        _, _, _, st = run(keys, vals, debug_flags=4)
        assert st == HS_TIMEOUT
        gk, gv, _, st = run(keys, vals)
        assert st == 0
        ek, ev, _ = oracle.sort(keys, vals)
        assert_equal(gk, ek, "sort after an expired scatter wait")
        if with_vals:
            assert_equal(gv, ev, "values after an expired scatter wait")


def test_caller_workspace(oracle):
    keys = I.generate("zipf", 50_000, seed=11)
    need = hs.workspace_size(0, keys.size)
    ws = torch.empty(need, dtype=torch.uint8, device=dev())
    tk = to_dev(keys)
    hs.sort_keys(tk, workspace=ws)
    assert hs.stream_error() == 0
    assert_equal(tk.cpu().numpy(), oracle.sort(keys)[0], "sort in a caller work space")
    with pytest.raises(hs.HsError):
        hs.sort_keys(tk, workspace=ws[: need // 2])
    big = torch.empty(need + 512, dtype=torch.uint8, device=dev())
    with pytest.raises(hs.HsError):  # the work space must be 256-byte aligned
        hs.sort_keys(tk, workspace=big[16:16 + need])


# (distribution, n, partition): pinned memory is read by the histogram kernel
# itself (several blocks per CTA, a ragged last block; negative int32 keys
# also take the flipped-image pass, which then reads the device copy); with
# partition 1 or n of at most one tile there is no histogram and the sort
# copies the keys in first
# merge = 1 puts the merge passes in the persistent queue launch, whose last
# pass of every packet writes straight back to pinned host memory (and a small
# kernel copies the packets that need no merge pass: uniform [0, 2^31) at 100K
# keys has a third packet of one tile); merge = 2 keeps a launch per pass and
# a copy out after the sort
HOST_CASES = [("uniform1e9", 200_000, 10, 2), ("int32full", 1_500_001, 10, 2), ("uniform64", 777_777, 10, 2),
              ("uniform32", 300_003, 256, 2), ("zipf", 250_000, 1, 2), ("uniform31", 5_000, 10, 0),
              ("uniform64", 1, 10, 0), ("uniform31", 100_000, 10, 1), ("int32full", 1_500_001, 10, 1),
              ("uniform64", 777_777, 10, 1), ("zipf", 2_000_000, 10, 1), ("uniform32", 300_003, 256, 1),
              ("uniform31", 250_000, 1, 1), ("equal", 400_000, 10, 1),
              # ten packets of a few tiles each: many packets whose only merge pass is their last
              # (host tickets only in the merge queue), then packets of two passes
              ("uniform1e9", 158_720, 10, 1), ("uniform1e9", 317_445, 10, 1)]


@pytest.mark.parametrize("dist,n,nb,merge", HOST_CASES, ids=[f"{d}-{n}-{nb}-m{m}" for d, n, nb, m in HOST_CASES])
def test_host_buffers(oracle, dist, n, nb, merge):
    fan = 2 if merge == 1 else 0  # (the tuned rule takes fan-in 4 up to 2^21 keys)
    keys = I.generate(dist, n, seed=12)
    exp = oracle.sort(keys, nbuckets=nb)[0]
    h = keys.copy()  # pageable: copied in and out by cudaMemcpyAsync
    hs.sort_keys_host(h, partition=nb, merge=merge, fan_in=fan)
    assert_equal(h, exp, "host-buffer sort")
    pinned = torch.from_numpy(keys.copy()).pin_memory()  # device-addressable: read (and written) by the sort itself
    for _ in range(2):  # the second call sorts sorted keys, same result
        hs.sort_keys_host(pinned, partition=nb, merge=merge, fan_in=fan)
        assert hs.stream_error() == 0
        assert_equal(pinned.numpy(), exp, "pinned host-buffer sort")
    # which path ran: the histogram that reads host memory or a copy in; the
    # merge queue writing back to host memory or a copy out
    pinned.copy_(torch.from_numpy(keys))
    hs.timing_read()
    hs.timing_enable(True)
    try:
        hs.sort_keys_host(pinned, partition=nb, merge=merge, fan_in=fan)
        names = set(hs.timing_read())
    finally:
        hs.timing_enable(False)
    assert_equal(pinned.numpy(), exp, "pinned host-buffer sort, timed")
    code = {np.dtype(np.int32): 0, np.dtype(np.uint32): 1, np.dtype(np.uint64): 2}[keys.dtype]
    plan = hs.plan(code, n, partition=nb, merge=merge, fan_in=fan)
    fused = nb != 1 and n > plan["tile"]
    assert ("hist_copy_in" in names) == fused and ("copy_in" in names) == (not fused), sorted(names)
    queue = merge == 1 and plan["fan_in"] == 2 and plan["merge_passes"] > 0
    assert ("copy_unmerged" in names) == queue, sorted(names)


def test_streams_do_not_share_work_space(oracle):
    a = I.generate("uniform31", 200_000, seed=13)
    b = I.generate("uniform64", 150_000, seed=14)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    ta, tb = to_dev(a), to_dev(b)
    torch.cuda.synchronize()
    for _ in range(3):
        hs.sort_keys(ta, stream=s1)
        hs.sort_keys(tb, stream=s2)
    torch.cuda.synchronize()
    assert_equal(ta.cpu().numpy(), oracle.sort(a)[0], "stream 1")
    assert_equal(tb.cpu().numpy(), oracle.sort(b)[0], "stream 2")


@pytest.mark.parametrize("fan,merge", SHAPES, ids=SHAPE_IDS)
@pytest.mark.parametrize("nb", [10, 256])
def test_batch_graph_replay(oracle, nb, fan, merge):
    # the whole call captured once in a CUDA graph, then replayed on new data
    off = make_batch(500, 1, 30_000, seed=15)
    n = int(off[-1])
    st = torch.cuda.Stream()
    to = to_dev(off)
    work = torch.empty(n, dtype=torch.int32, device=dev())
    for seed in (16, 17, 18):
        keys = I.generate("uniform31", n, seed=seed)
        ek, _ = oracle.sort_batch(keys, off, nbuckets=nb)
        with torch.cuda.stream(st):
            work.copy_(torch.from_numpy(keys))
            hs.sort_batch(work, to, partition=nb, graph=True, fan_in=fan, merge=merge)
        assert hs.stream_error(st) == 0
        assert_equal(work.cpu().numpy(), ek, f"graph replay seed {seed}")
    hs.graph_cache_clear()


def test_keys_graph_replay_counts_launches(oracle):
    st = torch.cuda.Stream()
    n = 100_000
    work = torch.empty(n, dtype=torch.uint64, device=dev())
    launches = []
    for seed in (20, 21):
        keys = I.generate("uniform64", n, seed=seed)
        with torch.cuda.stream(st):
            work.copy_(torch.from_numpy(keys))
            l0 = hs.kernel_launches()
            hs.sort_keys(work, graph=True)
            launches.append(hs.kernel_launches() - l0)
        assert hs.stream_error(st) == 0
        assert_equal(work.cpu().numpy(), oracle.sort(keys)[0], f"graph sort seed {seed}")
    assert launches[0] == launches[1] == hs.plan(2, n)["launches"]
    hs.graph_cache_clear()


def test_autotune_installs_a_correct_choice(oracle):
    from paper_2003_01216_gb300 import tune
    tune.clear()
    try:
        entries = tune.autotune(0, [1 << 16, 3 << 18], reps=2)
        assert [e["log2n"] for e in entries] == [16, 20]
        shapes = tune.candidates(0)
        assert len(shapes) == 3 * len(hs.tiles(0))
        for e in entries:
            assert set(e["ms"]) == {tune._key(*sh) for sh in shapes}
            best = min(shapes, key=lambda sh: e["ms"][tune._key(*sh)])
            assert (e["fan_in"], e["tile"], e["merge"]) == best
            f, t, m = tune.get_shape(0, 1 << e["log2n"])
            assert (f, t) == best[:2] and (m == best[2] or best[0] == 4)
            assert hs.plan(0, 1 << e["log2n"])["tile"] == e["tile"]
        keys = I.generate("zipf", 3 << 18, seed=44)
        gk, _, _, st = run(keys)  # fan_in = 0, tile = 0: the tuned entry
        assert st == 0
        assert_equal(gk, oracle.sort(keys)[0], "sort with the tuned shape")
        # every tile the tuner may install sorts correctly at this size
        for f, t, m in shapes:
            gk, _, _, st = run(keys, fan_in=f, tile=t, merge=m)
            assert st == 0
            assert_equal(gk, oracle.sort(keys)[0], f"sort with shape {tune._key(f, t, m)}")
    finally:
        tune.clear()


def test_merge_queue_wait_expires_and_context_survives(oracle):
    # the merge passes run as one persistent queue; the first merge block of
    # pass 1 never publishes its completion (debug flag 2) and the wait limit
    # is 2 ms: the pass-2 blocks that read its run give up and the call
    # reports HS_ERR_TIMEOUT
    keys = I.generate("uniform31", 100_000, seed=15)  # two packets of ~6 tiles: three passes
    assert hs.plan(0, keys.size, fan_in=2)["merge_passes"] >= 2
    _, _, _, st = run(keys, debug_flags=2, fan_in=2, merge=1)
    assert st == HS_TIMEOUT
    # the context stays usable and the next call is correct
    gk, _, _, st = run(keys, fan_in=2, merge=1)
    assert st == 0
    assert_equal(gk, oracle.sort(keys)[0], "sort after an expired merge-queue wait")


def test_host_merge_queue_wait_expires_and_context_survives(oracle):
    # a host-buffer call whose merge passes run in the queue's host-memory
    # instantiation (device tickets packet by packet, last passes from the
    # second counter, a few CTAs on it from the start): the first device
    # ticket's block never publishes its completion (debug flag 2, wait limit
    # 2 ms), so the device tickets that read its run and the host tickets of
    # its packet give up, and hs_stream_error reports HS_ERR_TIMEOUT
    import ctypes

    from paper_2003_01216_gb300 import _native as N
    keys = I.generate("uniform31", 300_000, seed=17)
    assert hs.plan(0, keys.size, fan_in=2, merge=1)["merge_passes"] >= 2
    pinned = torch.from_numpy(keys.copy()).pin_memory()
    o = N.make_opts(partition=10, fan_in=2, merge=1, debug_flags=2)
    assert N.lib().hs_sort_keys_host(N.HS_INT32, pinned.data_ptr(), keys.size, ctypes.byref(o),
                                      torch.cuda.current_stream().cuda_stream) == 0
    assert hs.stream_error() == HS_TIMEOUT
    # the context stays usable and the next call is correct
    pinned.copy_(torch.from_numpy(keys))
    hs.sort_keys_host(pinned, fan_in=2, merge=1)
    assert hs.stream_error() == 0
    assert_equal(pinned.numpy(), oracle.sort(keys)[0], "host-buffer sort after an expired merge-queue wait")


@pytest.mark.parametrize("dist,n,with_vals", [("uniform31", 3_000_000, False), ("zipf", 1_500_000, True),
                                              ("uniform64", 1_000_000, True), ("sorted", 2_000_000, False)])
def test_merge_queue_equals_per_pass_launches(oracle, dist, n, with_vals):
    # one persistent merge launch (merge = 1) against one co-rank and one
    # merge launch per pass (merge = 2): the same bits, and the oracle's
    keys = I.generate(dist, n, seed=16)
    vals = I.index_values(n) if with_vals else None
    a = run(keys, vals, fan_in=2, merge=1)
    b = run(keys, vals, fan_in=2, merge=2)
    assert a[3] == 0 and b[3] == 0
    assert_equal(a[0], b[0], "keys: queue vs per-pass")
    ek, ev, eo = oracle.sort(keys, vals)
    assert_equal(a[0], ek, "keys")
    assert_equal(a[2], eo, "packet offsets")
    if with_vals:
        assert_equal(a[1], b[1], "values: queue vs per-pass")
        assert_equal(a[1], ev, "stable values")
