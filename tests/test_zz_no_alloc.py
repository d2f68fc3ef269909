"""hs_sort_keys_noalloc: the keys-only sort for callers that cannot allocate
device memory (its scratch is a fixed array inside the library).  Called
through the C ABI and compared with hs_sort_keys and with the CPU oracle, bit
for bit, on two calls in a row; a call made after a warm call changes neither
the device's free memory nor PyTorch's allocation count.  Collected last, so a
run stopping at its first failure has already run every other test; it also
passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as orc
import paper_2003_01216_gb300 as hs
from paper_2003_01216_gb300 import _native as N
from paper_2003_01216_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MAX_KEYS = 1 << 20


def _noalloc(t, partition=10):
    stream = torch.cuda.current_stream().cuda_stream
    return N.lib().hs_sort_keys_noalloc(hs.dtype_code(t), t.data_ptr(), t.numel(), partition, stream)


# ("uniform64", 256) at 2^20 keys is the call with the largest scratch need
@pytest.mark.parametrize("dist,partition", [("uniform1e9", 10), ("int32full", 256), ("uniform64", 10),
                                            ("uniform64", 256), ("uniform32", 10)])
def test_noalloc_matches_sort_keys_twice(dist, partition):
    hs.timing_enable(False)
    dev = torch.device("cuda", 0)
    for call, (n, seed) in enumerate([(MAX_KEYS, 21), (300_001, 22)]):
        keys = I.generate(dist, n, seed=seed)
        ref = torch.from_numpy(keys).to(dev)
        hs.sort_keys(ref, partition=partition)
        got = torch.from_numpy(keys).to(dev)
        assert _noalloc(got, partition) == N.HS_OK, f"call {call}"
        assert hs.stream_error() == 0
        g = got.cpu().numpy()
        assert np.array_equal(g, ref.cpu().numpy()), f"call {call}: differs from hs_sort_keys"
        exp, _, _ = orc.get().sort(keys, None, partition)
        assert np.array_equal(g, exp), f"call {call}: differs from the oracle"


@pytest.mark.parametrize("dist,partition", [("uniform31", 10), ("uniform64", 256)])
def test_noalloc_allocates_nothing(dist, partition):
    hs.timing_enable(False)
    dev = torch.device("cuda", 0)
    keys = I.generate(dist, MAX_KEYS, seed=5)
    warm = torch.from_numpy(keys).to(dev)
    got = torch.from_numpy(keys).to(dev)
    # the warm call loads this path's kernels (module loading may take memory)
    assert _noalloc(warm, partition) == N.HS_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    alloc0 = torch.cuda.memory_allocated(dev)
    assert _noalloc(got, partition) == N.HS_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    alloc1 = torch.cuda.memory_allocated(dev)
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
    assert alloc1 == alloc0
    assert hs.stream_error() == 0
    assert torch.equal(got, warm)
    exp, _, _ = orc.get().sort(keys, None, partition)
    assert np.array_equal(got.cpu().numpy(), exp)


def test_noalloc_rejects_oversize_and_timing():
    dev = torch.device("cuda", 0)
    big = torch.zeros(MAX_KEYS + 1, dtype=torch.int32, device=dev)
    assert _noalloc(big) == N.HS_ERR_INVALID
    assert b"exceeds the maximum" in N.lib().hs_last_error()
    small = torch.arange(1000, 0, -1, dtype=torch.int32, device=dev)
    hs.timing_enable(True)
    try:
        assert _noalloc(small) == N.HS_ERR_INVALID
    finally:
        hs.timing_enable(False)
    assert _noalloc(small) == N.HS_OK
    assert hs.stream_error() == 0
    assert torch.equal(small.cpu(), torch.arange(1, 1001, dtype=torch.int32))


def test_noalloc_symbol_declared():
    assert hasattr(N.lib(), "hs_sort_keys_noalloc")
    assert ctypes.sizeof(ctypes.c_void_p) == 8
