"""Serving loop on the GPU: requests arriving over time (Poisson), mixed
int32/uint64 and mixed lengths, admitted by slots and HBM budget, small ones
continuously batched.  Every request's result in the mix must equal the same
request sorted alone, bit for bit; a sample is checked against the oracle."""
import numpy as np
import pytest
import torch

import paper_2003_01216_gb300 as hs
from paper_2003_01216_gb300 import inputs as I
from paper_2003_01216_gb300 import serve

pytestmark = pytest.mark.gpu


def alone(r, seed):
    t = I.device_generate(I.request_dist(r.dtype_code), r.n, seed=seed, stream=r.rid)
    hs.sort_keys(t)
    assert hs.stream_error() == 0
    return t.cpu().numpy()


def test_mix_equals_alone_and_oracle(oracle):
    reqs = serve.make_requests(rate=20_000, duration=0.004, lo=1024, hi=1 << 18, seed=3)
    assert len(reqs) >= 40
    srv = serve.Server(slots=4, budget_bytes=1 << 30, small_keys=1 << 14, seed=3, keep_results=True)
    stats = srv.run(reqs)
    assert stats["batches"] > 0 and stats["singles"] > 0      # both paths ran
    assert stats["peak_inflight"] > 1                          # work overlapped on the device
    for r in reqs:
        got = srv.results[r.rid]
        assert np.array_equal(got, alone(r, 3)), f"request {r.rid} differs alone vs in the mix"
    for r in reqs[::7]:
        keys = I.generate(I.request_dist(r.dtype_code), r.n, seed=3, stream=r.rid)
        assert np.array_equal(srv.results[r.rid], oracle.sort(keys)[0]), f"request {r.rid} vs oracle"


def test_two_hundred_requests_vs_oracle(oracle):
    # a seeded sample of over 200 requests of both key types, served with
    # batching and single sorts overlapping on 8 streams: every result equals
    # the oracle's sort of the same request's keys (made on the host by the
    # seeded generator)
    reqs = serve.make_requests(rate=50_000, duration=0.005, lo=1024, hi=1 << 17, seed=6)
    assert len(reqs) >= 200
    srv = serve.Server(slots=8, budget_bytes=1 << 30, small_keys=1 << 13, seed=6, keep_results=True)
    stats = srv.run(reqs)
    assert stats["batches"] > 0 and stats["singles"] > 0
    assert {r.dtype_code for r in reqs} == {0, 2}
    for r in reqs:
        keys = I.generate(I.request_dist(r.dtype_code), r.n, seed=6, stream=r.rid)
        assert np.array_equal(srv.results[r.rid], oracle.sort(keys)[0]), f"request {r.rid} vs oracle"


def test_small_budget_still_serves_everything():
    reqs = serve.make_requests(rate=5_000, duration=0.01, lo=1024, hi=1 << 16, seed=4)
    srv = serve.Server(slots=4, budget_bytes=64 << 10, small_keys=1 << 12, seed=4, keep_results=True)
    stats = srv.run(reqs)
    assert stats["requests"] == len(reqs) == len(srv.results)
    for r in reqs:
        assert np.all(srv.results[r.rid][1:] >= srv.results[r.rid][:-1])


def test_serial_baseline_runs():
    reqs = serve.make_requests(rate=2_000, duration=0.01, lo=1024, hi=1 << 16, seed=5)
    st = serve.serial(reqs, seed=5)
    assert st["requests"] == len(reqs) and st["keys_per_s"] > 0
    torch.cuda.synchronize()
