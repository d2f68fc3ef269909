"""Serving loop: sort requests arriving over time, with continuous batching.

Requests (an int32 or uint64 array each) arrive at their own times.  The
loop keeps every request's buffers on the device and admits waiting
requests whenever a stream slot and enough of the HBM budget are free:

  * a request longer than `small_keys` gets a slot of its own and one
    `hs_sort_keys` call;
  * requests up to `small_keys` that are waiting together (same key type) are
    packed back to back into one buffer and sorted by one `hs_sort_batch`
    call, each request a segment;
  * admitted work from different slots overlaps on the device (one CUDA
    stream per slot); completion is observed with CUDA events.

Memory: a request holds its keys plus the sort's work space (both from
PyTorch's caching allocator, on the slot's stream), counted against the budget
from admission to completion.  Payloads are produced on the device by the
seeded generator (stream = request id) at admission, so no host traffic sits
on the critical path; latency runs from the scheduled arrival time to the
moment the loop sees the completion event.

`serial()` replays the same request stream through one stream, one plain
`hs_sort_keys` call per request, in arrival order: the per-array baseline.
"""
from __future__ import annotations

import collections
import dataclasses
import statistics
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    t_arrival: float  # seconds after the start of the run
    dtype_code: int   # 0 = int32, 2 = uint64
    n: int


def make_requests(rate: float, duration: float, lo: int, hi: int, seed: int = 0) -> list[Request]:
    from . import inputs as I
    t, codes, lens = I.poisson_requests(rate, duration, lo, hi, seed)
    return [Request(i, float(t[i]), int(codes[i]), int(lens[i])) for i in range(t.size)]


def _torch_dtype(code: int):
    import torch
    return torch.int32 if code == 0 else torch.uint64


def _key_bytes(code: int) -> int:
    return 4 if code == 0 else 8


class _Work:
    """One admitted unit: a single large request or a batch of small ones."""

    def __init__(self, reqs, slot, keys, ws, offsets, event, nbytes):
        self.reqs = reqs
        self.slot = slot
        self.keys = keys
        self.ws = ws
        self.offsets = offsets
        self.event = event
        self.nbytes = nbytes


class Server:
    def __init__(self, slots: int = 8, budget_bytes: int = 64 << 30, small_keys: int = 1 << 20,
                 batch_max_keys: int = 1 << 24, batch_max_reqs: int = 512, seed: int = 0,
                 keep_results: bool = False, device=None):
        import torch
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.streams = [torch.cuda.Stream(self.device) for _ in range(slots)]
        self.free_slots = list(range(slots))
        self.budget = budget_bytes
        self.small_keys = small_keys
        self.batch_max_keys = batch_max_keys
        self.batch_max_reqs = batch_max_reqs
        self.seed = seed
        self.keep = keep_results
        self.results: dict[int, np.ndarray] = {}

    def _bytes_for(self, code: int, n: int, nseg: int = 1) -> int:
        from . import workspace_size
        return n * _key_bytes(code) + workspace_size(code, n, False, nseg)

    def _launch(self, reqs: list[Request], slot: int, now: float) -> _Work:
        import torch

        import paper_2003_01216_gb300 as hs
        from . import inputs as I
        code = reqs[0].dtype_code
        dist = I.request_dist(code)
        st = self.streams[slot]
        total = sum(r.n for r in reqs)
        with torch.cuda.stream(st):
            keys = torch.empty(total, dtype=_torch_dtype(code), device=self.device)
            off = 0
            for r in reqs:
                I.device_generate(dist, r.n, seed=self.seed, stream=r.rid, out=keys[off:off + r.n])
                off += r.n
            if len(reqs) == 1:
                nbytes = self._bytes_for(code, total)
                ws = torch.empty(nbytes - total * _key_bytes(code), dtype=torch.uint8, device=self.device)
                hs.sort_keys(keys, workspace=ws)
                offsets = None
            else:
                offs = np.zeros(len(reqs) + 1, dtype=np.uint64)
                offs[1:] = np.cumsum([r.n for r in reqs])
                offsets = torch.from_numpy(offs).to(self.device, non_blocking=False)
                nbytes = self._bytes_for(code, total, len(reqs))
                ws = torch.empty(nbytes - total * _key_bytes(code), dtype=torch.uint8, device=self.device)
                hs.sort_batch(keys, offsets, workspace=ws)
            ev = torch.cuda.Event()
            ev.record(st)
        return _Work(reqs, slot, keys, ws, offsets, ev, nbytes)

    def run(self, requests: list[Request]) -> dict:
        """Serve `requests` in real time; returns throughput, latency
        percentiles and queue statistics."""
        pending = collections.deque(sorted(requests, key=lambda r: r.t_arrival))
        waiting: collections.deque[Request] = collections.deque()
        inflight: list[_Work] = []
        used = 0
        lat: dict[int, float] = {}
        depth_samples = []
        peak_used = peak_inflight = 0
        batches = singles = 0
        keys_done = 0
        t0 = time.perf_counter()
        while pending or waiting or inflight:
            now = time.perf_counter() - t0
            while pending and pending[0].t_arrival <= now:
                waiting.append(pending.popleft())
            still = []
            for w in inflight:  # completions
                if w.event.query():
                    t_done = time.perf_counter() - t0
                    for r in w.reqs:
                        lat[r.rid] = t_done - r.t_arrival
                        keys_done += r.n
                    if self.keep:
                        host = w.keys.cpu().numpy()
                        off = 0
                        for r in w.reqs:
                            self.results[r.rid] = host[off:off + r.n].copy()
                            off += r.n
                    used -= w.nbytes
                    self.free_slots.append(w.slot)
                else:
                    still.append(w)
            inflight = still
            groups = plan_admissions(waiting, len(self.free_slots), used, self.budget, len(inflight),
                                     self._bytes_for, self.small_keys, self.batch_max_keys, self.batch_max_reqs)
            for group, need in groups:
                if len(group) == 1 and group[0].n > self.small_keys:
                    singles += 1
                else:
                    batches += 1
                w = self._launch(group, self.free_slots.pop(), now)
                used += w.nbytes
                inflight.append(w)
            peak_used = max(peak_used, used)
            peak_inflight = max(peak_inflight, len(inflight))
            depth_samples.append(len(waiting))
            if not groups:
                time.sleep(20e-6)
        wall = time.perf_counter() - t0
        lats = np.array([lat[r.rid] for r in requests]) * 1e3
        return {
            "requests": len(requests), "keys": int(sum(r.n for r in requests)), "wall_s": wall,
            "keys_per_s": keys_done / wall,
            "p50_ms": float(np.percentile(lats, 50)), "p99_ms": float(np.percentile(lats, 99)),
            "mean_ms": float(lats.mean()), "max_ms": float(lats.max()),
            "batches": batches, "singles": singles, "peak_hbm_bytes": peak_used, "peak_inflight": peak_inflight,
            "queue_depth_mean": statistics.mean(depth_samples) if depth_samples else 0,
            "queue_depth_max": max(depth_samples) if depth_samples else 0,
        }


def plan_admissions(waiting, free_slots: int, used: int, budget: int, inflight: int, bytes_for, small_keys: int,
                    batch_max_keys: int, batch_max_reqs: int):
    """Admission policy (pure host logic).  Takes requests off the front of
    `waiting` (a deque, modified in place) while slots and budget allow:
    a large head goes alone; a small head takes the following small requests
    of its key type into one batch (up to batch_max_keys / batch_max_reqs).
    A unit that does not fit in the budget waits, unless nothing is in flight
    (then it runs alone, so the loop cannot stall).  Returns [(group, bytes)]."""
    out = []
    while waiting and free_slots > 0:
        head = waiting[0]
        if head.n > small_keys:
            group = [head]
        else:
            group, total = [], 0
            for r in waiting:
                if len(group) >= batch_max_reqs or r.n > small_keys or r.dtype_code != head.dtype_code:
                    break
                if group and total + r.n > batch_max_keys:
                    break
                group.append(r)
                total += r.n
        need = bytes_for(head.dtype_code, sum(r.n for r in group), len(group))
        if used + need > budget and (inflight > 0 or out):
            break
        for _ in group:
            waiting.popleft()
        out.append((group, need))
        used += need
        free_slots -= 1
    return out


def serial(requests: list[Request], seed: int = 0, device=None) -> dict:
    """The per-array baseline: one stream, one hs_sort_keys call per request,
    in arrival order, each started no earlier than its arrival."""
    import torch

    import paper_2003_01216_gb300 as hs
    from . import inputs as I
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    st = torch.cuda.Stream(dev)
    lat = []
    keys_done = 0
    t0 = time.perf_counter()
    for r in sorted(requests, key=lambda r: r.t_arrival):
        while time.perf_counter() - t0 < r.t_arrival:
            time.sleep(20e-6)
        with torch.cuda.stream(st):
            keys = torch.empty(r.n, dtype=_torch_dtype(r.dtype_code), device=dev)
            I.device_generate(I.request_dist(r.dtype_code), r.n, seed=seed, stream=r.rid, out=keys)
            hs.sort_keys(keys)
        st.synchronize()
        done = time.perf_counter() - t0
        lat.append(done - r.t_arrival)
        keys_done += r.n
    wall = time.perf_counter() - t0
    lats = np.array(lat) * 1e3
    return {"requests": len(requests), "keys_per_s": keys_done / wall, "wall_s": wall,
            "p50_ms": float(np.percentile(lats, 50)), "p99_ms": float(np.percentile(lats, 99)),
            "mean_ms": float(lats.mean())}
