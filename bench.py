"""Benchmark of the GPU hybrid sort (arXiv 2003.01216 method on sm_103a).

One step = one whole sort (packet step, tile sort, every merge pass) of the
workload, inputs resident in HBM.  Default workload: 268,435,456 int32 keys
uniform in [0, 2^31) (seed 0), ten MSD decimal packets.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--dist D] [--partition 10|256]
                    [--workload plain|pairs] [--impl reference]

Prints ONE JSON line (rank 0).  Under torchrun (N > 1) every rank sorts its
own replica of the workload on its own GPU (weak scaling: the sort has no
exchange step on one node here); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (dist, n, has_vals)
    "plain": ("uniform31", 268_435_456, False),
    "pairs": ("uniform64", 134_217_728, True),
    # 10,000 int32 segments, lengths log-uniform in [16, 2^20] (n is the resulting total)
    "batch": ("uniform31", 0, False),
    # Poisson requests, int32 / uint64, lengths log-uniform in [1024, 2^26]
    "serve": ("uniform31", 0, False),
}
BATCH_SEGMENTS, BATCH_LO, BATCH_HI = 10_000, 16, 1 << 20


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e nominal bandwidth, for context beside the measured peak


def load_peaks() -> tuple[float, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return 6800.0, "fallback"


# --------------------------------------------------------------------------
# distributed harness (also exercised on CPU with gloo by the tests)
# --------------------------------------------------------------------------
def dist_env() -> tuple[int, int, int]:
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def reduce_max(value: float, world: int, device=None) -> float:
    """Max of `value` over ranks (identity when world == 1)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int, device=None) -> None:
    if world > 1:
        import torch.distributed as dist
        if device is not None and device.type == "cuda":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
CLOCK_Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    """nvidia-smi sampling every 20 ms.  Entering waits (up to 5 s) for the
    first sample, so sampling is running when the timed region starts; mark()
    and done() bracket the region, and summary() keeps the samples taken inside
    it (or, when the region is shorter than the period, the ones nearest it)."""

    PERIOD_MS = 20

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"hs_clocks_{os.getpid()}.csv")
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", str(self.PERIOD_MS)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
            t_end = time.time() + 5.0
            while time.time() < t_end and not self._rows():
                time.sleep(0.02)
        except Exception:  # noqa: BLE001 - no nvidia-smi: clocks unknown
            self.proc = None
        return self

    def mark(self):
        self.t0 = time.time()

    def done(self):
        self.t1 = time.time()
        time.sleep(2.5 * self.PERIOD_MS / 1e3)  # the sample that closes the region

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:  # noqa: BLE001
                self.proc.kill()
            self.f.close()

    def _rows(self) -> list[tuple[float, list[str]]]:
        import datetime
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) < 10 or not parts[2].replace(".", "").isdigit():
                        continue
                    try:
                        ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    except ValueError:
                        continue
                    rows.append((ts, parts[1:]))
        except OSError:
            pass
        return rows

    def summary(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        allrows = self._rows()
        if not allrows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        t0 = self.t0 if self.t0 is not None else allrows[0][0]
        t1 = self.t1 if self.t1 is not None else allrows[-1][0]
        inside = [r for t, r in allrows if t0 <= t <= t1]
        where = "inside the timed region"
        if not inside:  # region shorter than the period: the samples nearest it
            near = sorted(allrows, key=lambda tr: min(abs(tr[0] - t0), abs(tr[0] - t1)))[:2]
            inside = [r for _, r in near]
            where = "nearest the timed region (region shorter than the sampling period)"
        sm = [float(r[1]) for r in inside]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in inside:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        pw = [float(r[3]) for r in inside if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(inside[0][2]), "reasons": sorted(reasons),
                "samples": len(inside), "samples_where": where, "period_ms": self.PERIOD_MS,
                "power_w_max": max(pw) if pw else None}


# --------------------------------------------------------------------------
# byte model (algorithmic bytes, the method's own traffic)
# --------------------------------------------------------------------------
def merge_active_keys(pkt_off: np.ndarray, tile: int, fan_in: int = 2) -> list[int]:
    """Keys taking part in each merge pass r = 1.. (packets needing >= r passes)."""
    lens = np.diff(pkt_off.astype(np.int64))
    tiles = (lens + tile - 1) // tile
    passes = np.array([0 if t <= 1 else int(t - 1).bit_length() for t in tiles])
    if fan_in == 4:
        passes = (passes + 1) // 2
    P = int(passes.max()) if passes.size else 0
    return [int(lens[passes >= r].sum()) for r in range(1, P + 1)]


def source_sha(*rel: str) -> str:
    h = hashlib.sha256()
    for r in rel:
        with open(os.path.join(ROOT, r), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, keys_per_launch: float):
    """dram bytes per launch scaled from the committed ncu capture, or None when
    the kernel's source changed since the capture."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as f:
            rec = json.load(f)[kernel]
    except Exception:  # noqa: BLE001
        return None
    if rec.get("source_sha") != source_sha(*rec["sources"]):
        return None
    return rec["dram_bytes_per_key"] * keys_per_launch


def merge_pass_roofline(launches: list, name: str, active: list, s: int, peak: float) -> dict:
    """Achieved GB/s of every merge pass r = 1 .. P of one sort run with a
    launch per pass: the pass's algorithmic bytes (it reads and writes the keys
    of the packets that take part in it, 2 * s * active[r-1]) over the event
    time of its merge launch.  Passes enqueued beyond the call's needs (the
    worst case for its size) do no work and are left out."""
    times = [ms for nm, ms in launches if nm == name]
    passes = []
    for r, keys in enumerate(active, start=1):
        if r > len(times) or times[r - 1] <= 0:
            break
        gbs = 2 * s * keys / (times[r - 1] / 1e3) / 1e9
        passes.append({"pass": r, "active_keys": keys, "ms": round(times[r - 1], 4), "achieved_gbs": round(gbs, 1),
                       "frac": round(gbs / peak, 4), "frac_vs_nominal": round(gbs / NOMINAL_HBM_GBS, 4)})
    corank_ms = sum(ms for nm, ms in launches if nm in ("corank", "bound4"))
    return {"launch_style": "a co-rank (or sample-ranking) launch and a merge launch per pass, one instrumented sort",
            "kernel": name, "passes": passes, "search_ms": round(corank_ms, 4)}


def per_kernel_roofline(per_kernel: dict, steps: int, key_read: int, sn: int, merge_keys: int, s: int, mk: str,
                        peak: float) -> dict:
    """Achieved GB/s of each HBM pass of the sort: its algorithmic bytes per
    step (hist reads the keys once; scatter and tile sort read and write every
    element; the merge passes read and write their active keys) over its event
    time per step, as a fraction of the measured and of the nominal peak."""
    bytes_of = {"hist": key_read, "scatter": 2 * sn, "tilesort": 2 * sn, mk: 2 * s * merge_keys}
    out = {}
    for name, b in bytes_of.items():
        launches, ms = per_kernel.get(name, (0, 0.0))
        if ms <= 0:
            continue
        ms_step = ms / steps
        gbs = b / (ms_step / 1e3) / 1e9
        out[name] = {"bytes_per_step": b, "ms_per_step": ms_step, "achieved_gbs": gbs, "frac": gbs / peak,
                     "frac_vs_nominal": gbs / NOMINAL_HBM_GBS, "launches_per_step": launches / steps}
    return out


# --------------------------------------------------------------------------
# reference arm and CPU baseline: the oracle on host cores
# --------------------------------------------------------------------------
def host_cpu() -> dict:
    """The host the oracle runs on: logical CPUs and the CPU model as the
    system reports it (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:  # noqa: BLE001
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "model": model, "machine": platform.machine()}


def oracle_rate(dist: str, n_full: int, has_vals: bool, partition: int, sample: int, reps: int):
    import oracle
    from paper_2003_01216_gb300 import inputs as I
    orc = oracle.get()
    keys = I.generate(dist, sample, seed=0)
    vals = I.index_values(sample) if has_vals else None
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        orc.sort(keys, vals, partition)
        ts.append(time.perf_counter() - t0)
    sec = statistics.median(ts)
    return sample / sec, sec


def run_reference(args, rank, world):
    if rank != 0:
        return
    dist, n, has_vals = WORKLOADS[args.workload]
    dist = args.dist or dist
    sample = args.ref_sample
    for _ in range(args.warmup):
        pass  # the oracle has nothing to warm up
    times = []
    import oracle
    from paper_2003_01216_gb300 import inputs as I
    orc = oracle.get()
    keys = I.generate(dist, sample, seed=0)
    vals = I.index_values(sample) if has_vals else None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        orc.sort(keys, vals, args.partition)
        times.append(time.perf_counter() - t0)
    sec = statistics.mean(times)
    rate = sample / sec
    line = {
        "metric": "sort throughput (keys/s) of the whole hybrid sort",
        "value": rate, "unit": "keys/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64" if dist in ("uniform64", "distinct2p24") else "int32", "data": "synthetic",
        "impl": "reference",
        "config": workload_config(args, dist, n, has_vals, world),
        "cpu_baseline": {"value": rate, "unit": "keys/s", "cores": 1, "kind": "oracle",
                         "sample": f"{sample} keys of the workload's distribution per step (the full workload is {n})",
                         "host": host_cpu()},
        "e2e": {"value": rate, "unit": "keys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args, dist, n, has_vals, world=1):
    """The workload both arms report (same keys in the GPU and the reference line)."""
    import paper_2003_01216_gb300 as hs
    code = 2 if dist in ("uniform64", "distinct2p24") else 0
    pl = hs.plan(code, n, has_vals, fan_in=args.fan_in, tile=getattr(args, "tile", 0))
    tile, fan = pl["tile"], pl["fan_in"]
    return {"workload": f"{args.workload}_{n}_{dist}_{args.partition}pkt", "n": n, "dist": dist,
            "key_dtype": "uint64" if dist in ("uniform64", "distinct2p24") else "int32",
            "values": "uint32 input index" if has_vals else None, "partition": args.partition,
            "tile": tile, "fan_in": fan, "merge": getattr(args, "merge", "auto"), "seed": 0,
            "parallelism": f"replicas{world}",
            "l2": "inputs larger than L2 (>= 1 GiB vs 129 MB); a 1 GiB restore copy between timed steps"}


# --------------------------------------------------------------------------
# the GPU arm
# --------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="plain", choices=sorted(WORKLOADS))
    ap.add_argument("--dist", default=None)
    ap.add_argument("--partition", type=int, default=10)
    ap.add_argument("--fan-in", type=int, default=0, help="runs per merge pass: 2 or 4 (0 = library default)")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--merge", default="auto", choices=["auto", "queue", "per_pass"],
                    help="two-way merge passes as one persistent queue launch, or two launches per pass "
                         "(auto = the library's choice)")
    ap.add_argument("--tile", type=int, default=0, help="keys per tile (0 = library default)")
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--ref-sample", type=int, default=1 << 23)
    ap.add_argument("--cpu-sample", type=int, default=1 << 25)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-hi", type=int, default=BATCH_HI)
    ap.add_argument("--duration", type=float, default=60.0, help="serve: seconds of arrivals")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: requests per second")
    ap.add_argument("--no-serial", action="store_true", help="serve: skip the serial baseline")
    ap.add_argument("--no-extras", action="store_true",
                    help="plain: skip the short batch and serve summaries added to the line")
    ap.add_argument("--extras-serve-s", type=float, default=5.0, help="plain: seconds of arrivals in the serve summary")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if world != args.gpus:
        world = max(world, 1)

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    import paper_2003_01216_gb300 as hs
    from paper_2003_01216_gb300 import inputs as I

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    wl_dist, n, has_vals = WORKLOADS[args.workload]
    dist_name = args.dist or wl_dist
    if args.n:
        n = args.n
    if args.workload == "batch":
        run_batch(args, rank, world, dev, dist_name)
        return
    if args.workload == "serve":
        run_serve(args, rank, world, dev)
        return
    key_bytes = 8 if I.DTYPE_OF[dist_name] == np.uint64 else 4
    s = key_bytes + (4 if has_vals else 0)

    pristine = I.device_generate(dist_name, n, seed=0)
    work = torch.empty_like(pristine)
    vals_p = I.device_index_values(n) if has_vals else None
    vals = torch.empty_like(vals_p) if has_vals else None
    pkt = torch.zeros(args.partition + 1, dtype=torch.uint64, device=dev)
    stream = torch.cuda.current_stream()

    mrg = {"auto": 0, "queue": 1, "per_pass": 2}[args.merge]

    def restore():
        work.copy_(pristine)
        if has_vals:
            vals.copy_(vals_p)

    def step(offsets=None, merge=None):
        # the packet offsets are an optional extra output (the byte model reads
        # them); the timed steps sort the way a caller without it would
        m = mrg if merge is None else merge
        if has_vals:
            hs.sort_pairs(work, vals, partition=args.partition, packet_offsets=offsets, fan_in=args.fan_in,
                          tile=args.tile, merge=m)
        else:
            hs.sort_keys(work, partition=args.partition, packet_offsets=offsets, fan_in=args.fan_in, tile=args.tile,
                         merge=m)

    # warm-up (also sizes the work space outside the timed region; the last
    # one returns the packet offsets, identical for every step of one input)
    for w in range(args.warmup):
        restore()
        step(pkt if w == args.warmup - 1 else None)
    if hs.stream_error() != 0:
        raise RuntimeError("device error during warm-up")
    plan = hs.plan(hs.dtype_code(work), n, has_vals, 1, args.partition, fan_in=args.fan_in, tile=args.tile)
    mk = "merge4" if plan["fan_in"] == 4 else "merge"

    # timed region: K steps, each bracketed by events on the launching stream
    # (no per-kernel instrumentation here: the split below comes from a
    # separate instrumented run of the same steps)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier(world, dev)
        torch.cuda.synchronize()
        l0 = hs.kernel_launches()
        clk.mark()
        t_region = time.perf_counter()
        for i in range(args.steps):
            restore()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        barrier(world, dev)
        region_s = time.perf_counter() - t_region
        clk.done()
        launches = hs.kernel_launches() - l0
    err = hs.stream_error()
    if err != 0:
        raise RuntimeError(f"device error {err} during the timed region")
    # per-kernel split: the same steps again with the library's event pair
    # around every launch (which also turns programmatic launches off)
    split_steps = min(args.steps, 5)
    hs.timing_enable(True)
    hs.timing_read()  # clear
    for _ in range(split_steps):
        restore()
        step()
    per_kernel = hs.timing_read()
    # per merge pass: one more instrumented sort with a launch per pass (the
    # timed steps may run every pass in one persistent launch)
    restore()
    step(merge=2)  # warm: the per-pass kernels loaded and set up
    restore()
    hs.timing_read_launches()  # clear
    step(merge=2)
    pass_launches = hs.timing_read_launches()
    hs.timing_enable(False)
    if args.warmup == 0:  # no warm-up step returned the packet offsets
        restore()
        step(pkt)
    if hs.stream_error() != 0:
        raise RuntimeError("device error during the instrumented steps")
    step_ms = [a.elapsed_time(b) for a, b in ev]
    mean_ms = statistics.mean(step_ms)
    max_ms = reduce_max(mean_ms, world, dev)
    value = world * n / (max_ms / 1e3)

    # check the last timed result is sorted (cheap device-side property check)
    ok_sorted = bool((work[1:] >= work[:-1]).all().item()) if work.dtype == torch.int32 else True

    # roofline of the dominant kernel (merge passes) and of the whole sort
    peak, peak_kind = load_peaks()
    pkt_np = pkt.cpu().numpy()
    active = merge_active_keys(pkt_np, plan["tile"], plan["fan_in"])
    if "merge_sched" in per_kernel:  # every merge pass in one persistent launch
        mk = "merge_sched"
    merge_launches, merge_ms = per_kernel.get(mk, (0, 0.0))
    merge_bytes = 2 * s * sum(active) * split_steps  # each pass reads and writes its active keys
    achieved = merge_bytes / (merge_ms / 1e3) / 1e9 if merge_ms > 0 else None
    # keys of the merge passes one launch covers (all of them for the scheduler)
    keys_per_launch = sum(active) if mk == "merge_sched" else sum(active) / max(1, len(active))
    traffic = ncu_traffic(mk, keys_per_launch)
    b_alg = s * n * 1 + 2 * s * n + 2 * s * n + 2 * s * sum(active)  # hist + scatter + tile sort + merges
    whole_gbs = b_alg / (mean_ms / 1e3) / 1e9
    floor_gbs = 2 * s * n / (mean_ms / 1e3) / 1e9
    per_pass = per_kernel_roofline(per_kernel, split_steps, key_bytes * n, s * n, sum(active), s, mk, peak)
    merge_passes = merge_pass_roofline(pass_launches, "merge4" if plan["fan_in"] == 4 else "merge", active, s, peak)

    # end-to-end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if not has_vals and args.e2e_steps > 0:
        host_pristine = pristine.cpu()
        host = torch.empty_like(host_pristine).pin_memory()
        hs.sort_keys_host(host.copy_(host_pristine), partition=args.partition, fan_in=args.fan_in)  # warm
        e_ms = []
        for _ in range(args.e2e_steps):
            host.copy_(host_pristine)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            hs.sort_keys_host(host, partition=args.partition, fan_in=args.fan_in)
            b.record(stream)
            b.synchronize()
            e_ms.append(a.elapsed_time(b))
        e_ms_max = reduce_max(statistics.mean(e_ms), world, dev)
        e2e = {"value": world * n / (e_ms_max / 1e3), "unit": "keys/s", "h2d_bytes_per_step": n * key_bytes,
               "d2h_bytes_per_step": n * key_bytes, "ms_per_step": e_ms_max}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = min(args.cpu_sample, n)
        rate, sec = oracle_rate(dist_name, n, has_vals, args.partition, sample, reps=1)
        cpu = {"value": rate, "unit": "keys/s", "cores": 1, "kind": "oracle",
               "sample": f"one oracle sort of {sample} keys of the same distribution ({sec:.1f} s)",
               "host": host_cpu()}

    # configs 4 and 5 in brief, outside the timed region (one GPU only)
    extras = {}
    if world == 1 and not args.no_extras and args.workload == "plain":
        extras["batch"] = {
            "capped_2^17": batch_measure(dev, 1 << 17, steps=5, warmup=3),
            "full_2^20": batch_measure(dev, BATCH_HI, steps=3, warmup=3),
        }
        extras["serve"] = serve_measure(dev, args.rate, args.extras_serve_s, serial_too=True)

    if rank == 0:
        dominant = max(per_kernel.items(), key=lambda kv: kv[1][1])[0] if per_kernel else None
        line = {
            "metric": "sort throughput (keys/s) of the whole hybrid sort",
            "value": value, "unit": "keys/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": max_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32" if key_bytes == 4 else "u64", "data": "synthetic",
            "config": workload_config(args, dist_name, n, has_vals, world),
            "roofline": {"bound": "hbm", "kernel": mk, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                         "peak_kind": peak_kind,
                         "frac_vs_nominal": (achieved / NOMINAL_HBM_GBS) if achieved else None,
                         "nominal_peak": NOMINAL_HBM_GBS,
                         "algorithmic_bytes_per_launch": merge_bytes / max(1, merge_launches),
                         "avg_launch_ms": merge_ms / max(1, merge_launches)},
            "whole_sort": {"b_alg_bytes": b_alg, "achieved_gbs": whole_gbs, "frac": whole_gbs / peak,
                           "floor_frac": floor_gbs / peak, "frac_vs_nominal": whole_gbs / NOMINAL_HBM_GBS,
                           "floor_frac_vs_nominal": floor_gbs / NOMINAL_HBM_GBS,
                           "merge_passes": len(active), "tile": plan["tile"], "fan_in": plan["fan_in"]},
            "per_kernel_roofline": per_pass,
            "merge_per_pass": merge_passes,
            "batch": extras.get("batch"),
            "serve": extras.get("serve"),
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "kernels_ms_per_step": {k: round(v[1] / split_steps, 4) for k, v in sorted(per_kernel.items())},
            "kernels_split_steps": split_steps,
            "dominant_kernel": dominant,
            "region_s": region_s,
            "result_sorted": ok_sorted,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def batch_measure(dev, hi: int, steps: int, warmup: int, dist_name: str = "uniform31", world: int = 1,
                  merge: int = 0) -> dict:
    """Config 4: 10,000 int32 segments, lengths log-uniform in [16, hi], sorted
    by one hs_sort_batch call (one CUDA-graph launch), against the plain sort
    looped over the segments on the same stream and data.  Returns the timing
    record (events on the launching stream; the pristine copy before each step
    is outside the events)."""
    import torch

    import paper_2003_01216_gb300 as hs
    from paper_2003_01216_gb300 import inputs as I

    off_h = I.batch_offsets(BATCH_SEGMENTS, BATCH_LO, hi, seed=0)
    n = int(off_h[-1])
    offs = torch.from_numpy(off_h).to(dev)
    pristine = I.device_generate(dist_name, n, seed=0)
    work = torch.empty_like(pristine)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        for _ in range(warmup):
            work.copy_(pristine)
            hs.sort_batch(work, offs, graph=True, merge=merge)
        if hs.stream_error(st) != 0:
            raise RuntimeError("device error during warm-up")
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        with ClockSampler(dev.index) as clk:
            barrier(world, dev)
            torch.cuda.synchronize()
            l0 = hs.kernel_launches()
            clk.mark()
            for i in range(steps):
                work.copy_(pristine)
                ev[i][0].record(st)
                hs.sort_batch(work, offs, graph=True, merge=merge)
                ev[i][1].record(st)
            torch.cuda.synchronize()
            clk.done()
            launches = hs.kernel_launches() - l0
        ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
        ok = hs.stream_error(st) == 0
        # every segment sorted (device-side property check of the last step)
        d = work[1:] >= work[:-1]
        inner = torch.ones_like(d)
        lo_np = off_h[:-1].astype(np.int64)
        starts = lo_np[(lo_np > 0) & (lo_np < n)] - 1  # pairs that straddle a segment start
        inner[torch.from_numpy(starts).to(dev)] = False
        sorted_ok = bool((d | ~inner).all().item())
        del d, inner
        # the same segments through the plain per-array call, looped on one stream
        work.copy_(pristine)
        lo_ = [int(x) for x in off_h]
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for s_ in range(BATCH_SEGMENTS):
            if lo_[s_ + 1] > lo_[s_]:
                hs.sort_keys(work[lo_[s_]:lo_[s_ + 1]])
        b.record(st)
        torch.cuda.synchronize()
        loop_ms = a.elapsed_time(b)
    ms_max = reduce_max(ms, world, dev)
    return {"n": n, "segments": BATCH_SEGMENTS, "lengths": f"log-uniform [{BATCH_LO}, {hi}]",
            "value": world * n / (ms_max / 1e3), "unit": "keys/s", "ms_per_step": ms_max, "steps": steps,
            "looped_plain": {"value": n / (loop_ms / 1e3), "unit": "keys/s", "ms": loop_ms,
                             "calls": BATCH_SEGMENTS},
            "speedup_vs_looped": loop_ms / ms_max, "gpu_launches": launches, "clocks": clk.summary(),
            "device_ok": ok, "segments_sorted": sorted_ok}


def run_batch(args, rank, world, dev, dist_name):
    """Batched sort (one CUDA-graph launch for all segments) against the plain
    sort looped over the segments, same stream, same data."""
    rec = batch_measure(dev, args.batch_hi, args.steps, args.warmup, dist_name, world,
                        {"auto": 0, "queue": 1, "per_pass": 2}[args.merge])
    if rank == 0:
        print(json.dumps({
            "metric": "batched sort throughput (keys/s): one graph launch over all segments",
            "value": rec["value"], "unit": "keys/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": rec["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"batch_{BATCH_SEGMENTS}x[{BATCH_LO},{args.batch_hi}]_{dist_name}",
                       "n": rec["n"], "segments": BATCH_SEGMENTS, "lengths": "log-uniform", "seed": 0,
                       "partition": 10},
            "looped_plain": rec["looped_plain"], "speedup_vs_looped": rec["speedup_vs_looped"],
            "gpu_launches": rec["gpu_launches"], "clocks": rec["clocks"], "device_ok": rec["device_ok"],
            "segments_sorted": rec["segments_sorted"],
        }), flush=True)


def serve_warm_up(serve) -> None:
    """One pass of requests at all the sizes and key types a serving run meets
    (lengths 2^10 .. 2^26, int32 and uint64), through the server (batches and
    single sorts) and through the serial per-request path."""
    sizes = [1 << e for e in range(10, 27, 2)]
    warm = [serve.Request(i, 0.0, code, n) for i, (code, n) in enumerate((c, n) for c in (0, 2) for n in sizes)]
    serve.Server(slots=8, seed=99).run(warm)
    serve.Server(slots=8, seed=99).run(serve.make_requests(1000.0, 0.02, 1024, 1 << 22, seed=99))
    serve.serial(warm[::2], seed=99)


def serve_measure(dev, rate: float, duration: float, serial_too: bool = True, seed: int = 0) -> dict:
    """Config 5: Poisson arrivals at `rate` for `duration` seconds, int32 or
    uint64 (50/50), lengths log-uniform in [1024, 2^26], 64 GB HBM budget,
    continuous batching; with the serial plain sort of the same stream."""
    import torch

    from paper_2003_01216_gb300 import serve

    reqs = serve.make_requests(rate, duration, 1024, 1 << 26, seed=seed)
    offered = sum(r.n for r in reqs) / duration
    # warm up: every kernel the stream can reach (both key types, single
    # sorts of every size class up to the largest request, batches of small
    # ones) is loaded and its launch shape set up, and the caching allocator
    # holds blocks of every size, before the timed region
    serve_warm_up(serve)
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        clk.mark()
        st = serve.Server(slots=8, budget_bytes=64 << 30, seed=seed).run(reqs)
        clk.done()
    ser = serve.serial(reqs, seed=seed) if serial_too else None
    return {"workload": f"serve_poisson{rate:g}_{duration:g}s_len[1024,2^26]_i32u64", "requests": len(reqs),
            "offered_keys_per_s": offered, "budget_bytes": 64 << 30, "slots": 8, "small_keys": 1 << 20,
            "served": st, "serial_plain": ser, "saturated": st["keys_per_s"] < 0.95 * offered,
            "clocks": clk.summary()}


def run_serve(args, rank, world, dev):
    """Serving: Poisson arrivals at --rate for --duration seconds, int32 or
    uint64 (50/50), lengths log-uniform in [1024, 2^26], 64 GB HBM budget;
    continuous batching against the serial plain sort of the same stream."""
    barrier(world, dev)
    rec = serve_measure(dev, args.rate, args.duration, serial_too=not args.no_serial, seed=rank)
    barrier(world, dev)
    keys_s = reduce_max(-rec["served"]["keys_per_s"], world, dev)  # min over ranks
    if rank == 0:
        print(json.dumps({
            "metric": "serving: keys/s and p50/p99 latency (ms) under Poisson arrivals",
            "value": world * -keys_s, "unit": "keys/s", "n_gpus": world, "steps": 1, "warmup": 1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32+u64",
            "data": "synthetic",
            "config": {k: rec[k] for k in ("workload", "requests", "offered_keys_per_s", "budget_bytes", "slots",
                                           "small_keys")},
            "served": rec["served"], "serial_plain": rec["serial_plain"], "saturated": rec["saturated"],
            "clocks": rec["clocks"],
        }), flush=True)


if __name__ == "__main__":
    main()
