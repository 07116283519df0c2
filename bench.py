#!/usr/bin/env python3
"""Benchmark of the length-bucketed word sort on GB300.

One step = the whole path (strip, bucket by length, sort every bucket, emit)
over one synthetic document resident in HBM, through the C ABI's device entry
point.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Workloads (seeded synthetic text shaped like the paper's Hamlet files, which
are not available here): plain_1m38 (default, 1,447,000 B), plain_190k
(194,560 B), plain_256m (268,435,456 B).

For N > 1 (launched by torch.distributed.run) every rank sorts its own copy of
the document on its own GPU: the work is independent per document, so there is
no collective on the data path (weak scaling); a barrier and a max-reduction
of the timings are the only communication.

--impl reference times the CPU oracle (the paper's bubble sort per length
bucket, OpenMP over buckets) on the host cores instead; under torchrun only
rank 0 runs it.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "input MB/s and words/s sorted on 1 GB300 (% HBM roofline); batched vs plain; p99"
L2_FLUSH_BYTES = 256 << 20  # larger than the 129 MB L2
FALLBACK_HBM_GBS = 6800.0

# Kernel families and the source file that holds each (for the traffic record).
KERNEL_SOURCE = {
    "tokenize": "k_tokenize1p.cu", "scatter": "k_scatter.cu", "emit": "k_scatter.cu",
    "tile_sort": "k_sort2.cu", "merge_pass": "k_sort2.cu",
}


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="plain_1m38", choices=["plain_190k", "plain_1m38", "plain_256m"])
    p.add_argument("--e2e-steps", type=int, default=None)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--prefix-bytes", type=int, default=None,
                   help="use only the first B bytes of the workload (profiling captures on smaller cases)")
    return p.parse_args(argv)


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def reduce_max(value: float, world: int) -> float:
    """Max of a float over all ranks (the process group must be initialised when world > 1)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def aggregate(bytes_per_step: int, words_per_step: int, steps: int, world: int, max_time_s: float) -> dict:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    total_bytes = bytes_per_step * steps * world
    return {"mb_per_s": total_bytes / max_time_s / 1e6,
            "words_per_s": words_per_step * steps * world / max_time_s}


def measured_peaks() -> tuple[float, str]:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_sha(family: str) -> str:
    src = os.path.join(ROOT, "paper_1407_6603_gb300", "csrc", KERNEL_SOURCE[family])
    h = hashlib.sha256()
    for f in (src, os.path.join(ROOT, "paper_1407_6603_gb300", "csrc", "bsort_dev.cuh")):
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(family: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source and this workload; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(path):
        return None
    sha = kernel_source_sha(family)
    for line in open(path):
        cells = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cells) >= 4 and cells[0] == family and cells[1] == workload and cells[3] == sha:
            try:
                return float(cells[2])
            except ValueError:
                return None
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile

        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, samples = [], [], set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            cells = [c.strip() for c in line.split(",")]
            if len(cells) < 9:
                continue
            try:
                sm.append(float(cells[1]))
                smax.append(float(cells[2]))
            except ValueError:
                continue
            samples += 1
            for name, cell in zip(names, cells[5:9]):
                if cell.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": samples}


def cpu_baseline(data, workload: str) -> dict:
    """The oracle as it stands, on the host cores: bubble sort per length bucket
    with OpenMP over buckets (the paper's design) for the paper-sized documents;
    its stable_sort path for the 256 MiB one."""
    import oracle

    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    if workload == "plain_256m":
        r = oracle.stable(data, nthreads=cores)
        kind_s = "O2 stable_sort per length bucket"
    else:
        r = oracle.bubble(data, nthreads=cores)
        kind_s = "O1 bubble sort per length bucket"
    dt = time.perf_counter() - t0
    return {"value": data.size / dt / 1e6, "unit": "MB/s", "cores": cores, "kind": "oracle",
            "sample": f"whole {workload} document ({data.size} B, {r['n_words']} words), {kind_s}, "
                      f"OpenMP over buckets on {cores} threads, {dt:.2f} s",
            "words_per_s": r["n_words"] / dt}


def run_reference(args) -> None:
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle
    import synth

    data = synth.plain(args.workload)
    cores = os.cpu_count() or 1
    if args.workload == "plain_256m":
        sample = data[: 16 << 20]
        fn, kind_s = oracle.stable, "O2 stable_sort per length bucket"
    else:
        # bubble sort is quadratic in the largest bucket: bound each step with a
        # prefix of the document (about a second of work per step)
        size = min(data.size, 512 << 10)
        if args.steps + args.warmup > 30:
            size = int(size * ((30 / (args.steps + args.warmup)) ** 0.5))
        sample = data[:size]
        fn, kind_s = oracle.bubble, "O1 bubble sort per length bucket"
    n_words = 0
    for _ in range(args.warmup):
        n_words = fn(sample, nthreads=cores)["n_words"]
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        n_words = fn(sample, nthreads=cores)["n_words"]
        times.append(time.perf_counter() - t0)
    total = sum(times)
    mbs = sample.size * args.steps / total / 1e6
    desc = (f"first {sample.size} B of the {args.workload} document per step, {kind_s}, "
            f"OpenMP over buckets on {cores} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": mbs, "unit": "MB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded text generator)",
        "config": {"workload": args.workload, "sample_bytes": int(sample.size), "words_per_step": n_words},
        "words_per_s": n_words * args.steps / total,
        "cpu_baseline": {"value": mbs, "unit": "MB/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": mbs, "unit": "MB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args) -> None:
    import numpy as np
    import torch

    import paper_1407_6603_gb300 as bs
    import synth

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    else:
        torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    bs.load()
    data = synth.plain(args.workload)
    if args.prefix_bytes:
        data = data[: args.prefix_bytes]
    nbytes = int(data.size)
    d_in = torch.from_numpy(data).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(dev)
    ctx = bs.Context(profile=True, device=local_rank)
    sampler = ClockSampler(local_rank).start()

    r = None
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            r = ctx.text_device_raw(d_in, stream)
        stream.synchronize()
    n_words = int(r.n_words)
    s_bytes = int(r.stream_bytes)
    ctx.profile_read()  # drop the warm-up records
    launches0 = ctx.launch_count()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(i & 0xFF)  # evict the previous step's data from L2 (not timed)
            starts[i].record(stream)
            ctx.text_device_raw(d_in, stream)
            ends[i].record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    launches = ctx.launch_count() - launches0
    prof = ctx.profile_read()

    # end to end through the host entry point: input H2D and results D2H each step
    e2e_steps = args.e2e_steps or max(3, min(args.steps, 20))
    host = np.ascontiguousarray(data)
    ctx.text(host)
    torch.cuda.synchronize(dev)
    e2e_t = []
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        res = ctx.text(host)
        e2e_t.append(time.perf_counter() - t0)
    assert res.n_words == n_words
    clocks = sampler.stop()

    local_time = sum(step_ms) / 1e3
    max_time = reduce_max(local_time, world)
    e2e_max = reduce_max(sum(e2e_t), world)
    agg = aggregate(nbytes, n_words, args.steps, world, max_time)
    e2e_agg = aggregate(nbytes, n_words, e2e_steps, world, e2e_max)
    ctx.close()

    if rank != 0:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return

    # roofline of the dominant kernel family (largest device time in the timed region)
    fams = {k: v for k, v in prof.items() if v[0] > 0}
    dom = max(fams, key=lambda k: fams[k][1])
    launches_d, ms_d, bytes_d = fams[dom]
    peak, peak_src = measured_peaks()
    achieved = bytes_d / (ms_d / 1e3) / 1e9 if ms_d > 0 else 0.0
    traffic = recorded_traffic(dom, args.workload)
    kernels = {k: {"launches_per_step": v[0] / args.steps, "ms_per_step": v[1] / args.steps,
                   "algorithmic_bytes_per_step": v[2] / args.steps,
                   "achieved_gbs": (v[2] / (v[1] / 1e3) / 1e9) if v[1] > 0 else None}
               for k, v in fams.items()}
    # the oracle baseline runs on rank 0 at N=1 only
    cpu = cpu_baseline(data, args.workload) if (world == 1 and not args.no_cpu_baseline) else None
    step_sorted = sorted(step_ms)
    d2h = 4 * (n_words + 1) + s_bytes + 1536 + 32
    line = {
        "metric": METRIC, "value": agg["mb_per_s"], "unit": "MB/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded text generator shaped like the paper's Hamlet files)",
        "config": {"workload": args.workload + (f" (first {nbytes} B)" if args.prefix_bytes else ""),
                   "bytes": nbytes, "words": n_words, "stream_bytes": s_bytes,
                   "entry": "bsort_text_device (input resident in HBM)", "parallelism": f"replicas x{world}",
                   "l2": "flushed between timed steps by writing a 256 MiB buffer"},
        "words_per_s": agg["words_per_s"],
        "p50_ms": step_sorted[len(step_sorted) // 2],
        "p99_ms": step_sorted[min(len(step_sorted) - 1, int(round(0.99 * (len(step_sorted) - 1))))],
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if peak else None, "peak_source": peak_src,
                     "traffic": traffic, "launches_per_step": launches_d / args.steps,
                     "algorithmic_bytes_per_launch": bytes_d / launches_d if launches_d else None},
        "kernels": kernels,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_agg["mb_per_s"], "unit": "MB/s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": d2h, "entry": "bsort_text (host buffers)",
                "ms_per_step": statistics.mean(e2e_t) * 1e3},
        "clocks": clocks,
        "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def main(argv=None) -> None:
    args = parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
