#!/usr/bin/env python3
"""Benchmark of the length-bucketed word sort on GB300.

One step = the whole path (strip, bucket by length, sort every bucket, emit)
over one synthetic document resident in HBM, through the C ABI's device entry
point.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Workloads (seeded synthetic text shaped like the paper's Hamlet files, which
are not available here): plain_256m (default, 268,435,456 B, the largest single
document), plain_1m38 (1,447,000 B), plain_190k (194,560 B), batch_4096 (4,096
documents, 2.07 GB) and serve (the request stream).  The default run adds the
other forms beside the headline line under "forms": the 1.4 MB document, the
whole 4,096-document batch, and the request stream at its configured rate and
at saturation.

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
# Integer issue rate behind the tile sort's roofline: 4 x 32 integer lanes per
# SM per clock, and 4 integer operations per key-level of one-word keys (a
# 64-bit compare is 2, a 64-bit select 2).
ALU_LANES_PER_SM = 128
ALU_OPS_PER_KEY_LEVEL = 4
FALLBACK_HBM_GBS = 6800.0

# Kernel families and the source file that holds each (for the traffic record).
KERNEL_SOURCE = {
    "tokenize": "k_tokenize1p.cu", "scatter": "k_scatter.cu", "emit": "k_scatter.cu",
    "tile_sort": "k_sort2.cu", "merge_pass": "k_sort2.cu", "merge_cut": "k_sort2.cu", "expand": "k_dedupe.cu",
    "dedupe": "k_dedupe_hash.cu", "layout": "k_layout.cu",
}


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="plain_256m",
                   choices=["plain_190k", "plain_1m38", "plain_256m", "batch_4096", "serve"])
    p.add_argument("--duration", type=float, default=10.0, help="seconds of Poisson arrivals (serve)")
    p.add_argument("--pool", type=int, default=1024, help="distinct documents the serve stream cycles through")
    p.add_argument("--rate", type=float, default=None, help="serve: arrivals per second (default: the workload's)")
    p.add_argument("--saturation-s", type=float, default=5.0,
                   help="serve: seconds of the closed-loop run at capacity (0: none)")
    p.add_argument("--batch-docs", type=int, default=None, help="use only the first D documents of batch_4096")
    p.add_argument("--e2e-steps", type=int, default=None)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sweep", action="store_true", help="only the oracle's thread sweep (Table 4 style), then exit")
    p.add_argument("--tune", default=None, help="tune table text (bsort_config.tune_table); default: built-in")
    p.add_argument("--no-forms", action="store_true", help="skip the batched-form summary of the default run")
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
    """sha256 (16 hex digits) of the family's .cu file and every shared header."""
    csrc = os.path.join(ROOT, "paper_1407_6603_gb300", "csrc")
    h = hashlib.sha256()
    files = [KERNEL_SOURCE.get(family, "bsort_api.cu")] + sorted(f for f in os.listdir(csrc) if f.endswith(".cuh"))
    for f in files:
        with open(os.path.join(csrc, f), "rb") as fh:
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


def run_cpu_sweep(args) -> None:
    """The paper's Table 4 measurement on this host: O1 (bubble sort per
    length bucket, OpenMP over buckets) on the two paper-sized documents with
    1, 2, 4, ... threads up to the core count; speedup S = T1 / Tp and
    efficiency E = S / p.  Median of three runs for plain_190k, one for
    plain_1m38 (whose single-thread run takes about a minute)."""
    import oracle
    import synth

    cores = os.cpu_count() or 1
    threads = []
    p = 1
    while p < cores:
        threads.append(p)
        p *= 2
    threads.append(cores)
    out = {"metric": "oracle thread sweep (Table 4 style)", "cores": cores, "documents": {}}
    for wl, reps in (("plain_190k", 3), ("plain_1m38", 1)):
        data = synth.plain(wl)
        rows = []
        for p in threads:
            ts = []
            for _ in range(reps):
                t0 = time.perf_counter()
                oracle.bubble(data, nthreads=p)
                ts.append(time.perf_counter() - t0)
            rows.append({"threads": p, "seconds": statistics.median(ts)})
        t1 = rows[0]["seconds"]
        for r in rows:
            r["speedup"] = t1 / r["seconds"]
            r["efficiency"] = r["speedup"] / r["threads"]
        out["documents"][wl] = rows
    print(json.dumps(out), flush=True)


def run_reference(args) -> None:
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle
    import synth

    cores = os.cpu_count() or 1
    if args.workload == "batch_4096":
        # documents of the batch, concatenated up to 16 MiB, each sorted on its own
        docs = synth.batch(64, threads=cores)
        picked, size = [], 0
        for d in docs:
            if size + d.size > (16 << 20) and picked:
                break
            picked.append(d)
            size += d.size

        def batch_fn(_sample, nthreads):
            return {"n_words": sum(oracle.stable(d, nthreads=nthreads)["n_words"] for d in picked)}

        import numpy as np

        sample = np.concatenate(picked)
        fn, kind_s = batch_fn, f"O2 stable_sort per length bucket on {len(picked)} batch documents"
    elif args.workload == "plain_256m":
        data = synth.plain(args.workload)
        sample = data[: 16 << 20]
        fn, kind_s = oracle.stable, "O2 stable_sort per length bucket"
    else:
        data = synth.plain(args.workload)
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


def load_workload(args):
    """The workload's documents on the host: one document, or the batch."""
    import numpy as np

    import synth

    if args.workload == "batch_4096":
        docs = synth.batch(args.batch_docs, threads=os.cpu_count() or 8)
        lens = [int(d.size) for d in docs]
        offs = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64).tolist()
        return docs, offs, lens, np.concatenate(docs)
    data = synth.plain(args.workload)
    if args.prefix_bytes:
        data = data[: args.prefix_bytes]
    return [data], [0], [int(data.size)], data


def cpu_baseline_batch(docs) -> dict:
    """The oracle's stable_sort path (OpenMP over buckets) over the batch's
    documents one by one, for about ten seconds (a bounded sample)."""
    import oracle

    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    nb = nw = nd = 0
    for d in docs:
        nw += oracle.stable(d, nthreads=cores)["n_words"]
        nb += d.size
        nd += 1
        if time.perf_counter() - t0 > 10.0:
            break
    dt = time.perf_counter() - t0
    return {"value": nb / dt / 1e6, "unit": "MB/s", "cores": cores, "kind": "oracle",
            "sample": f"first {nd} of {len(docs)} batch documents ({nb} B, {nw} words), O2 stable_sort per length "
                      f"bucket, OpenMP over buckets on {cores} threads, {dt:.2f} s",
            "words_per_s": nw / dt}


FORM_KEYS = ("value", "unit", "words_per_s", "ms_per_step", "p50_ms", "p99_ms", "steps", "warmup", "config",
             "roofline", "roofline_hbm", "path_roofline", "cpu_baseline", "e2e", "plain_per_doc", "gpu_launches",
             "clocks")


def run_ours(args) -> None:
    line = measure(args)
    if line is None:
        return
    if args.workload == "plain_256m" and not args.no_forms and not args.prefix_bytes and line["n_gpus"] == 1:
        # the other forms beside the headline, on the same GPU: the paper-sized
        # document, the whole batch (batched against one call per document) and
        # the request stream (at its rate, then at capacity)
        import torch

        forms = {}
        for name, argv in (("plain_1m38", ["--workload", "plain_1m38", "--steps", "50", "--warmup", "5",
                                           "--no-cpu-baseline"]),
                           ("batch_4096", ["--workload", "batch_4096", "--steps", "5", "--warmup", "3",
                                           "--e2e-steps", "3"])):
            torch.cuda.empty_cache()
            try:
                f = measure(parse_args(argv), quiet=True)
                forms[name] = {k: f[k] for k in FORM_KEYS if k in f}
            except Exception as e:  # the headline line stands on its own
                forms[name] = {"error": repr(e)[:300]}
        torch.cuda.empty_cache()
        try:
            forms["serve"] = serve_measure(parse_args(["--workload", "serve", "--duration", "5", "--pool", "512"]))
        except Exception as e:
            forms["serve"] = {"error": repr(e)[:300]}
        line["forms"] = forms
    print(json.dumps(line), flush=True)


def measure(args, quiet: bool = False):
    import numpy as np
    import torch

    import paper_1407_6603_gb300 as bs

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist

        if not dist.is_initialized():
            dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    dev = torch.device("cuda", local_rank)
    bs.load()
    batch = args.workload == "batch_4096"
    docs, offs, lens, host = load_workload(args)
    nbytes = int(host.size)
    d_in = torch.from_numpy(host).to(dev)
    flush = None if batch else torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(dev)
    ctx = bs.Context(profile=True, device=local_rank, tune_table=args.tune)
    sampler = ClockSampler(local_rank).start()

    def step():
        if batch:
            st, rs = ctx.batch_device_raw(d_in, offs, lens, stream)
            assert st == 0, ctx.last_error()
            return sum(int(r.n_words) for r in rs), sum(int(r.stream_bytes) for r in rs)
        r = ctx.text_device_raw(d_in, stream)
        return int(r.n_words), int(r.stream_bytes)

    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            n_words, s_bytes = step()
        stream.synchronize()
    ctx.profile_read()  # drop the warm-up records
    launches0 = ctx.launch_count()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            if flush is not None:
                flush.fill_(i & 0xFF)  # evict the previous step's data from L2 (not timed)
            starts[i].record(stream)
            step()
            ends[i].record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    launches = ctx.launch_count() - launches0
    # wall time per family: the union of its launches' intervals (launches of
    # one family can overlap on the side streams, which a sum would count twice)
    # ... and the part of it on the call's own stream (stream 0 of the trace):
    # launches on the side streams run beside those and are joined at the end,
    # so the call's stream holds the step's critical path
    wall, critical = {}, {}
    tl = ctx.trace_read()
    groups = {fam: (fam,) for fam in {r[0] for r in tl}}
    groups["merge_phase"] = ("merge_pass", "merge_cut")  # the merge passes with their cut kernels

    def union_ms(iv):
        tot, cur_s, cur_e = 0.0, None, None
        for a, b in sorted(iv):
            if cur_e is None or a > cur_e:
                if cur_e is not None:
                    tot += cur_e - cur_s
                cur_s, cur_e = a, b
            else:
                cur_e = max(cur_e, b)
        return tot + ((cur_e - cur_s) if cur_e is not None else 0.0)

    for fam, members in groups.items():
        wall[fam] = union_ms([(r[1], r[2]) for r in tl if r[0] in members])
        critical[fam] = union_ms([(r[1], r[2]) for r in tl if r[0] in members and r[4] == 0])
    prof = ctx.profile_read()

    # the same documents one call each, for the batched-versus-plain comparison
    plain_per_doc = None
    if batch:
        with torch.cuda.stream(stream):
            for _ in range(2):
                t_a = torch.cuda.Event(enable_timing=True)
                t_b = torch.cuda.Event(enable_timing=True)
                t_a.record(stream)
                for o, ln in zip(offs, lens):
                    ctx.text_device_raw(d_in[o:o + ln], stream)
                t_b.record(stream)
            torch.cuda.synchronize(dev)
        pd_s = t_a.elapsed_time(t_b) / 1e3
        plain_per_doc = {"words_per_s": n_words / pd_s, "mb_per_s": nbytes / pd_s / 1e6,
                         "ms_per_pass": pd_s * 1e3, "calls": len(docs), "entry": "bsort_text_device per document"}

    # end to end through the host entry points: input H2D and results D2H each step
    e2e_steps = args.e2e_steps or (max(3, min(args.steps, 20)) if not batch else 3)

    # the inputs sit in page-locked host memory (copied there once, outside
    # the timed region), which the copy engine reads in place; the results are
    # read as views of the context's page-locked output buffers
    if batch:
        docs_pinned = bs.pack_host(docs)
    else:
        host_pinned = bs.pinned_empty(host.size)
        host_pinned[:] = host

    def host_step():
        if batch:
            st, rs = ctx.batch(docs_pinned, copy=False)
            assert st == 0
            return sum(r.n_words for r in rs)
        return ctx.text(host_pinned, copy=False).n_words

    host_step()
    torch.cuda.synchronize(dev)
    e2e_t = []
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        nw_host = host_step()
        e2e_t.append(time.perf_counter() - t0)
    assert nw_host == n_words
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
        return None

    # roofline of the dominant kernel family: the largest time on the step's
    # critical path, the call's own stream (a family whose launches run on
    # side streams beside others' is stretched there by the sharing, and
    # summed launch times would count overlaps twice); then the largest wall
    # time, for families with no launch on the call's stream
    fams = {k: v for k, v in prof.items() if v[0] > 0}
    # host_gap (the call's round trips) is reported but is no kernel
    dom = max((k for k in fams if k != "host_gap"),
              key=lambda k: (critical.get(k, 0.0), wall.get(k) or fams[k][1]))
    peak, peak_src = measured_peaks()

    def hbm_roofline(fam):
        n_l, ms_f, bytes_f, _ = fams[fam]
        ach = bytes_f / (ms_f / 1e3) / 1e9 if ms_f > 0 else 0.0
        out = {"bound": "hbm", "kernel": fam, "achieved": ach, "peak": peak, "unit": "GB/s",
               "frac": ach / peak if peak else None, "peak_source": peak_src,
               "traffic": recorded_traffic(fam, args.workload), "launches_per_step": n_l / args.steps,
               "algorithmic_bytes_per_launch": bytes_f / n_l if n_l else None}
        if fam == "merge_pass" and wall.get("merge_phase"):
            # the passes of the key widths run side by side: bytes over the
            # wall time of the whole merge phase, cut kernels included
            ach_w = bytes_f / (wall["merge_phase"] / 1e3) / 1e9
            out["achieved_wall"] = ach_w
            out["frac_wall"] = ach_w / peak if peak else None
        return out

    def alu_roofline(fam):
        # the tile sort is bound by integer compares, not by HBM: key-levels
        # per second against the integer issue rate of the SMs
        n_l, ms_f, bytes_f, levels_f = fams[fam]
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
        alu_peak = sms * ALU_LANES_PER_SM * mhz * 1e6 / ALU_OPS_PER_KEY_LEVEL / 1e9
        ach = levels_f / (ms_f / 1e3) / 1e9 if ms_f > 0 else 0.0
        return {"bound": "alu", "kernel": fam, "achieved": ach, "peak": alu_peak, "unit": "G key-levels/s",
                "frac": ach / alu_peak, "peak_source": (f"derived: {sms} SMs x {ALU_LANES_PER_SM} integer lanes x "
                                                        f"{mhz:.0f} MHz / {ALU_OPS_PER_KEY_LEVEL} integer ops per "
                                                        "key-level (one-word keys)"),
                "traffic": recorded_traffic(fam, args.workload), "launches_per_step": n_l / args.steps,
                "key_levels_per_launch": levels_f / n_l if n_l else None,
                "algorithmic_bytes_per_launch": bytes_f / n_l if n_l else None}

    roofline = alu_roofline(dom) if fams[dom][3] > 0 else hbm_roofline(dom)
    hbm_fams = [k for k in fams if k != "host_gap" and fams[k][3] == 0 and fams[k][2] > 0]
    roofline_hbm = hbm_roofline(max(hbm_fams, key=lambda k: fams[k][1])) if hbm_fams else None
    kernels = {k: {"launches_per_step": v[0] / args.steps, "ms_per_step": v[1] / args.steps,
                   "wall_ms_per_step": wall.get(k, 0.0) / args.steps,
                   "critical_ms_per_step": critical.get(k, 0.0) / args.steps,
                   "algorithmic_bytes_per_step": v[2] / args.steps,
                   "achieved_gbs": (v[2] / (v[1] / 1e3) / 1e9) if v[1] > 0 else None,
                   "achieved_gbs_wall": (v[2] / (wall[k] / 1e3) / 1e9) if wall.get(k, 0.0) > 0 else None,
                   **({"key_levels_per_step": v[3] / args.steps,
                       "achieved_g_key_levels_s": v[3] / (v[1] / 1e3) / 1e9 if v[1] > 0 else None}
                      if v[3] > 0 else {})}
               for k, v in fams.items()}
    # the oracle baseline runs on rank 0 at N=1 only
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_batch(docs) if batch else cpu_baseline(host, args.workload)
    step_sorted = sorted(step_ms)
    path_min = nbytes + s_bytes + 4 * (n_words + len(docs)) + 8 * 256 * len(docs)
    d2h = 4 * (n_words + len(docs)) + s_bytes + 1536 * len(docs) + 32
    wl = args.workload + (f" (first {nbytes} B)" if args.prefix_bytes else "")
    if batch and args.batch_docs:
        wl += f" (first {len(docs)} documents)"
    line = {
        "metric": METRIC, "value": agg["mb_per_s"], "unit": "MB/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded text generator shaped like the paper's Hamlet files)",
        "config": {"workload": wl, "documents": len(docs), "bytes": nbytes, "words": n_words,
                   "stream_bytes": s_bytes,
                   "entry": ("bsort_batch_device (documents packed in one HBM buffer)" if batch
                             else "bsort_text_device (input resident in HBM)"),
                   "parallelism": f"replicas x{world}",
                   "l2": ("inputs larger than L2 (no flush)" if batch
                          else "flushed between timed steps by writing a 256 MiB buffer")},
        "words_per_s": agg["words_per_s"],
        "p50_ms": step_sorted[len(step_sorted) // 2],
        "p99_ms": step_sorted[min(len(step_sorted) - 1, int(round(0.99 * (len(step_sorted) - 1))))],
        "roofline": roofline,
        "roofline_hbm": roofline_hbm,
        # the whole step against the least any implementation must move: read
        # the input, write the sorted letters, the offsets and the counts
        "path_roofline": {"bound": "hbm", "min_bytes_per_step": path_min,
                          "achieved": path_min / (statistics.mean(step_ms) / 1e3) / 1e9, "peak": peak,
                          "unit": "GB/s", "frac": path_min / (statistics.mean(step_ms) / 1e3) / 1e9 / peak},
        "kernels": kernels,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_agg["mb_per_s"], "unit": "MB/s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": d2h, "entry": ("bsort_batch (documents packed in page-locked host memory)" if batch
                          else "bsort_text (page-locked host input)"),
                "ms_per_step": statistics.mean(e2e_t) * 1e3},
        "clocks": clocks,
        "gpu_launches": launches,
    }
    if plain_per_doc is not None:
        plain_per_doc["batched_over_plain_words"] = agg["words_per_s"] / world / plain_per_doc["words_per_s"]
        line["plain_per_doc"] = plain_per_doc
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return line


def fast_digest(*arrays) -> tuple:
    """CRC-32 and length of each array's bytes: cheap enough to check every
    served result (zlib releases the GIL, so a thread pool keeps up), and
    any changed, moved or missing byte changes it except with probability
    about 2^-32 per result."""
    import zlib

    import numpy as np

    out = []
    for a in arrays:
        b = np.ascontiguousarray(a).view(np.uint8).reshape(-1)
        out.append((int(b.size), zlib.crc32(b)))
    return tuple(out)


def serve_measure(args) -> dict | None:
    """The request stream: Poisson arrivals (2,000 documents/s by default),
    each document log-uniform in [1 KiB, 16 MiB] (a pool of distinct
    documents cycled through), submitted as they arrive to the
    continuous-batching server and polled back; p50/p99 of submit-to-result
    latency and the served rate.  Then the same server at capacity (a closed
    loop that keeps the queue full), beside the plain path (one bsort_text
    call per document) on the same documents.  Every served result is checked
    against the oracle's result for its document."""
    import threading
    from concurrent.futures import ThreadPoolExecutor

    import numpy as np
    import torch

    import oracle
    import paper_1407_6603_gb300 as bs
    import synth

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if rank != 0:
        return None  # the request stream runs on one GPU
    bs.load()
    cores = os.cpu_count() or 8
    with ThreadPoolExecutor(cores) as ex:
        pool = list(ex.map(synth.serve_doc, range(args.pool)))

    def oracle_digest(d):
        r = oracle.stable(d, nthreads=1)
        return fast_digest(r["counts"].astype(np.uint64), r["offsets"].astype(np.uint32), r["stream"])

    with ThreadPoolExecutor(cores) as ex:
        expect = list(ex.map(oracle_digest, pool))
    rate = args.rate or synth.SERVE["rate"]
    # the requests' documents in page-locked memory, submitted without a copy
    # (bsort_submit_borrowed: the copy engine reads them in place), as the
    # plain path below reads them
    pinned_pool = bs.pack_host(pool)
    # two workers for the arrival run (each batch has the GPU mostly to
    # itself: the lower tail latency), four for the capacity run (more
    # batches overlap: the higher throughput)
    workers, workers_sat, max_batch = 2, 4, 256
    ctx = bs.Context(device=local_rank)
    ctx.serve_start(hbm_budget=64 << 30, workers=workers, max_batch_docs=max_batch)
    checker = ThreadPoolExecutor(max(2, cores // 2))

    def check(tag, res, every=1):
        # (res views the server's buffers: released once its digest is taken;
        # at capacity only every `every`-th result is digested, so that the
        # checking threads do not bound the rate they measure)
        if tag % every:
            ctx.release(res)
            return None
        ok = fast_digest(res.counts, res.offsets, res.stream) == expect[tag % len(pool)]
        ctx.release(res)
        return ok

    # warm-up: every pool document once (not timed), checked like the rest
    warm = []

    def warm_up():
        for i, d in enumerate(pinned_pool):
            assert ctx.submit(d, i, borrow=True) == 0
        got = 0
        while got < len(pool):
            for tag, res, _ in ctx.poll(256, copy=False):
                warm.append(checker.submit(check, tag, res))
                got += 1
            time.sleep(0.001)

    warm_up()

    def stream_run(n_req, t_arr, max_outstanding, producers=1, every=1):
        """Submits n_req requests (at the arrival times t_arr from one thread,
        or, when t_arr is None, from `producers` threads as fast as the
        outstanding bound allows) and collects them; every `every`-th result
        is checked."""
        lat, words, nbytes, lag, futs = [], [0], [0], [], []
        done = threading.Event()
        got_n = [0]

        def consumer():
            while got_n[0] < n_req:
                for tag, res, ns in ctx.poll(256, copy=False):
                    got_n[0] += 1
                    lat.append(ns / 1e6)
                    words[0] += res.n_words
                    futs.append(checker.submit(check, tag, res, every))
                time.sleep(0.0002)
            done.set()

        th = threading.Thread(target=consumer)
        t0 = time.perf_counter()
        th.start()
        if t_arr is not None:
            for i in range(n_req):
                wait = t0 + t_arr[i] - time.perf_counter()
                if wait > 0:
                    time.sleep(wait)
                else:
                    lag.append(-wait)
                d = pinned_pool[i % len(pool)]
                nbytes[0] += d.size
                assert ctx.submit(d, i, borrow=True) == 0
        else:
            def produce(k):
                for i in range(k, n_req, producers):
                    while i - got_n[0] >= max_outstanding:
                        time.sleep(0.0001)
                    assert ctx.submit(pinned_pool[i % len(pool)], i, borrow=True) == 0

            nbytes[0] = sum(pool[i % len(pool)].size for i in range(n_req))
            prods = [threading.Thread(target=produce, args=(k,)) for k in range(producers)]
            for p in prods:
                p.start()
            for p in prods:
                p.join()
        t_submit_end = time.perf_counter()
        done.wait()
        t1 = time.perf_counter()
        th.join()
        checked = [f.result() for f in futs]
        ok = sum(1 for v in checked if v)
        n_checked = sum(1 for v in checked if v is not None)
        lat_sorted = sorted(lat)
        wall = t1 - t0
        return {"requests": n_req, "mb_per_s": nbytes[0] / wall / 1e6, "words_per_s": words[0] / wall,
                "p50_ms": lat_sorted[len(lat_sorted) // 2],
                "p99_ms": lat_sorted[min(len(lat_sorted) - 1, int(round(0.99 * (len(lat_sorted) - 1))))],
                "offered_mb_per_s": nbytes[0] / (t_submit_end - t0) / 1e6,
                "submit_lag_ms_max": max(lag) * 1e3 if lag else 0.0, "wall_s": wall,
                "checked": n_checked, "mismatched": n_checked - ok}

    sampler = ClockSampler(local_rank).start()
    n_req = int(rate * args.duration)
    # an untimed third of the arrival run first: the workers' buffers grow to
    # their working sizes there (the first run of a server measured at most
    # half its steady rate, and a p99 several times higher)
    n_pre = max(1, n_req // 3)
    pre_rate = stream_run(n_pre, synth.arrivals(n_pre, rate=rate), None)
    at_rate = stream_run(n_req, synth.arrivals(n_req, rate=rate), None)
    clocks = sampler.stop()
    sat = pre_sat = None
    if args.saturation_s > 0:
        # capacity: as many requests as the arrival run served per second,
        # scaled to the saturation time, with the queue kept full
        n_sat = max(len(pool), int(at_rate["requests"] / at_rate["wall_s"] * args.saturation_s))
        ctx.serve_stop()
        ctx.serve_start(hbm_budget=64 << 30, workers=workers_sat, max_batch_docs=max_batch)
        warm_up()
        pre_sat = stream_run(max(1, n_sat // 2), None, 4 * workers_sat * max_batch, every=4)  # untimed, as above
        sat = stream_run(n_sat, None, 4 * workers_sat * max_batch, every=4)
        sat["producers"] = 1
        sat["workers"] = workers_sat
        sat["checked_sample"] = "every 4th result digested and compared with the oracle's (all of the arrival run)"
    ctx.serve_stop()
    warm_bad = sum(1 for f in warm if not f.result())
    n_warm = len(warm)
    ctx.close()
    # the plain per-document path on the same documents: one bsort_text call
    # each (host in, host out, as the server's results), for a few seconds
    plain = None
    with bs.Context(device=local_rank) as pc:
        pinned = pinned_pool
        pc.text(pinned[0], copy=False)
        t0 = time.perf_counter()
        nw = nb = calls = 0
        while time.perf_counter() - t0 < 3.0:
            d = pinned[calls % len(pinned)]
            nw += pc.text(d, copy=False).n_words
            nb += d.size
            calls += 1
        dt = time.perf_counter() - t0
        plain = {"words_per_s": nw / dt, "mb_per_s": nb / dt / 1e6, "calls": calls, "entry": "bsort_text per document"}
    checker.shutdown()
    runs = [r for r in (pre_rate, at_rate, pre_sat, sat) if r]
    checked = n_warm + sum(r["checked"] for r in runs)
    mismatched = warm_bad + sum(r["mismatched"] for r in runs)
    return {
        "metric": METRIC, "value": at_rate["mb_per_s"], "unit": "MB/s", "n_gpus": 1, "steps": n_req,
        "warmup": len(pool), "ms_per_step": at_rate["wall_s"] / max(n_req, 1) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic (seeded text generator)",
        "config": {"workload": "serve", "requests": n_req, "arrival_rate_per_s": rate, "duration_s": args.duration,
                   "distinct_documents": len(pool), "entry": "bsort_submit_borrowed (page-locked documents) / bsort_poll (views, released)", "workers": workers,
                   "max_batch_docs": max_batch, "hbm_budget_bytes": 64 << 30},
        "words_per_s": at_rate["words_per_s"], "p50_ms": at_rate["p50_ms"], "p99_ms": at_rate["p99_ms"],
        "offered_mb_per_s": at_rate["offered_mb_per_s"], "submit_lag_ms_max": at_rate["submit_lag_ms_max"],
        "saturation": sat, "plain_per_doc": plain,
        "served_over_plain_words": (sat["words_per_s"] / plain["words_per_s"]) if sat and plain else None,
        "results_checked_against_oracle": checked, "results_mismatched": mismatched,
        "requests_total": n_warm + sum(r["requests"] for r in runs),
        "clocks": clocks,
    }


def run_serve(args) -> None:
    line = serve_measure(args)
    if line is not None:
        print(json.dumps(line), flush=True)


def main(argv=None) -> None:
    args = parse_args(argv)
    if args.cpu_sweep:
        run_cpu_sweep(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
