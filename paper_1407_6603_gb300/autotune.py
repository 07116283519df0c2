"""Autotuner of the sort's per-class choices.

The tile sort (K4) handles a bucket with a thread-block cluster of 1, 2, 4 or
8 CTAs depending on its size (one size class per cluster size).  Per class it
tunes the odd-even/merge cutoff: how many lanes (2, 4 or 8) run odd-even
transposition together before merge path takes over, i.e. runs of lanes x
keys-per-thread keys leave the transposition stage; and the keys per thread
(CTAs of 256 or 512 threads on the same 2048-word tile).  For the merge passes (K5)
it tunes the run length the tile sort leaves for them (clusters of 1, 2, 4 or 8
CTAs for buckets larger than one cluster of 8 tiles) and the threshold, in
tiles per resident CTA, above which a pass is pipelined (cut kernel, then
double-buffered merge).

Every candidate runs on the same seeded synthetic documents (the plain
190 KB and 1.38 MB shapes, a 32 MiB slice of the 256 MiB generator and 256
documents of the batch generator), resident on the current GPU, through the
library's device entry points.  The two choices that only large inputs meet
(the run length before pipelined merges, and the threshold that pipelines
them) are timed on the whole 256 MiB document and the 4096-document batch as
well.  The library traces each launch with CUDA
events and tags tile-sort launches with their cluster size.  Each class is
first timed alone (k4_streams=0 puts every tile sort on the call's stream),
then the per-class choice is checked against uniform ones on whole calls with
the classes side by side, as they run in production; the merge threshold is
chosen on whole calls too.  The result is a tune table
(bsort_config.tune_table); the library's built-in tuning is the one this
program chose on a GB300 (tune_table.txt beside it):

    python -m paper_1407_6603_gb300.autotune [--out FILE] [--reps N]
"""
from __future__ import annotations

import argparse
import os
import sys
import time

CLUSTERS = (1, 2, 4, 8)
LANES = (2, 4, 8)
PIPED = (1, 2, 4, 8)
RUNS = (8, 4, 2, 1)
RUNS_SMALL = (8, 16)
THREADS = ("256,256,256,256", "512,512,512,256", "512,512,512,512")
DEFAULT_OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_table.txt")


def _documents():
    """Seeded inputs with the workloads' shapes, as (name, list of uint8 arrays)."""
    import numpy as np

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import synth

    big = synth.plain("plain_256m")
    return [("plain_190k", [synth.plain("plain_190k")]), ("plain_1m38", [synth.plain("plain_1m38")]),
            ("plain_256m[:32MiB]", [np.ascontiguousarray(big[: 32 << 20])]), ("batch_256", synth.batch(256))], \
           [("plain_256m", [big]), ("batch_4096", synth.batch(4096))]


def _time(table: str, sets, reps: int) -> tuple[dict, float]:
    """Summed launch time per (family, variant) and summed call span (ms)."""
    import numpy as np
    import torch

    from . import Context

    per = {}
    span = 0.0
    with Context(profile=True, tune_table=table) as c:
        dev_sets = []
        for _, docs in sets:
            lens = [d.size for d in docs]
            offs = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.uint64).tolist()
            dev_sets.append((torch.from_numpy(np.concatenate(docs)).cuda(), offs, lens))

        def run(d, offs, lens):
            if len(lens) == 1:
                c.text_device(d)
            else:
                st, _ = c.batch_device(d, offs, lens)
                assert st == 0, c.last_error()

        for s in dev_sets:  # warm-up: buffers grown, kernels loaded
            run(*s)
        torch.cuda.synchronize()
        for _ in range(reps):
            for s in dev_sets:
                c.profile_read()
                run(*s)
                torch.cuda.synchronize()
                tl = c.trace_read()
                for fam, t0, t1, _, _, var in tl:
                    per[(fam, var)] = per.get((fam, var), 0.0) + (t1 - t0)
                span += max(r[2] for r in tl) - min(r[1] for r in tl)
    return per, span


def tune(reps: int = 5, log=print) -> str:
    import torch

    sets, large = _documents()
    # 1. each class timed alone (its tile sorts on the call's stream, one
    #    launch after another), for every lane count
    class_ms = {}
    for g in LANES:
        per, _ = _time(f"k4_lanes={g},{g},{g},{g} k4_streams=0", sets, reps)
        for cl in CLUSTERS:
            class_ms[(cl, g)] = per.get(("tile_sort", cl), 0.0) / reps
            log(f"  tile sort, clusters of {cl}, {g} lanes: {class_ms[(cl, g)]:9.3f} ms per round")
    best = ",".join(str(min(LANES, key=lambda g: (class_ms[(cl, g)], abs(g - 4)))) for cl in CLUSTERS)
    # 2. the per-class choice against uniform ones, on whole calls with the
    #    classes running side by side as in production
    span_of = {}
    for lanes in dict.fromkeys([best, "4,4,4,4", "2,2,2,2", "8,8,8,8"]):
        _, span = _time(f"k4_lanes={lanes}", sets, reps)
        span_of[lanes] = span / reps
        log(f"  lanes {lanes}: {span_of[lanes]:9.3f} ms per round (whole calls)")
    lanes = min(span_of, key=lambda k: (span_of[k], k != best))
    # 2b. keys per thread: tile-sort CTAs of 256 threads (8 / W keys each) or
    #     512 (4 / W), per class, on whole calls
    threads_of = {}
    for th in THREADS:
        _, span = _time(f"k4_lanes={lanes} k4_threads={th}", sets, reps)
        threads_of[th] = span / reps
        log(f"  tile-sort CTA sizes {th}: {threads_of[th]:9.3f} ms per round (whole calls)")
    threads = min(threads_of, key=lambda k: (threads_of[k], k != THREADS[0]))
    # 3. the runs the tile sort leaves for the merge passes (clusters of
    #    k4_runs CTAs) for buckets larger than one cluster of 8 tiles
    runs_of = {}
    for r in RUNS:
        _, span = _time(f"k4_lanes={lanes} k4_threads={threads} k4_runs={r}", sets + large, reps)
        runs_of[r] = span / reps
        log(f"  runs of {r} tiles before the merge passes: {runs_of[r]:9.3f} ms per round (whole calls)")
    runs = min(RUNS, key=lambda r: (runs_of[r], -r))
    # 3b. the run length when the merges are too small to pipeline
    small_of = {}
    for r in RUNS_SMALL:
        _, span = _time(f"k4_lanes={lanes} k4_threads={threads} k4_runs={runs} k4_runs_small={r}", sets, reps)
        small_of[r] = span / reps
        log(f"  runs of {r} tiles before small merges: {small_of[r]:9.3f} ms per round (whole calls)")
    runs_small = min(RUNS_SMALL, key=lambda r: (small_of[r], r))
    # 4. the merge threshold
    piped_of = {}
    for p in PIPED:
        _, span = _time(f"k4_lanes={lanes} k4_threads={threads} k4_runs={runs} k4_runs_small={runs_small} "
                        f"piped_min={p}", sets + large, reps)
        piped_of[p] = span / reps
        log(f"  merge threshold {p} tiles per CTA: {piped_of[p]:9.3f} ms per round (whole calls)")
    piped = min(PIPED, key=lambda p: (piped_of[p], p))
    gpu = torch.cuda.get_device_name()
    lines = [f"# tuned on {gpu}, {time.strftime('%Y-%m-%d')}, {reps} rounds over "
             + ", ".join(n for n, _ in sets) + " (run length and merge threshold: also " + ", ".join(n for n, _ in large) + ")",
             "# tile sort per class alone (clusters of 1, 2, 4, 8 CTAs), ms per round:"]
    for cl in CLUSTERS:
        lines.append("#   clusters of %d: " % cl + "  ".join(f"{g} lanes {class_ms[(cl, g)]:.3f}" for g in LANES))
    lines.append("# whole calls, ms per round: " + "  ".join(f"lanes {k}: {v:.3f}" for k, v in span_of.items()))
    lines.append("# runs before the merge passes, whole calls, ms per round: "
                 + "  ".join(f"{r}: {v:.3f}" for r, v in runs_of.items()))
    lines.append("# merge threshold, whole calls, ms per round: "
                 + "  ".join(f"{p}: {v:.3f}" for p, v in piped_of.items()))
    lines.append("# tile-sort CTA sizes, whole calls, ms per round: "
                 + "  ".join(f"{k}: {v:.3f}" for k, v in threads_of.items()))
    lines.append(f"k4_lanes={lanes}")
    lines.append(f"k4_threads={threads}")
    lines.append("# runs before small merges, whole calls, ms per round: "
                 + "  ".join(f"{r}: {v:.3f}" for r, v in small_of.items()))
    lines.append(f"k4_runs={runs}")
    lines.append(f"k4_runs_small={runs_small}")
    lines.append(f"piped_min={piped}")
    return "\n".join(lines) + "\n"


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", default=DEFAULT_OUT, help="where to write the tune table")
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args(argv)
    table = tune(args.reps)
    with open(args.out, "w") as f:
        f.write(table)
    print(table, end="")


if __name__ == "__main__":
    main()
