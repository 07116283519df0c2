"""The benchmark's multi-rank logic on CPU: two gloo ranks, the max-over-
ranks timing and the whole-job aggregate (no GPU, no data-path collective:
each rank sorts its own documents)."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"]); world = int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
bench.barrier(world)
t = bench.reduce_max(1.5 + rank, world)          # rank 1 is the slower one
agg = bench.aggregate(1000, 10, 4, world, t)      # 1000 B and 10 words per step, 4 steps
print(json.dumps({{"rank": rank, "max": t, "agg": agg}}))
dist.destroy_process_group()
"""


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_max_and_aggregate():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    import json

    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    res = [json.loads(o.strip().splitlines()[-1]) for o, _ in outs]
    for r in res:
        assert r["max"] == 2.5  # both ranks see the slowest rank's time
        # whole job: 2 ranks x 4 steps x 1000 B over 2.5 s
        assert r["agg"]["mb_per_s"] == pytest.approx(2 * 4 * 1000 / 2.5 / 1e6)
        assert r["agg"]["words_per_s"] == pytest.approx(2 * 4 * 10 / 2.5)


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1"], env=env, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_max(3.0, 1) == 3.0
    a = bench.parse_args([])
    assert a.gpus == 1 and a.warmup >= 3 and a.workload == "plain_256m"
