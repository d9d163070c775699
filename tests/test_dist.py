"""The benchmark's multi-process path on CPU ranks (gloo, world size 2):
each rank draws its own batch (weak scaling, no data exchange) and the
timing/pixel reductions give the max and the sum over ranks."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import bench
from paper_1401_5245_gb300 import synth
rank, world, local = bench.rank_info()
dist = bench.init_dist(world, "gloo")
seed = bench.shard_seed(rank)
shapes = synth.batch_shapes(seed, 64)
pixels = float(sum(w * h for w, h in shapes))
t = 1.0 + rank                       # a per-rank "step time"
bench.barrier(dist)
out = {{"rank": rank, "seed": seed, "pixels": pixels,
        "t_max": bench.reduce_max(dist, t), "px_sum": bench.reduce_sum(dist, pixels)}}
print(json.dumps(out), flush=True)
dist.destroy_process_group()
"""


def test_two_gloo_ranks():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER.format(root=ROOT)],
                                      env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=300)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    outs.sort(key=lambda d: d["rank"])
    assert outs[0]["seed"] != outs[1]["seed"]                 # distinct batches
    assert outs[0]["pixels"] != outs[1]["pixels"]
    for d in outs:
        assert d["t_max"] == 2.0
        assert d["px_sum"] == outs[0]["pixels"] + outs[1]["pixels"]


def test_reference_arm_prints_one_line():
    """bench.py --impl reference times the CPU oracle and prints the
    contract's JSON line (no GPU needed)."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl",
                        "reference", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "Gpixel/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl",
                        "reference", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=120, cwd=ROOT, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""
