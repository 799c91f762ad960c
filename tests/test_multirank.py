"""The replicas path of the benchmark on two CPU ranks (gloo): the only
cross-rank steps are the barrier around each timed step and the maximum of the
per-rank times; the reference arm prints from rank 0 only."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
bench.barrier(world)
v = bench.max_over_ranks(float(10 * (rank + 1)), world)
bench.barrier(world)
with open(os.path.join(os.environ["OUT"], f"rank{rank}.json"), "w") as f:
    json.dump({"rank": rank, "world": world, "max": v}, f)
dist.destroy_process_group()
"""


def _launch(nproc, args, port, out=""):
    env = dict(os.environ, ROOT=ROOT, OMP_NUM_THREADS="1", OUT=str(out))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={nproc}",
           "--master-addr=127.0.0.1", f"--master-port={port}"] + args
    return subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=240, cwd=ROOT)


def test_two_rank_barrier_and_max(tmp_path):
    pytest.importorskip("torch")
    script = tmp_path / "worker.py"
    script.write_text(WORKER)
    r = _launch(2, [str(script)], 29611, tmp_path)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.load(open(tmp_path / f"rank{i}.json")) for i in range(2)]
    assert sorted(l["rank"] for l in lines) == [0, 1]
    assert all(l["world"] == 2 and l["max"] == 20.0 for l in lines)


def test_reference_arm_prints_from_rank_zero_only():
    """bench.py --impl reference under two ranks: one JSON line (rank 0), the
    oracle timed on a bounded sample of the 16 x 16 grid solve."""
    pytest.importorskip("torch")
    r = _launch(2, ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0", "--workload", "grid",
                    "--grid", "16", "--ref-iters", "50"], 29612)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["extrapolated"] and "EXTRAPOLATED" in d["cpu_baseline"]["sample"]
    assert d["ms_per_step"] > 0 and d["cpu_baseline"]["cores"] >= 1
