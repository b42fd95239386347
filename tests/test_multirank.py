"""The N > 1 paths of bench.py on CPU processes (gloo, world size 2).

The march shards by replicas: every rank renders its own copy of the
workload, so the only cross-rank steps are the timing and rate reductions
(max of the timed region, sums of rates, worst-rank latencies) and the rule
that rank 0 alone prints.  Both are exercised here without a GPU.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    got = {
        "max": bench.reduce_over_ranks(10.0 + 5.0 * rank, "max", "cpu"),
        "sum": bench.reduce_over_ranks(1.5 + rank, "sum", "cpu"),
    }
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out, f"rank{rank}.json"), "w") as f:
        json.dump(got, f)


def test_reductions_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = 29500 + (os.getpid() % 1000)
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    for rank in (0, 1):
        got = json.load(open(tmp_path / f"rank{rank}.json"))
        assert got["max"] == 15.0          # the slowest rank's timed region
        assert got["sum"] == 1.5 + 2.5     # rates add up over replicas


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(3.25, "max", "cpu") == 3.25
    assert bench.reduce_over_ranks(3.25, "sum", "cpu") == 3.25


def test_reference_arm_under_torchrun_prints_once(tmp_path):
    """Under torchrun the reference arm runs on rank 0 alone; the other rank
    exits 0 without output."""
    pytest.importorskip("torch")
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(30500 + os.getpid() % 1000),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3",
           "--scale", "0.125"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
