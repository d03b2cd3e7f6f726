"""The multi-rank paths of bench.py on CPU: world size 2 over gloo.

Replicas are weak-scaled: the whole-job value is the units every rank
processed over the slowest rank's time.  The reference arm (the CPU oracle)
runs on rank 0 only; other ranks exit without work.
"""
import json
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took (r + 1) * 10 ms for 1000 units
    total_ms, value = bench.aggregate(world, (rank + 1) * 10.0, 1000.0)
    q.put((rank, total_ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, total_ms, value in got:
        assert total_ms == 20.0                      # slowest rank
        assert abs(value - 2000.0 / 0.020) < 1e-6    # all units / slowest time


def run_reference(rank, world):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--gpus", str(world), "--steps", "2", "--warmup", "1",
                           "--workload", "sphere_l1"],
                          capture_output=True, text=True, env=env, timeout=600)


def test_reference_arm_rank0_prints_other_ranks_exit():
    r1 = run_reference(1, 2)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    r0 = run_reference(0, 2)
    assert r0.returncode == 0, r0.stderr
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["unit"] == "cell-interactions/s" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
