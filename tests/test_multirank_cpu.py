"""The benchmark's multi-rank path on CPU: world_size 2 over gloo. Each rank
reports its own timing; the job value uses the slowest rank, and ranks other
than 0 of the reference arm exit without work."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank  # rank 1 is slower
    mx = bench.max_over_ranks(local_ms, world, torch.device("cpu"))
    value = bench.aggregate_mlups(1000, 10, mx, world)
    out.put((rank, mx, value))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[1] for g in got] == [150.0, 150.0]
    # 2 ranks x 1000 nodes x 10 steps in 150 ms
    assert got[0][2] == pytest.approx(2 * 1000 * 10 / 0.150 / 1e6)


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "64",
                          "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0 and res.stdout.strip() == ""


def test_reference_arm_prints_one_line():
    import json

    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "64",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0
    lines = [ln for ln in res.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_cpu_baseline_legs_time_the_oracle():
    """The GPU arm's CPU-baseline legs: all host threads on the workload's grid, and one thread on
    a band of rows of the same flow; both positive rates, the thread count restored after."""
    sys.path.insert(0, ROOT)
    import bench
    from oracle import oracle as O

    w = bench.workload(256)
    before = O.set_threads(0)
    v, cores, sample = bench.oracle_mlups(w, "complete", target_s=0.2)
    assert v > 0 and cores >= 1 and "256x256" in sample
    v1, sample1 = bench.oracle_single_thread_mlups(w, "complete", target_s=0.2, rows=16)
    assert v1 > 0 and "256x16" in sample1
    assert O.set_threads(0) == before or O.set_threads(0) == cores
