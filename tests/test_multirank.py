"""The bench's multi-GPU path on CPU: two gloo ranks (one process each, as
torchrun starts them) take the maximum of their timed regions and report the
whole-job throughput of N replicas; the reference arm does its work on rank 0
only.  The hot path itself has no exchange step (replicas)."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_max_time_and_whole_job_value():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import multirank_worker

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times, steps, world = [120.0, 150.0], 10, 2
    port = _free_port()
    procs = [ctx.Process(target=multirank_worker.run, args=(r, world, port, times, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == max(times)
        assert value == pytest.approx(world * steps / (max(times) * 1e-3))


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
