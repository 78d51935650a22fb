"""Multi-rank paths on CPU with two gloo ranks (one process each, as torchrun
starts them): the bench's replicas take the maximum of their timed regions and
report the whole-job throughput; the reference arm works on rank 0 only; and
the row-sharding plan (contiguous row blocks per rank, one all-reduce of the
six sums) reproduces the unsharded NLL and gradient."""
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


def test_row_sharded_nll_grad_equals_unsharded():
    pytest.importorskip("torch")
    import numpy as np
    import torch.multiprocessing as mp
    import multirank_worker
    import oracle
    import synthetic_inputs as si

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world = 2
    port = _free_port()
    procs = [ctx.Process(target=multirank_worker.shard_rows, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = si.tiny_uniform()
    th = oracle.theta_native(w.theta)
    nn, cnt, _, _ = oracle.knn(w.xy, w.t, th, w.m)
    v, g = oracle.nll_grad(w.xy, w.t, th, w.m, nn, cnt, w.z)
    const = 0.5 * w.n * np.log(2 * np.pi)
    for _, part in out:
        assert part[0] + const == pytest.approx(v, rel=1e-13)
        np.testing.assert_allclose(part[1:], g, rtol=1e-11, atol=1e-11)
