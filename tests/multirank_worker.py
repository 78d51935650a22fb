"""Child process of test_multirank.py: one rank of a gloo job that drives the
bench's multi-rank helpers (barrier, max over ranks, whole-job value)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(rank, world, port, times, steps, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.ranks_barrier(dist)
        ms = bench.max_over_ranks(times[rank], dist, "cpu")
        bench.ranks_barrier(dist)
        q.put((rank, ms, bench.whole_job_value(world, steps, ms)))
    finally:
        dist.destroy_process_group()


def shard_rows(rank, world, port, q):
    """Row-sharded NLL + gradient: this rank's contiguous block of rows (the
    rows are independent given the neighbour sets), then one all-reduce of the
    six sums.  Evaluated with the oracle, since the ranks run on CPU."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle
    import synthetic_inputs as si
    w = si.tiny_uniform()
    th = oracle.theta_native(w.theta)
    nn, cnt, _, _ = oracle.knn(w.xy, w.t, th, w.m, threads=1)
    lo, hi = rank * w.n // world, (rank + 1) * w.n // world
    rows = np.arange(lo, hi, dtype=np.int64)
    v, g = oracle.nll_grad_rows(w.xy, w.t, th, w.m, rows, nn[lo:hi], cnt[lo:hi], w.z, threads=1)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        part = torch.tensor([v, *g], dtype=torch.float64)
        dist.all_reduce(part, op=dist.ReduceOp.SUM)
        q.put((rank, part.tolist()))
    finally:
        dist.destroy_process_group()
