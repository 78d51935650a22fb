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
