"""Multi-rank plumbing for the benchmark (one process per GPU, replicas only).

The time stepper of one model does not shard without a halo exchange, so N
ranks run N independent replicas of the same workload; there is no collective
on the data path.  The only communication is the barrier around the timed
region and the reduction of the timings: the job time is the maximum over
ranks and the work is the sum over ranks.
"""
from __future__ import annotations

import os


def world():
    """(rank, world_size, local_rank) from the torchrun environment (1 rank if absent)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str | None = None):
    """Initialise torch.distributed when WORLD_SIZE > 1; returns the module or None."""
    rank, ws, _ = world()
    if ws <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        if backend is None:
            import torch
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend, rank=rank, world_size=ws)
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def reduce_time_and_work(dist, seconds: float, units: float, device=None):
    """Job time = max over ranks, work = sum over ranks."""
    if dist is None:
        return seconds, units
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def finalize(dist):
    if dist is not None and dist.is_initialized():
        dist.destroy_process_group()
