"""Host-side logic of runs with one independent cavity per GPU (replicas).

Cavities never exchange data, so several GPUs run independent problems and
the only collective traffic is bookkeeping: a barrier around the timed
region and the maximum of the per-rank times.  ``torchrun`` supplies RANK,
WORLD_SIZE and LOCAL_RANK; the backend is NCCL on GPUs and gloo on CPU.
"""

from __future__ import annotations

import os


def world() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str = "nccl") -> tuple[int, int, int]:
    """Join the process group when launched with more than one rank."""
    rank, size, local = world()
    if size > 1:
        import torch.distributed as dist

        if backend == "nccl":
            import torch

            torch.cuda.set_device(local)
        if not dist.is_initialized():
            dist.init_process_group(backend)
        rank, size = dist.get_rank(), dist.get_world_size()
    return rank, size, local


def barrier(size: int) -> None:
    if size > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, size: int, device: str = "cuda") -> float:
    """The largest value of x over all ranks (every rank gets it)."""
    if size == 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, size: int, seconds: float) -> float:
    """Throughput of the whole job: every rank's units over the slowest rank's time."""
    return units_per_rank * size / seconds
