"""Host-side logic of multi-GPU runs of independent cavities.

Cavities never exchange data: several GPUs run independent problems (one
cavity per GPU, or a batch's cavities sharded across GPUs), and the only
collective traffic is bookkeeping: a barrier around the timed region, the
maximum of the per-rank times and a gather of per-cavity results.
``torchrun`` supplies RANK, WORLD_SIZE and LOCAL_RANK; the backend is NCCL on
GPUs and gloo on CPU.
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


def shard(costs, size: int) -> list[list[int]]:
    """Indices of the items each rank takes: longest-processing-time-first
    over the given per-item costs (largest first, each to the least loaded
    rank, ties to the lower rank), so the ranks' loads stay within the
    largest single cost of each other.  Deterministic; every index appears
    once."""
    loads = [0.0] * size
    out: list[list[int]] = [[] for _ in range(size)]
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        r = min(range(size), key=lambda q: (loads[q], q))
        out[r].append(i)
        loads[r] += costs[i]
    return [sorted(x) for x in out]


def gather_rows(rows: list, size: int) -> list:
    """Every rank's list of per-item rows, concatenated in rank order (every
    rank gets the whole list)."""
    if size == 1:
        return list(rows)
    import torch.distributed as dist

    parts: list = [None] * size
    dist.all_gather_object(parts, list(rows))
    return [r for p in parts for r in p]
