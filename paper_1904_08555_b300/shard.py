"""Multi-GPU sharding of the hot path: one process per GPU, no data-path
collective.

Update-chain instances are independent, so rank r of W holds instances
[r * batch, (r + 1) * batch) of a larger virtual batch (weak scaling: every
rank keeps its per-GPU batch).  The only communication is a barrier around
the timed region and the maximum of the ranks' elapsed times, over whatever
process group torch.distributed was initialised with (NCCL on GPUs, gloo in
the CPU tests).
"""
from __future__ import annotations

import os


def world() -> tuple[int, int, int]:
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def first_instance(rank: int, per_rank: int) -> int:
    """Index of the rank's first instance in the virtual batch."""
    return rank * per_rank


def element_offset(rank: int, per_rank: int, n: int) -> int:
    """Canonical element index of the rank's first A entry (row-major instances)."""
    return first_instance(rank, per_rank) * n * n


def barrier(world_size: int) -> None:
    if world_size > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world_size: int, value: float, device=None) -> float:
    """The maximum of `value` over all ranks (the job's elapsed time)."""
    if world_size == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
