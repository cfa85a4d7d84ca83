"""Replica runs on one node: one process per GPU, each restoring its own images.

Images and requests are independent (the method has no exchange step between
them), so N GPUs run N replicas of the workload (weak scaling).  The only
collectives are a barrier around the timed region and the maximum over ranks
of its duration; no image data crosses ranks.
"""
from __future__ import annotations

import os


def env():
    """(rank, world_size, local_rank) from the torchrun environment (1 process if unset)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(world: int, backend: str, device=None) -> None:
    if world > 1:
        import torch.distributed as dist

        kwargs = {"device_id": device} if device is not None else {}
        dist.init_process_group(backend, **kwargs)


def finalize(world: int) -> None:
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """The largest x over all ranks (every rank receives it)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, steps: int, world: int, max_ms: float) -> float:
    """Whole-job throughput in units/s: every rank processed units_per_rank per step,
    and the job took the slowest rank's time."""
    return units_per_rank * steps * world / (max_ms / 1e3)
