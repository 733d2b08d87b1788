"""Host-side logic of multi-GPU runs: one process per GPU, each rank solving
its own independent recovery problem (the patches of one problem are not
sharded), so the data path has no collective; the only cross-rank steps are
a barrier before the timed region and the maximum of the ranks' timed
durations after it (weak scaling: whole-job throughput = ranks x steps / the
slowest rank's time)."""
from __future__ import annotations

import os

import torch


def dist_env():
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s problem: every rank solves a different one."""
    return base + rank


def barrier(world: int) -> None:
    if world > 1:
        torch.distributed.barrier()


def job_time_ms(local_ms: float, world: int, device="cpu") -> float:
    """The slowest rank's duration (all ranks receive it)."""
    if world <= 1:
        return float(local_ms)
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, steps_per_rank: int, job_ms: float) -> float:
    """Whole-job iterations per second."""
    return world * steps_per_rank / (job_ms / 1e3)
