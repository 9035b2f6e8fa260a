"""Replica orchestration for a run on several GPUs of one node.

A relit frame does not shard: every GPU renders its own frames of the same
workload with its own scene copy and workspace, and no collective touches
the data path.  What the ranks share is bookkeeping, done on the host:
which views each rank renders, a barrier around the timed region, and the
slowest rank's elapsed time, from which the whole-job rate is
(all ranks' units) / (slowest rank's time).  The process group is the
caller's (NCCL under torchrun on GPUs, gloo in the CPU tests).
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def rank_env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the torchrun environment, (1, 0, 0) without it."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def view_index(step: int, rank: int, world: int, offset: int = 0, nviews: int = 100) -> int:
    """The view a rank renders at a step: ranks interleave over the views, so
    their views are disjoint while steps * world <= nviews (and with one rank
    the views are offset, offset + 1, ...)."""
    return (offset + rank + world * step) % nviews


def _active() -> bool:
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def max_over_ranks(x: float, device=None) -> float:
    """The largest of every rank's x (x itself with one process)."""
    if not _active():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier() -> None:
    if _active():
        dist.barrier()


def whole_job_rate(units_per_rank: float, slowest_seconds: float, world: int) -> float:
    """Units per second of the whole job: every rank's units over the slowest rank's time."""
    return world * units_per_rank / slowest_seconds
