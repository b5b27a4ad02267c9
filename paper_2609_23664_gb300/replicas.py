"""Multi-GPU replicas (one process per GPU, launched by torchrun).

After planning, the tasks of a workload are independent, so N GPUs run N
independent seeded workloads (weak scaling) with no collective on the data
path; the only communication is a barrier around the timed region and one
max-reduction of the step time, so the whole-job rate is
    N * tasks_per_rank / max_over_ranks(step time).
The helpers take the backend and device explicitly so the same code runs
over NCCL on GPUs and over gloo on host processes.
"""
from __future__ import annotations

import os
from typing import Tuple


def env_ranks() -> Tuple[int, int, int]:
    """(world size, rank, local rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(world: int, backend: str, device=None, init_method: str = None, rank: int = None):
    """Joins the process group when world > 1 (env:// unless init_method)."""
    if world <= 1:
        return
    import torch.distributed as dist
    kw = {}
    if device is not None:
        kw["device_id"] = device
    if init_method is not None:
        kw["init_method"] = init_method
        kw["rank"] = rank
        kw["world_size"] = world
    dist.init_process_group(backend, **kw)


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank r's workload: independent replicas of one family."""
    return base + 1000 * rank


def whole_job_rate(units_per_rank: int, world: int, step_ms_max: float) -> float:
    """Units per second of the whole job, timed by the slowest rank."""
    return world * units_per_rank / (step_ms_max / 1e3)


def finish(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
