"""Multi-GPU execution: replicas only.

One scenario is not sharded.  With N GPUs of one node, N processes (one per
GPU, launched by torchrun) each run their own replica of the workload; the
only exchanges are a barrier around the timed region and a MAX reduction of
the timed duration, so the whole-job throughput is N x (one replica's units)
over the slowest rank's time.  The helpers work with any torch.distributed
backend: NCCL for CUDA tensors on the GPU machine, gloo for CPU tensors in tests.
"""
from __future__ import annotations

import os


def dist_env():
    """(world size, rank, local rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def slowest(value: float, device=None) -> float:
    """The largest value over the ranks of the default process group (the
    value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world_size: int, seconds: float) -> float:
    """Units processed by all ranks per second of the slowest rank."""
    return world_size * units_per_rank / seconds


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
