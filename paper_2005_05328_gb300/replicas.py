"""Host-side logic of multi-GPU runs: independent replicas, no data-path
collective.

The DZS step of one lightcone mock does not shard (one mock per GPU address
space; independent mocks share nothing), so N GPUs run N independent mocks,
one process per GPU.  The only collectives are the timing barrier and the
final reduction of the work done and the slowest rank's time, which is what
these helpers do (works with NCCL on GPUs and gloo on CPU).
"""
from __future__ import annotations

import os


def rank_info():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(base_seed: int, rank: int) -> int:
    """Seed of the mock a rank runs: distinct, reproducible per rank."""
    return int(base_seed) + 1000003 * int(rank)


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def aggregate(units_local: float, seconds_local: float, device=None):
    """Sum of the units every rank processed and the maximum of the ranks'
    timed seconds (the job's wall time).  Single process: the inputs."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(units_local), float(seconds_local)
    dev = device if device is not None else torch.device("cpu")
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=dev)
    s = torch.tensor([float(seconds_local)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()), float(s.item())


def throughput(units_total: float, seconds_max: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return units_total / seconds_max if seconds_max > 0 else float("nan")
