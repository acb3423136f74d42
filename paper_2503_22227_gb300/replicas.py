"""Multi-GPU runs as independent replicas: one process per GPU, each with
its own context, keys and batch of ciphertexts.  The operations of the hot
path are independent per ciphertext, so nothing is exchanged on the data
path; only the timing is combined: a barrier on both sides of the timed
region, the maximum elapsed time over ranks, and throughput = all ranks'
operations / that slowest time (weak scaling)."""
from __future__ import annotations

import os


def init_from_env(backend: str | None = None) -> tuple[int, int, int]:
    """(rank, world, local rank) from the torchrun environment; creates the
    process group when world > 1 (NCCL on GPUs, gloo otherwise)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if not dist.is_initialized():
            if backend is None:
                backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend)
    return rank, world, local


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(units_per_rank: float, world: int, slowest_seconds: float) -> float:
    """Whole-job rate: every rank processed `units_per_rank` units."""
    return world * units_per_rank / slowest_seconds
