"""Host-side helpers for running independent grids on several GPUs (one process per GPU).

The hyperbolic sub-steps of independent problems (separate grids, or the members of a batch) need no exchange, so
ranks share nothing on the data path: each rank takes its own share of the problems, and the only collectives are a
barrier and a max-reduction of the elapsed time for reporting.  A single grid split across GPUs would need a halo
exchange per sub-step; that is not provided.
"""
from __future__ import annotations

import os


def env_ranks():
    """(rank, world_size, local_rank) from the launcher's environment (1 process when unset)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str, device=None) -> None:
    """Join the process group when there is more than one rank (rendezvous from MASTER_ADDR/MASTER_PORT)."""
    import torch.distributed as dist

    _, world, _ = env_ranks()
    if world > 1 and not dist.is_initialized():
        if device is not None and backend == "nccl":
            dist.init_process_group(backend, device_id=device)
        else:
            dist.init_process_group(backend)


def shard(items, rank: int, world: int):
    """This rank's share of independent problems: items rank, rank + world, ... (every item exactly once)."""
    return list(items)[rank::world]


def barrier() -> None:
    import torch.distributed as dist

    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(x: float, device=None) -> float:
    """The maximum of x over all ranks (the job's time is the slowest rank's)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_initialized() and dist.get_world_size() > 1):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def finalize() -> None:
    import torch.distributed as dist

    if dist.is_initialized():
        dist.destroy_process_group()
