"""Data-parallel replicas: matrices are independent, so a batch is split across ranks with
no collective on the data path; the only collective is the timing reduction of a
benchmark (the slowest rank sets the step time).

Ranks come from the usual torch.distributed environment (RANK, WORLD_SIZE, MASTER_ADDR,
MASTER_PORT); the benchmark uses NCCL on GPUs, the tests gloo on CPU."""
from __future__ import annotations

import os


def world() -> tuple[int, int]:
    """(rank, world size) from the environment; (0, 1) outside a launcher."""
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def init(backend: str = "nccl") -> tuple[int, int]:
    """Initializes the process group when WORLD_SIZE > 1; returns (rank, world size)."""
    import torch.distributed as dist
    rank, ws = world()
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend)
    return (dist.get_rank(), dist.get_world_size()) if ws > 1 else (0, 1)


def shard(batch: int, rank: int, world_size: int) -> range:
    """Contiguous share of `batch` matrices for `rank`: the first batch % world_size ranks
    take one more, every matrix belongs to exactly one rank."""
    q, r = divmod(batch, world_size)
    start = rank * q + min(rank, r)
    return range(start, start + q + (1 if rank < r else 0))


def max_over_ranks(values, device=None):
    """Element-wise maximum over ranks of a list of floats (identity with one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()
