"""Multi-GPU layout of the work: one process per GPU, launched by torchrun.

A single film is one Markov chain whose colour passes are separated by a barrier, so it does not
shard across GPUs: N GPUs run N independent replicas of it (each rank its own seed).  Batched and
served films are independent problems: they are dealt out across ranks, so each rank advances
its own share with no collective on the data path (weak scaling).  The only collectives are the
timing ones: a barrier before and after the timed region and a max over ranks of the elapsed
time.
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass
class Ranks:
    rank: int
    world: int
    local: int

    @property
    def is_root(self) -> bool:
        return self.rank == 0


def env_ranks() -> Ranks:
    return Ranks(int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
                 int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str) -> Ranks:
    """Join the process group named by the torchrun environment (127.0.0.1 rendezvous)."""
    r = env_ranks()
    if r.world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        if not dist.is_initialized():
            dist.init_process_group(backend, rank=r.rank, world_size=r.world)
    return r


def replica_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s replica of a film: distinct per rank, rank 0 keeps the base seed."""
    return int(base) + 1000003 * int(rank)


def shard(n_items: int, rank: int, world: int) -> list[int]:
    """Indices of the independent films rank `rank` runs: round-robin over the list, so that a
    list sorted by size spreads large and small films evenly."""
    return list(range(rank, n_items, world))


def barrier(r: Ranks):
    if r.world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value: float, r: Ranks, device=None) -> float:
    if r.world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, r: Ranks, device=None) -> float:
    if r.world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def finish(r: Ranks):
    if r.world > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()
