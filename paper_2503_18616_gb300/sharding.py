"""Environment sharding across GPUs (one process per GPU).

Environments are independent (each env's variables live in its own slice of
every array, FF-SRL Sec. III-B), so a multi-GPU run shards envs across ranks
with no exchange on the data path. These helpers hold the host-side logic: the
per-rank seed, contiguous env ranges for a fixed total, and the timing
reduction that turns per-rank times into one whole-job throughput.
"""
from __future__ import annotations

RANK_SEED_STRIDE = 1000003


def rank_seed(seed: int, rank: int) -> int:
    """Seed of the env shard owned by `rank` (distinct streams per rank)."""
    return seed + RANK_SEED_STRIDE * rank


def env_range(n_total: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous [begin, end) share of n_total envs for `rank` (sizes differ by at most one)."""
    base, extra = divmod(n_total, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank float over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized():
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(envs_per_rank: int, world: int, steps: int, seconds: float) -> float:
    """Whole-job env-steps/s when every rank advanced its envs `steps` times."""
    return world * envs_per_rank * steps / seconds
