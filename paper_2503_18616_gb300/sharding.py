"""Environment sharding across GPUs (one process per GPU).

Environments are independent (each env's variables live in its own slice of
every array, FF-SRL Sec. III-B), so a multi-GPU run shards envs across ranks
with no exchange on the data path. Every env keeps its global id, which the
simulator's counter-based draws use (ffsrl_set_env_ids): a shard draws for
its envs exactly what a one-process run draws for them, whatever the split.
These helpers hold the host-side logic: contiguous shares of a fixed env set,
greedy bin-packing of uneven envs by their work, and the timing reduction
that turns per-rank times into one whole-job throughput.
"""
from __future__ import annotations


def env_range(n_total: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous [begin, end) share of n_total envs for `rank` (sizes differ by at most one)."""
    base, extra = divmod(n_total, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def env_work(V: int, E: int, T: int) -> int:
    """Work of one env-step in constraint-and-vertex units: V + E + T."""
    return V + E + T


def balanced_shards(work, world: int) -> list[list[int]]:
    """Greedy bin-packing (longest processing time first): envs in order of
    decreasing work (ties: lower id first) go one by one to the rank with the
    least work so far (ties: lower rank). Returns each rank's env ids, sorted."""
    order = sorted(range(len(work)), key=lambda e: (-work[e], e))
    load = [0] * world
    shards: list[list[int]] = [[] for _ in range(world)]
    for e in order:
        r = min(range(world), key=lambda q: (load[q], q))
        shards[r].append(e)
        load[r] += work[e]
    return [sorted(s) for s in shards]


def shard_envs(n_total: int, world: int, rank: int, work=None) -> list[int]:
    """Global ids of the envs `rank` owns: a contiguous share, or (with a
    per-env work list) the rank's bin of balanced_shards."""
    if work is None:
        b, e = env_range(n_total, world, rank)
        return list(range(b, e))
    if len(work) != n_total:
        raise ValueError("need one work value per env")
    return balanced_shards(work, world)[rank]


def weak_shard(n_per_rank: int, rank: int) -> list[int]:
    """Global ids of a weak-scaling shard: every rank owns n_per_rank envs of
    its own, ids rank * n_per_rank ... (rank + 1) * n_per_rank - 1."""
    return list(range(rank * n_per_rank, (rank + 1) * n_per_rank))


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank float over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized():
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    """Sum of a per-rank float over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized():
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def throughput(envs_per_rank: int, world: int, steps: int, seconds: float) -> float:
    """Whole-job env-steps/s when every rank advanced its envs `steps` times."""
    return world * envs_per_rank * steps / seconds
