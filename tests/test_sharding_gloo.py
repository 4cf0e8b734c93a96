"""Multi-rank host logic of the env-sharded benchmark, on CPU with gloo.

Envs are independent slices of one batch (FF-SRL Sec. III-B), so a split of
a fixed env set across ranks must reproduce, env by env, what one process
computes for the same global env ids. Two gloo ranks each take their shard
of a small uneven batch (bin-packed by V + E + T), advance their envs with
the FP64 oracle under the global ids, and gather the results; they must
equal the one-rank run bit for bit, the shards must partition the env set,
and the bin-packed loads must be balanced as the greedy rule guarantees.
"""
import os

import numpy as np

from paper_2503_18616_gb300 import inputs, sharding


def test_env_ranges_partition_the_envs():
    for n, world in [(4096, 2), (1024, 3), (7, 4), (5, 8)]:
        ranges = [sharding.env_range(n, world, r) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == n
        for (a, b), (c, d) in zip(ranges, ranges[1:]):
            assert b == c
        sizes = [b - a for a, b in ranges]
        assert max(sizes) - min(sizes) <= 1
        assert [sharding.shard_envs(n, world, r) for r in range(world)] == [list(range(a, b)) for a, b in ranges]


def test_balanced_shards_partition_and_balance():
    """Greedy longest-first packing: a partition of the envs, and the largest
    load exceeds the smallest by at most the largest single env's work."""
    rng = np.random.default_rng(4)
    for world in (2, 3, 8):
        work = [int(w) for w in np.exp(rng.uniform(np.log(500), np.log(20000), 257))]
        shards = sharding.balanced_shards(work, world)
        flat = sorted(e for s in shards for e in s)
        assert flat == list(range(len(work)))
        loads = [sum(work[e] for e in s) for s in shards]
        assert max(loads) - min(loads) <= max(work)
    # by hand: works 5, 4, 3, 3, 1 on two ranks: 5 -> r0; 4 -> r1; the first 3
    # -> r1 (4 < 5); the second 3 -> r0 (5 < 7); 1 -> r1 (7 < 8): loads 8 and 8
    assert sharding.balanced_shards([5, 4, 3, 3, 1], 2) == [[0, 3], [1, 2, 4]]


def test_weak_shards_are_disjoint_id_ranges():
    assert sharding.weak_shard(4, 0) == [0, 1, 2, 3]
    assert sharding.weak_shard(4, 2) == [8, 9, 10, 11]


N_ENV, STEPS, SEED = 12, 3, 17


def _batch():
    shapes, env_mesh = inputs.uneven_batch(N_ENV, 60, 400, seed=3)
    meshes = [inputs.grid_block(*sh) for sh in shapes]
    work = []
    for e in range(N_ENV):
        rest, _, tets = meshes[env_mesh[e]]
        pairs = np.concatenate([tets[:, [a, b]] for a, b in ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))])
        work.append(sharding.env_work(len(rest), len(np.unique(np.sort(pairs, axis=1), axis=0)), len(tets)))
    return meshes, env_mesh, work


def _advance(ids):
    """The oracle's envs of the given global ids after STEPS device-drawn steps:
    {id: (positions, observed ids, target)}."""
    import oracle
    meshes, env_mesh, _ = _batch()
    om = {}
    out = {}
    p = inputs.default_params(n_obs=4)
    for g in ids:
        mi = int(env_mesh[g])
        if mi not in om:
            om[mi] = oracle.Mesh(*meshes[mi])
        oe = oracle.Env(om[mi], p)
        oe.reset(SEED, int(g))
        oe.run(STEPS, want_obs=False)
        ints = oe.ints()
        out[int(g)] = (oe.state()[0], ints["obs_ids"], ints["target"])
    return out


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    _, _, work = _batch()
    ids = sharding.shard_envs(N_ENV, world, rank, work)
    res = _advance(ids)
    gathered = [None] * world
    dist.all_gather_object(gathered, (rank, ids, res))
    t = 1.0 + rank                      # rank 1 is the slowest
    tmax = sharding.max_over_ranks(t, dist, "cpu")
    total = sharding.sum_over_ranks(float(len(ids)), dist, "cpu")
    if rank == 0:
        q.put((gathered, tmax, total))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_split_reproduces_the_one_rank_run():
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, tmax, total = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert tmax == 2.0 and total == N_ENV     # max time and the summed env count
    _, _, work = _batch()
    shards = [g[1] for g in sorted(gathered)]
    assert shards == sharding.balanced_shards(work, 2)
    assert sorted(e for s in shards for e in s) == list(range(N_ENV))
    split = {}
    for _, _, res in gathered:
        split.update(res)
    whole = _advance(range(N_ENV))
    for g in range(N_ENV):
        xs, os_, ts = split[g]
        xw, ow, tw = whole[g]
        assert np.array_equal(xs, xw) and np.array_equal(os_, ow) and ts == tw, g
    # distinct ids draw distinct episodes (the split is not a copy of one env)
    assert len({tuple(whole[g][1]) for g in range(N_ENV)}) > 1
