"""Environment sharding and the max-over-ranks timing of the multi-GPU path, on CPU with two
gloo ranks (the data path itself has no collective)."""
import os
import socket

import numpy as np
import pytest

from paper_2412_12089_gb300.sharding import max_over_ranks, shard_envs, sum_over_ranks


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shards_cover_every_env_once_and_balance(world):
    rng = np.random.default_rng(world)
    costs = list(np.exp(rng.uniform(np.log(2000), np.log(16000), 512)) * 20 * 32)
    ranges = shard_envs(costs, world)
    assert len(ranges) == world
    covered = []
    for s, c in ranges:
        covered.extend(range(s, s + c))
    assert covered == list(range(len(costs)))  # contiguous, in order, no overlap
    loads = [sum(costs[s:s + c]) for s, c in ranges]
    # greedy contiguous split: each rank within one environment's cost of the mean
    assert max(loads) - sum(loads) / world <= max(costs) + 1e-6


def test_more_ranks_than_envs():
    ranges = shard_envs([1.0, 2.0], 4)
    assert sum(c for _, c in ranges) == 2 and len(ranges) == 4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, costs, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s, c = shard_envs(costs, world)[rank]
        units = float(sum(costs[s:s + c]))
        t = max_over_ranks(1.0 + rank)           # per-rank "elapsed time"
        tot = sum_over_ranks(units)              # whole-job units
        dist.barrier()
        out.put((rank, s, c, t, tot))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as mp

    costs = [float(x) for x in range(1, 41)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, c0, t0, tot0), (r1, s1, c1, t1, tot1) = res
    assert (s0, s0 + c0) == (0, s1) and s1 + c1 == len(costs)
    assert t0 == t1 == 2.0                        # max over ranks
    assert tot0 == tot1 == sum(costs)             # all units processed, counted once
