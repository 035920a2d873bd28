"""The multi-rank path of the benchmark on CPU (gloo, world size 2): every
rank grows its own replica of the workload (distinct seeds, no data
exchange), and the reported figures are the slowest rank's time and the sum
of all ranks' robot-link-steps."""
import os
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2509_15180_gb300 import scenes
    sc = scenes.design_batch(8, replicate=rank)
    units = scenes.robot_link_steps(sc["n_links"]) * (rank + 1)
    t, u = bench.reduce_over_ranks(1.5 + rank, units, "cpu")
    out[rank] = (t, u, float(sc["pressure"][0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_report_max_time_and_summed_units():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = 29000 + (os.getpid() % 1000)
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    (t0, u0, p0), (t1, u1, p1) = out[0], out[1]
    rls = 8 * 100 * 101 // 2
    assert t0 == t1 == 2.5
    assert u0 == u1 == rls * 3
    assert p0 != p1  # each rank grows a different replica


def _lpt_worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2509_15180_gb300 import scenes, shard
    sc = scenes.uneven_batch(512, replicate=2)
    cost = shard.robot_cost(sc)
    mine = shard.lpt_partition(cost, world)[rank]
    got = [None] * world
    dist.all_gather_object(got, (mine.tolist(), float(cost[mine].sum())))
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_lpt_shards_cover_the_batch_once_and_balance_cost():
    """Two gloo ranks compute their LPT shards independently (no data
    exchange is needed to agree): together they hold every robot exactly
    once, and the larger shard's cost is within LPT's bound."""
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = 30000 + (os.getpid() % 1000)
    mp.start_processes(_lpt_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    assert out[0] == out[1]
    (i0, c0), (i1, c1) = out[0]
    assert sorted(i0 + i1) == list(range(512)) and not set(i0) & set(i1)
    sys.path.insert(0, ROOT)
    from paper_2509_15180_gb300 import scenes, shard
    cost = shard.robot_cost(scenes.uneven_batch(512, replicate=2))
    assert max(c0, c1) <= cost.sum() / 2 + cost.max()
    assert max(c0, c1) <= 4.0 / 3.0 * max(cost.sum() / 2, cost.max())


def test_lpt_partition_small_cases():
    sys.path.insert(0, ROOT)
    from paper_2509_15180_gb300 import shard
    # Graham's worst case for 2 machines: 3, 3, 2, 2, 2 -> LPT 7 against the optimum 6
    parts = shard.lpt_partition([3, 3, 2, 2, 2], 2)
    loads = sorted(sum([3, 3, 2, 2, 2][i] for i in p) for p in parts)
    assert loads == [5, 7]
    assert [list(p) for p in shard.lpt_partition([5.0], 3)] == [[0], [], []]
    with pytest.raises(ValueError):
        shard.lpt_partition([1.0], 0)
