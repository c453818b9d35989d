"""Host logic of the multi-rank paths on CPU (gloo, world size 2). A single
mesh does not shard (replicas only): the benchmark's only cross-rank step
is the job time, the maximum over the ranks of each rank's own time, and
the value is all ranks' units over that time. A batch of independent
instances shards by instance (replicas.py): the split is balanced and
covers every instance once, and the per-instance results are gathered in
instance order on every rank. No GPU and no NCCL."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    own_ms = 100.0 + 25.0 * rank          # the ranks' own timed regions differ
    tmax = bench.max_over_ranks(own_ms, dist, "cpu")
    units = 200 * 5                       # PD steps per rank: T x benchmark steps
    out[rank] = (tmax, world * units / (tmax / 1e3))
    dist.barrier()
    dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_value_counts_all_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert set(res) == {0, 1}
    for r in range(world):
        tmax, value = res[r]
        assert tmax == 125.0
        assert value == pytest.approx(2 * 1000 / 0.125)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(42.0, None, "cpu") == 42.0


def test_replicas_are_distinct_instances():
    import numpy as np
    from paper_2605_14526_b300 import inputs
    a, b = inputs.hetero_bar(seed=2), inputs.hetero_bar(seed=3)
    assert a.X.shape == b.X.shape
    assert not np.array_equal(a.E, b.E) or not np.array_equal(a.target, b.target)


def test_shard_instances_covers_each_once_and_balances():
    from paper_2605_14526_b300.replicas import shard_instances
    rng = np.random.default_rng(3)
    costs = rng.integers(1000, 40000, 64)
    for world in (1, 2, 3, 8):
        share = shard_instances(costs, world)
        flat = sorted(i for s in share for i in s)
        assert flat == list(range(64))
        loads = [costs[s].sum() for s in share]
        # greedy LPT: the largest load is within the largest single cost of the mean
        assert max(loads) <= costs.sum() / world + costs.max()
        assert all(s == sorted(s) for s in share)
    assert shard_instances([5, 1], 4) == [[0], [1], [], []]
    assert shard_instances(costs, 2) == shard_instances(costs, 2)   # deterministic


def _gather_main(rank, world, port, out):
    import torch.distributed as dist

    from paper_2605_14526_b300.replicas import gather_instances, shard_instances
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    costs = [7, 3, 9, 1, 4, 4]
    share = shard_instances(costs, world)[rank]
    # each instance's "result": arrays that name the instance, computed by its owner only
    res = {"loss": [float(i) ** 2 for i in share], "dE": [np.full(i + 1, float(i)) for i in share]}
    full = gather_instances(share, res, len(costs), dist)
    out[rank] = (share, full["loss"], [a.tolist() for a in full["dE"]])
    dist.barrier()
    dist.destroy_process_group()


def test_gather_instances_over_two_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_gather_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    shares = [res[r][0] for r in range(world)]
    assert sorted(shares[0] + shares[1]) == list(range(6)) and shares[0] and shares[1]
    for r in range(world):   # every rank holds every instance, in instance order
        assert res[r][1] == [float(i) ** 2 for i in range(6)]
        assert res[r][2] == [[float(i)] * (i + 1) for i in range(6)]


def test_gather_instances_refuses_incomplete_shares():
    from paper_2605_14526_b300.replicas import gather_instances
    with pytest.raises(ValueError):
        gather_instances([0, 2], {"loss": [1.0, 2.0]}, 3, None)
