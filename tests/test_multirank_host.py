"""Host logic of the multi-rank benchmark on CPU (gloo, world size 2): the
path does not shard (replicas only), so the only cross-rank step is the job
time, the maximum over the ranks of each rank's own time, and the value is
all ranks' units over that time. No GPU and no NCCL."""
import os
import socket

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
