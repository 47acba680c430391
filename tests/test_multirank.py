"""The multi-GPU benchmark path on CPU: two gloo ranks.

Every rank solves its own batch (seed = rank); the only cross-rank operation
is the maximum of the step times (no collective on the data path), and the
reported value is the work of all ranks over that time.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2507_10290_gb300 import workloads as W
    ms, value = bench.aggregate_ranks(times[rank], 1000.0, world, device="cpu")
    w = W.batch(seed=rank, B=8)
    q.put((rank, ms, value, float(w.durations.sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_weak_scaling_value():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [12.5, 20.0]
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, ms, value, _ in out:
        assert ms == pytest.approx(20.0)
        assert value == pytest.approx(world * 1000.0 / 0.020)
    # the ranks drew different batches
    assert out[0][3] != out[1][3]


def test_single_rank_needs_no_process_group():
    import bench
    ms, value = bench.aggregate_ranks(10.0, 500.0, 1)
    assert ms == 10.0 and value == pytest.approx(500.0 / 0.01)
