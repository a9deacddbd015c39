"""Replica coordination of bench.py on CPU: two gloo ranks (no GPU, no collective on the data path).

The solve does not shard (one iterate, updated in place every step): N GPUs run N independent solves with their own sketch
stream (stream_id = rank), a barrier and a MAX over the ranks' timed regions, and the job value is all
ranks' solves over the slowest rank's time.  These tests run that host logic with world_size 2.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        mine = 1.5 + rank  # a rank's timed region (seconds)
        slowest = bench.max_over_ranks(world, mine, device="cpu")
        out[rank] = (slowest, bench.job_value(world, 3, slowest))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_job_value():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # every rank sees the slowest rank's time, and the job value counts all ranks' solves
    assert res[0][0] == res[1][0] == 2.5
    assert res[0][1] == res[1][1] == pytest.approx(2 * 3 / 2.5)


def test_replicas_draw_independent_sketch_streams():
    # rank r uses stream_id = r: the counter-based sketches of the replicas are independent draws
    from oracle import oracle as orc

    n, q = 512, 16
    s0 = orc.gauss_sketch(7, 0, 3, n, q)
    s1 = orc.gauss_sketch(7, 1, 3, n, q)
    assert not np.array_equal(s0, s1)
    assert abs(np.corrcoef(s0.ravel(), s1.ravel())[0, 1]) < 0.05
