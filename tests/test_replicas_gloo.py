"""The multi-GPU form of the bench is N independent replicas (one problem per GPU, no collective
on the data path); its only cross-rank step is the maximum of the ranks' step times. Here two
ranks on the CPU (gloo, 127.0.0.1) check that every rank gets the slowest rank's time and that a
single process needs no process group."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)
    os.environ["LOCAL_RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(world)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, local, w = bench.rank_info()
        t = bench.max_over_ranks(0.1 + r, dist)  # rank 1 is the slow one
        out[rank] = (r, local, w, t)
    finally:
        dist.destroy_process_group()


def test_single_process_needs_no_group():
    import bench

    assert bench.max_over_ranks(0.25) == 0.25


@pytest.mark.timeout(120)
def test_two_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (r, local, w, t) in res.items():
        assert (r, local, w) == (rank, rank, world)
        assert t == pytest.approx(1.1)
