"""The multi-process host logic of bench.py on CPU ranks (gloo, world size 2): the timed region
is the slowest rank's, and the slices of the batching workload are dealt so that every slice is
reconstructed by exactly one rank.  The data path itself has no exchange (replicas)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    t = bench.max_over_ranks(10.0 + 5.0 * rank, world, torch.device("cpu"))
    mine = bench.rank_slices(64, rank, world)
    got = [None] * world
    dist.all_gather_object(got, mine)
    out[rank] = (t, got)
    dist.destroy_process_group()


def test_max_over_ranks_and_slice_dealing():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, parts = res[r]
        assert t == 15.0
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        assert all(len(set(parts[a]) & set(parts[b])) == 0 for a in range(world)
                   for b in range(world) if a != b)


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, torch.device("cpu")) == 3.5
    assert bench.rank_slices(5, 0, 1) == [0, 1, 2, 3, 4]
