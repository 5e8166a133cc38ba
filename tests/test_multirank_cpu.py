"""The N > 1 bench path on CPU: two gloo ranks on 127.0.0.1 combine their
device times (slowest rank) and updates (all ranks) as bench.py does under
torchrun; each rank runs an independent replica with its own seed."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, u = bench.combine_ranks(10.0 + 5.0 * rank, 1000 * (rank + 1), "cpu")
        q.put((rank, t, u, bench.workload_for(rank).vortices.xc.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_like_the_bench():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, t, u, _ in out:
        assert t == 15.0          # the slowest rank's time
        assert u == 3000          # all ranks' updates
    assert out[0][3] != out[1][3]   # independent replicas: seeds differ by rank


def test_single_process_keeps_its_numbers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(7.5, 42, "cpu") == (7.5, 42)
