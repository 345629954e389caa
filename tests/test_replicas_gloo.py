"""The multi-rank path of bench.py (independent replicas, one per GPU) on CPU
with two gloo ranks: the whole-job time is the slowest rank's, the paths are
summed, and ranks sample different seeds."""

import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        seconds = [1.5, 2.25][rank]
        paths = [1000, 3000][rank]
        t, p = bench.reduce_replicas(dist, seconds, paths, "cpu")
        seeds = [bench.replica_seed(rank, i) for i in range(5)]
        out.put((rank, t, p, seeds))
    finally:
        dist.destroy_process_group()


def test_replicas_reduce_with_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort()
    for rank, t, p, seeds in res:
        assert t == 2.25 and p == 4000.0  # max time, summed paths, on every rank
    assert not set(res[0][3]) & set(res[1][3])  # different seeds per rank


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_replicas(None, 3.0, 7, "cpu") == (3.0, 7.0)
