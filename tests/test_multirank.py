"""Replica scaling path of bench.py on CPU with two gloo ranks: the ranks'
scan points are disjoint slices of one scan, and the job time every rank
reports is the slowest rank's (all_reduce MAX), so value = world x cells /
max time."""
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


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pts = bench.scan_points(8, rank, world)
    t = bench.max_over_ranks(1.0 + rank, dist, "cpu")
    q.put((rank, pts, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_points_and_take_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict((r, (pts, t)) for r, pts, t in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert res[0][0] + res[1][0] == bench.scan_points(16)
    assert res[0][1] == res[1][1] == 2.0
