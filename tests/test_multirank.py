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


def _rank_scan(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import numpy as np
    import torch.distributed as dist
    import bench
    from oracle import oracle as O
    from paper_1611_05293_b300 import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = {}
    for S, Pi in bench.scan_points(3, rank, world):
        op = O.Params(n=16, steps_per_period=50, beta=0.1, s_csr=S)
        zr, zi = O.impedance(op, 2, Pi)
        psi, P, _ = O.run(op, zr, zi, O.normalize(op, W.noisy_gaussian(16, 1612, 1e-6)), 20)
        out[(S, Pi)] = (psi, P)
    gathered = [None] * world
    dist.all_gather_object(gathered, out)
    q.put((rank, gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_ranks_compute_their_slice_of_the_scan():
    """Each rank advances only its own slice of the scan (no collective in the
    data path); gathering the ranks' results gives every point of the scan
    once, each the same bits as the point run alone.  The ranks run the FP64
    oracle on tiny grids (no GPU here); the slicing and gathering are what
    bench.py does across GPUs."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_scan, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import sys
    import numpy as np
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from oracle import oracle as O
    from paper_1611_05293_b300 import workloads as W
    merged = {}
    for part in res[0][1]:
        for k, v in part.items():
            assert k not in merged
            merged[k] = v
    assert sorted(merged) == sorted(bench.scan_points(6))
    for (S, Pi), (psi, P) in merged.items():
        op = O.Params(n=16, steps_per_period=50, beta=0.1, s_csr=S)
        zr, zi = O.impedance(op, 2, Pi)
        ref, Pref, _ = O.run(op, zr, zi, O.normalize(op, W.noisy_gaussian(16, 1612, 1e-6)), 20)
        assert np.array_equal(psi, ref) and np.array_equal(P, Pref)
