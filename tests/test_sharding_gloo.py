"""The multi-rank path on CPU with the gloo backend (world size 2).

Primaries are independent, so a run sharded by primary range needs only one
final sum: each rank forms the ordered pair sums of its primary range (the
benchmark's `shard_range`; here with the oracle, the only part of the path that
runs without a GPU) and the benchmark's `combine_shards` (one FP64 all-reduce)
reproduces the full sum.  The benchmark's rank combination (slowest rank's time,
summed work) is checked on the same group.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch

    import bench
    import oracle
    from paper_2005_01739_gb300 import catalogs

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    oracle.set_threads(2)
    pos, w = catalogs.thomas(1200, 80.0, 40, 1.5, seed=5, weights="u05_15")
    edges = catalogs.linear_edges(0.2, 2.0, 10)
    n = len(pos)
    # the benchmark's own shard layout and combination of the partial DD
    lo, hi = bench.shard_range(rank, world, n)
    DD, npairs = oracle.power_pair_sum(pos.astype(np.float64), w.astype(np.float64), 80.0, 15.0, edges, 4,
                                       primaries=np.arange(lo, hi))
    total = bench.combine_shards(DD, "cpu")
    c = torch.tensor([float(npairs)], dtype=torch.float64)
    dist.all_reduce(c)
    ranges = [bench.shard_range(r, world, n) for r in range(world)]
    ms, work = bench.combine_ranks(10.0 + rank, 100.0 * (rank + 1), "cpu")
    if rank == 0:
        full, nfull = oracle.power_pair_sum(pos.astype(np.float64), w.astype(np.float64), 80.0, 15.0, edges, 4)
        out.put((float(np.max(np.abs(total - full))), float(np.max(np.abs(full))), int(c.item()), nfull,
                 ms, work, ranges))
    dist.barrier()
    dist.destroy_process_group()


def test_primary_range_sharding_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    diff, scale, n_sum, n_full, ms, work, ranges = res
    assert ranges[0][0] == 0 and ranges[-1][1] == 1200
    assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))  # disjoint, covering
    assert n_sum == n_full
    assert diff < 1e-12 * scale
    assert ms == 11.0 and work == 300.0
