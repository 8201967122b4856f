"""The N > 1 path without GPUs: two gloo ranks on the CPU run the benchmark's
sharding and its max-over-ranks timing reduction.  Molecules are independent,
so the shards must be disjoint, cover the whole set, and give each rank the
same molecules the single-rank generator gives for those indices."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, nmol, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    idx = bench.shard_indices(nmol, rank, world)
    allm = bench.workload(nmol * world)
    natoms = [len(allm[i][0]) for i in idx]
    t = bench.max_over_ranks(10.0 * (rank + 1))
    got = [None] * world
    dist.all_gather_object(got, idx)
    dist.destroy_process_group()
    out.put((rank, idx, natoms, t, got))


def test_two_gloo_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port, nmol, world = _free_port(), 5, 2
    ps = [ctx.Process(target=_rank, args=(r, world, port, nmol, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    sys.path.insert(0, ROOT)
    import bench
    full = bench.workload(nmol * world)
    seen = []
    for rank, idx, natoms, t, got in res:
        assert len(idx) == nmol
        assert t == 10.0 * world  # max over ranks
        assert natoms == [len(full[i][0]) for i in idx]
        assert got[rank] == idx
        seen += idx
    assert sorted(seen) == list(range(nmol * world))
