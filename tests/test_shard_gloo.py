"""Multi-rank host logic on CPU (gloo, world size 2): distinct per-rank domains,
contiguous column splits, max/sum reductions of the timing and point counts,
and that a rank's columns step identically wherever they are computed."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2010_14823_gb300 import shard, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = shard.rank_env()
        seed = shard.rank_seed(1236, r)
        fld, dz, nc, nl, dt, _ = synth.workload("deep_512x512x150", ncols=64, nlev=30, seed=seed)
        # the rank's share of a split domain, stepped on its own
        lo, hi = shard.column_range(nc, r, w)
        sub = np.zeros((16, nl, 32 * ((hi - lo + 31) // 32)))
        sub[:, :, :hi - lo] = fld[:, :, lo:hi]
        O.step(sub, hi - lo, dz, dt)
        pts = shard.sum_over_ranks(nc * nl, dist)
        tmax = shard.max_over_ranks(float(r + 1), dist)
        q.put((r, seed, lo, hi, pts, tmax, sub[:, :, :hi - lo].copy(), fld[0, 0, 0]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=300) for _ in range(world)], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, lo0, hi0, pts0, t0, out0, f0), (r1, s1, lo1, hi1, pts1, t1, out1, f1) = res
    assert s0 != s1 and f0 != f1                 # distinct synthetic domains per rank
    assert (lo0, hi0, lo1, hi1) == (0, 32, 32, 64)
    assert pts0 == pts1 == 2 * 64 * 30           # points summed over ranks
    assert t0 == t1 == 2.0                       # the job's time is the slowest rank's
    # rank 0's half of its domain gives the same result as inside the whole domain
    fld, dz, nc, nl, dt, _ = synth.workload("deep_512x512x150", ncols=64, nlev=30, seed=s0)
    O.step(fld, nc, dz, dt)
    assert np.array_equal(fld[:, :, 0:32], out0)


def test_column_ranges_cover_exactly():
    for n in (0, 1, 7, 64, 1000):
        for w in (1, 2, 3, 8):
            rs = [shard.column_range(n, r, w) for r in range(w)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            assert max(b - a for a, b in rs) - min(b - a for a, b in rs) <= 1


def test_aligned_column_ranges_cover_exactly():
    from paper_2010_14823_gb300 import shard
    for ncols in (1, 31, 32, 33, 1000, 4096, 262144):
        for world in (1, 2, 3, 7, 8):
            parts = [shard.column_range_aligned(ncols, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == ncols
            for (a0, a1), (b0, b1) in zip(parts, parts[1:]):
                assert a1 == b0
            for a0, a1 in parts:
                assert a0 <= a1 and (a0 % 32 == 0 or a0 == a1)
            sizes = [max(0, (a1 - a0 + 31) // 32) for a0, a1 in parts]
            assert max(sizes) - min(sizes) <= 1 or ncols < 32 * world
