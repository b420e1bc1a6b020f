"""The N > 1 path of bench.py on CPU, with two gloo ranks.

Locations are independent, so the job shards with no data-path collective:
every rank holds the same design and responses and predicts its own
contiguous block of the job's locations (weak scaling).  The job's rate is all
ranks' units over the slowest rank's time, the same figure on every rank.  The
reference arm prints only on rank 0."""
import hashlib
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _digest(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, ROOT)
    import bench
    import torch
    import torch.distributed as dist
    r, w = bench.dist_init(None, backend="gloo")
    assert (r, w) == (rank, world)
    bench.barrier(w)
    # the rank's workload: same design everywhere, its own block of locations
    wl = bench.rank_workload(M=37, N=3000, rank=rank, world=world)
    design = _digest(wl.X, wl.Y)
    # every rank's design digest and locations reach rank 0 through the group
    digests = [None] * world
    dist.all_gather_object(digests, design)
    locs = [None] * world
    dist.all_gather_object(locs, wl.Xref)
    ms = 100.0 * (rank + 1)           # rank 1 is the slower one
    rate, ms_max = bench.whole_job_rate(wl.M, 5, ms, w)
    q.put((rank, rate, ms_max, digests, [np.asarray(a) for a in locs]))
    dist.destroy_process_group()


def _run(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=180) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    return out


def test_two_gloo_ranks_share_the_design_and_split_the_locations():
    import sys
    sys.path.insert(0, ROOT)
    from paper_1409_0074_gb300 import workloads as W
    out = _run(2)
    job = W.large_8d(M=2 * 37, N=3000)
    for rank, rate, ms_max, digests, locs in out:
        # one design, replicated
        assert len(set(digests)) == 1 and digests[0] == _digest(job.X, job.Y)
        # the blocks are disjoint, cover the job's locations and follow rank order
        assert [a.shape[0] for a in locs] == [37, 37]
        np.testing.assert_array_equal(np.concatenate(locs), job.Xref)
        # the job's rate: both ranks' locations over the slower rank's time
        assert ms_max == 200.0
        assert rate == pytest.approx(2 * 37 * 5 / 0.2)


def test_shard_blocks_cover_uneven_totals():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    for total in (0, 1, 7, 100, 101):
        for world in (1, 2, 3, 8):
            blocks = [bench.shard(total, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == total
            for (a, b), (c, d) in zip(blocks, blocks[1:]):
                assert b == c and a <= b
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1


def test_single_rank_rate():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    rate, ms = bench.whole_job_rate(100, 2, 50.0, 1)
    assert ms == 50.0 and rate == pytest.approx(4000.0)
