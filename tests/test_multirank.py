"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own
locations; the job's rate is all ranks' units over the slowest rank's time,
and every rank computes the same figure.  The reference arm prints only on
rank 0."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import torch.distributed as dist
    r, w = bench.dist_init(None, backend="gloo")
    assert (r, w) == (rank, world)
    bench.barrier(w)
    ms = 100.0 * (rank + 1)           # rank 1 is the slower one
    rate, ms_max = bench.whole_job_rate(1000, 5, ms, w)
    q.put((rank, rate, ms_max))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_whole_job_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, rate, ms_max in out:
        assert ms_max == 200.0
        assert rate == pytest.approx(2 * 1000 * 5 / 0.2)


def test_single_rank_rate():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    rate, ms = bench.whole_job_rate(100, 2, 50.0, 1)
    assert ms == 50.0 and rate == pytest.approx(4000.0)
