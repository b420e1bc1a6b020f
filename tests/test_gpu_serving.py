"""Serving context (laGP_ctx_*) and the continuous-batching loop on the GPU.

A location's prediction must be the same when its request runs alone, when it
is merged with other requests into one device batch, and when other batches
run concurrently; and the same as a direct laGP_build_and_predict call.
Admission must refuse (LAGP_BUSY) a request whose arena region is not free and
accept it once a completed request has been collected.
"""
import numpy as np
import pytest

from gpu_helpers import to_dev
from paper_1409_0074_gb300 import workloads as W
from paper_1409_0074_gb300.serve import CtxBackend, Request, Server, run_stream

pytestmark = pytest.mark.gpu

N_CLOSE, N0, NRAYS = 1000, 6, 8


@pytest.fixture(scope="module")
def lagp(cuda):
    from paper_1409_0074_gb300 import build
    build.build()
    from paper_1409_0074_gb300 import lagp as L
    L.load()
    return L


@pytest.fixture(scope="module")
def design():
    w = W.large_8d(M=4000)
    return w, to_dev(w.X), to_dev(w.Y)


def _ctx(lagp, design, arena_bytes, slots=4):
    w, X, Y = design
    return lagp.Context(X, Y, w.theta, w.g, N0, N_CLOSE, lagp.LAGP_RAY, NRAYS,
                        lagp.LAGP_FP32_SCORE, arena_bytes, max_inflight=slots)


def _pinned(shape, dtype):
    import torch
    return torch.empty(shape, dtype=dtype).pin_memory().numpy()


def test_solo_mix_and_direct_results_are_identical(lagp, design):
    import torch
    w, X, Y = design
    rng = np.random.default_rng(5)
    xa = w.Xref[:300]
    others = [(w.Xref[300:700], 100), (w.Xref[700:720], 30), (w.Xref[720:2720], 50)]
    # direct call
    d = lagp.predict(X, Y, to_dev(xa), N0, 50, N_CLOSE, w.theta, w.g, search="ray", nrays=NRAYS,
                     precision="fp32")
    dm, ds = d["mean"].cpu().numpy(), d["s2"].cpu().numpy()
    ctx = _ctx(lagp, design, 2 << 30)
    # alone through the context
    mean, s2 = _pinned(300, torch.float64), _pinned(300, torch.float64)
    t = ctx.submit(np.ascontiguousarray(xa), 50, mean, s2)
    ctx.wait(t)
    np.testing.assert_array_equal(mean, dm)
    np.testing.assert_array_equal(s2, ds)
    # in a mix: all arrive together; the server merges what fits into one batch
    # and runs the rest concurrently in other slots
    srv = Server(CtxBackend(ctx, max_batch=2048, slots=4), max_batch=2048)
    reqs = [Request(0, xa, 50, 0.0)] + [Request(k + 1, x, n, 0.0)
                                       for k, (x, n) in enumerate(others)]
    reqs = [reqs[0]] + [reqs[1 + i] for i in rng.permutation(3)]
    run_stream(srv, reqs)
    assert len(srv.done) == 4 and srv.batches >= 2
    a = [r for r in reqs if r.rid == 0][0]
    np.testing.assert_array_equal(a.mean, dm)
    np.testing.assert_array_equal(a.s2, ds)
    # every request of the mix equals its own direct call
    for r in reqs[1:]:
        dd = lagp.predict(X, Y, to_dev(r.xref), N0, r.n, N_CLOSE, w.theta, w.g, search="ray",
                          nrays=NRAYS, precision="fp32")
        np.testing.assert_array_equal(r.mean, dd["mean"].cpu().numpy())
        np.testing.assert_array_equal(r.s2, dd["s2"].cpu().numpy())
    ctx.close()


def test_admission_by_free_arena(lagp, design):
    import torch
    w, X, Y = design
    dbytes = lagp.load().laGP_ctx_design_bytes(w.N, w.p)
    rb = lagp.load().laGP_ctx_request_bytes(w.N, w.p, 500, 50, N_CLOSE, NRAYS, lagp.LAGP_RAY,
                                            lagp.LAGP_FP32_SCORE, 0)
    ctx = _ctx(lagp, design, dbytes + rb + 4096, slots=4)
    free, slots = ctx.capacity()
    assert free >= rb and slots == 4
    bufs = [(_pinned(500, torch.float64), _pinned(500, torch.float64)) for _ in range(2)]
    xa, xb = np.ascontiguousarray(w.Xref[:500]), np.ascontiguousarray(w.Xref[500:1000])
    ta = ctx.submit(xa, 50, *bufs[0])
    assert ta is not None
    assert ctx.submit(xb, 50, *bufs[1]) is None          # no room beside the first
    ctx.wait(ta)
    tb = ctx.submit(xb, 50, *bufs[1])
    assert tb is not None
    ctx.wait(tb)
    ref = lagp.predict(X, Y, to_dev(xb), N0, 50, N_CLOSE, w.theta, w.g, search="ray",
                       nrays=NRAYS, precision="fp32")
    np.testing.assert_array_equal(bufs[1][0], ref["mean"].cpu().numpy())
    ctx.close()
