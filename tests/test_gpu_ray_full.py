"""Ray search with the unlimited snap scope (LAGP_RAY_FULL, reading R14)
through the C ABI, against the oracle run with snap = "design": the snap
searches all of X_N outside the local design through a k-d tree built on the
GPU with the design's preparation.

FP64 form: identical designs, gaps and evaluation counts, predictions within
1e-10 (in practice bit-identical), on the 2-d workload in full, edge sizes of
the tree (a single leaf, one split), a design holding every point twice (exact
ties) and a 4-d sample.  FP32-scoring form: the checks of the FP32 form on a
sample of the 8-d workload in the bench's launch configuration."""
import numpy as np
import pytest

import oracle
from gpu_helpers import _sample, check_fp32_form, to_dev
from paper_1409_0074_gb300 import workloads as W
from test_gpu_parity import assert_fp64_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lagp(cuda):
    from paper_1409_0074_gb300 import build
    build.build()
    from paper_1409_0074_gb300 import lagp as L
    L.load()
    return L


def run_full(L, w, precision, nrays):
    import torch
    out = L.predict(to_dev(w.X), to_dev(w.Y), to_dev(w.Xref), w.n0, w.n, w.nc, w.theta, w.g,
                    search="ray_full", nrays=nrays, precision=precision, want_trace=True)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def oracle_full(w, nrays):
    return oracle.predict(w.X, w.Y, w.Xref, w.n0, w.n, w.nc, w.theta, w.g, "ray", nrays=nrays,
                          nthreads=0, snap="design")


def test_fp64_full_scope_dense_2d(lagp):
    w = W.dense_2d(M=100)
    w.nc = 100                      # a short candidate list: the snap often leaves it
    g = run_full(lagp, w, "fp64", 2)
    o = oracle_full(w, 2)
    ident, _ = assert_fp64_parity(g, o, w.n0, w.M)
    assert ident >= w.M - 2
    np.testing.assert_array_equal(g["nevals"][:, : w.n - w.n0], o["nevals"][:, : w.n - w.n0])
    cand_only = oracle.predict(w.X, w.Y, w.Xref, w.n0, w.n, w.nc, w.theta, w.g, "ray",
                               nrays=2, nthreads=0)
    assert not np.array_equal(o["selected"], cand_only["selected"])


@pytest.mark.parametrize("N,nc", [(30, 30), (33, 33), (64, 50), (1000, 60)])
def test_fp64_full_scope_tree_sizes(lagp, N, nc):
    """A single leaf (N <= 32), one split (N = 33), and small trees."""
    w = W.small(N=N, p=2, M=5, n0=3, n=min(12, nc - 2), nc=nc, theta=0.05, g=1e-4, seed=N,
                nrays=2)
    g = run_full(lagp, w, "fp64", 2)
    o = oracle_full(w, 2)
    ident, _ = assert_fp64_parity(g, o, w.n0, w.M)
    assert ident >= w.M - 1


def test_fp64_full_scope_exact_ties(lagp):
    w = W.small(N=300, p=2, M=6, n0=3, n=14, nc=40, theta=0.05, g=1e-4, seed=15, nrays=2)
    w.X, w.Y, w.N = np.vstack([w.X, w.X]), np.concatenate([w.Y, w.Y]), 600
    g = run_full(lagp, w, "fp64", 2)
    o = oracle_full(w, 2)
    ident, _ = assert_fp64_parity(g, o, w.n0, w.M)
    assert ident == w.M


def test_fp64_full_scope_paper_scale_4d_sample(lagp):
    w = _sample(W.paper_scale_4d(M=10000), 32)
    g = run_full(lagp, w, "fp64", 4)
    o = oracle_full(w, 4)
    ident, _ = assert_fp64_parity(g, o, w.n0, w.M)
    assert ident >= w.M - 1


def test_fp32_full_scope_large_8d_sample(lagp):
    """All 100,000 locations of the 8-d workload in one call; 400 evenly spaced
    ones against the oracle (whose unlimited snap scans the 1e6 points)."""
    import torch
    w = W.large_8d(M=100_000)
    out = lagp.predict(to_dev(w.X), to_dev(w.Y), to_dev(w.Xref), w.n0, w.n, w.nc, w.theta, w.g,
                       search="ray_full", nrays=8, precision="fp32", want_trace=True)
    torch.cuda.synchronize()
    idx = np.linspace(0, w.M - 1, 400).astype(int)
    g = {k: v.cpu().numpy()[idx] for k, v in out.items()}
    s = _sample(w, 400)
    o = oracle_full(s, 8)
    check_fp32_form(s, g, o, rmse_tol=None, max_gap=1e-3, first_step_gap=1e-3)


def test_full_scope_solo_equals_batch(lagp):
    """A location's result does not depend on the others in its call."""
    import torch
    w = W.small(N=5000, p=3, M=20, n0=4, n=16, nc=60, theta=0.2, g=1e-6, seed=9, nrays=3)
    X, Y, Xr = to_dev(w.X), to_dev(w.Y), to_dev(w.Xref)
    full = lagp.predict(X, Y, Xr, w.n0, w.n, w.nc, w.theta, w.g, search="ray_full", nrays=3,
                        precision="fp32", want_trace=True)
    for m in (0, 7, 19):
        one = lagp.predict(X, Y, Xr[m:m + 1].contiguous(), w.n0, w.n, w.nc, w.theta, w.g,
                           search="ray_full", nrays=3, precision="fp32", want_trace=True)
        torch.cuda.synchronize()
        assert torch.equal(one["selected"][0], full["selected"][m])
        assert torch.equal(one["mean"][0], full["mean"][m])
