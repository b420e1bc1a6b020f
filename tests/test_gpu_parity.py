"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 form: the selected-index sequences must equal the oracle's, except at a
step the oracle logged as a near-tie (relative gap below 1e-12), after which
that location is excused; mean and s2 of the other locations within 1e-10
relative.  (The kernels follow the oracle's operation order, so in practice
every location is bit-identical; the tests report that count.)
FP32-scoring form: s2 within 1e-4 relative at locations whose design equals
the oracle's, and out-of-sample RMSE within 1% of the oracle's (the point
estimate over the sampled locations).  On the 4-d workload, whose K_n reach
condition numbers of ~1e7, the FP32 form misses that bar; those tests are
marked as expected failures with the measured ratios.
kNN: candidate lists bit-exact (indices are integers).
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import _sample, check_fp32_form, rmse_ratio, to_dev
from paper_1409_0074_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TIE_TOL = 1e-12


@pytest.fixture(scope="module")
def lagp(cuda):
    from paper_1409_0074_gb300 import build
    build.build()
    from paper_1409_0074_gb300 import lagp as L
    L.load()
    return L


def gpu_run(L, w, search, precision, nrays=None, n_arr=None, nc_arr=None, want_promoted=False):
    """GPU results as numpy arrays (with want_promoted, also the int
    "promoted": locations the FP32 form re-solved in binary64)."""
    import torch
    n = int(max(w.n, n_arr.max() if n_arr is not None else 0))
    nc = int(max(w.nc, nc_arr.max() if nc_arr is not None else 0))
    out = L.predict(to_dev(w.X), to_dev(w.Y), to_dev(w.Xref), w.n0, n, nc, w.theta, w.g,
                    search=search, nrays=w.nrays if nrays is None else nrays,
                    precision=precision,
                    n_loc=to_dev(n_arr, torch.int32) if n_arr is not None else None,
                    nclose_loc=to_dev(nc_arr, torch.int32) if nc_arr is not None else None,
                    want_trace=True, want_promoted=want_promoted)
    torch.cuda.synchronize()
    return {k: (v if isinstance(v, int) else v.cpu().numpy()) for k, v in out.items()}


def same_rows(a, b):
    """Locations whose design, mean and s2 are bit-identical in two results."""
    return (np.all(a["selected"] == b["selected"], axis=1) &
            (a["mean"].view(np.int64) == b["mean"].view(np.int64)) &
            (a["s2"].view(np.int64) == b["s2"].view(np.int64)))


def oracle_run(w, search, nrays=None, n_arr=None, nc_arr=None):
    n = int(max(w.n, n_arr.max() if n_arr is not None else 0))
    nc = int(max(w.nc, nc_arr.max() if nc_arr is not None else 0))
    return oracle.predict(w.X, w.Y, w.Xref, w.n0, n, nc, w.theta, w.g, search,
                          nrays=w.nrays if nrays is None else nrays, n_arr=n_arr, nc_arr=nc_arr,
                          nthreads=0)


def assert_fp64_parity(g, o, n0, M, max_excused_frac=0.05):
    """Returns (bit-identical locations, excused locations)."""
    identical, excused = 0, 0
    for m in range(M):
        sg, so = g["selected"][m], o["selected"][m]
        if np.array_equal(sg, so):
            mo, mg = o["mean"][m], g["mean"][m]
            assert abs(mg - mo) <= 1e-10 * max(abs(mo), 1e-300), (m, mg, mo)
            assert abs(g["s2"][m] - o["s2"][m]) <= 1e-10 * abs(o["s2"][m]), m
            if (mg == mo and g["s2"][m] == o["s2"][m]
                    and np.array_equal(g["tie_gap"][m], o["gap"][m])):
                identical += 1
            continue
        t = int(np.argmax(sg != so))
        assert t >= n0, ("start (kNN) differs", m, t)
        gap = o["gap"][m, t - n0]
        assert gap < TIE_TOL, ("unexcused divergence", m, t, gap)
        excused += 1
    assert excused <= max_excused_frac * M
    return identical, excused


# --- kNN -------------------------------------------------------------------------

def knn_gpu(L, X, Xref, nc):
    import torch
    N, p = X.shape
    M = Xref.shape[0]
    ws = torch.empty(L.laGP_knn_workspace_bytes(N, p, M, nc), dtype=torch.uint8, device="cuda")
    cand = torch.empty((M, nc), dtype=torch.int32, device="cuda")
    L.laGP_knn(to_dev(X), to_dev(Xref), nc, cand, ws)
    rc, st = L.laGP_status(ws)
    assert rc == 0, st
    return cand.cpu().numpy()


@pytest.mark.parametrize("p,N,M,nc", [(1, 3001, 37, 200), (3, 5000, 70, 300), (8, 9999, 33, 1000),
                                      (13, 4097, 5, 700), (4, 257, 3, 257), (8, 12345, 97, 256),
                                      (2, 20000, 40, 4096)])
def test_knn_bit_exact(lagp, p, N, M, nc):
    rng = np.random.default_rng(p * 7 + N)
    X = rng.random((N, p))
    Xref = rng.random((M, p)) * 1.2 - 0.1          # some outside the design's box
    cand = knn_gpu(lagp, X, Xref, nc)
    for m in range(M):
        idx, _ = oracle.knn(X, Xref[m], nc)
        np.testing.assert_array_equal(cand[m], idx)


def test_knn_pilot_threshold_failure_is_streamed_again(lagp):
    """For N >= 32 N' the stream starts from a threshold estimated on the
    stride sample of rows i * (N / S).  Here those rows are exactly the points
    clustered at the locations, so the estimate is far too tight; the check at
    the end of the stream must catch it and the location must be streamed
    again: the candidate lists still equal the oracle's."""
    rng = np.random.default_rng(21)
    N, p, nc, M = 40000, 3, 1000, 24
    X = rng.random((N, p)) * 10.0                    # far away
    S = min(16384, N // 16)
    rows = np.arange(S) * (N // S)
    X[rows] = 5.0 + 0.05 * rng.standard_normal((S, p))   # sampled rows: a tight cluster
    Xref = 5.0 + 0.05 * rng.standard_normal((M, p))
    cand = knn_gpu(lagp, X, Xref, nc)
    for m in range(M):
        idx, _ = oracle.knn(X, Xref[m], nc)
        np.testing.assert_array_equal(cand[m], idx)


def test_knn_large_design_uneven_nclose(lagp):
    """Pilot thresholds with per-location N' (the uneven workload's kNN)."""
    import torch
    rng = np.random.default_rng(8)
    N, p, M = 300000, 8, 40
    X = rng.random((N, p))
    Xref = rng.random((M, p))
    ncl = rng.integers(300, 2001, M).astype(np.int32)
    nmax = int(ncl.max())
    Y = np.zeros(N)
    out = lagp.predict(to_dev(X), to_dev(Y), to_dev(Xref), 6, 20, nmax, 1.0, 1e-6,
                       search="exhaustive", precision="fp32", want_trace=True,
                       n_loc=to_dev(np.full(M, 20, np.int32), torch.int32),
                       nclose_loc=to_dev(ncl, torch.int32))
    torch.cuda.synchronize()
    sel = out["selected"].cpu().numpy()
    for m in range(M):
        idx, _ = oracle.knn(X, Xref[m], int(ncl[m]))
        np.testing.assert_array_equal(sel[m, :6], idx[:6])     # the n0 nearest start the design
        assert set(sel[m][sel[m] >= 0]) <= set(idx.tolist())   # every pick is a candidate


@pytest.mark.parametrize("M", [1, 7, 130])
def test_knn_small_batches_split_the_design(lagp, M):
    """Batches with fewer location tiles than SMs split the design's tiles into
    segments, one CTA each, appending to the locations' buffers through a
    counter: the candidate lists stay bit-exact."""
    rng = np.random.default_rng(40 + M)
    X = rng.random((300_000, 8))
    Xref = rng.random((M, 8))
    cand = knn_gpu(lagp, X, Xref, 1000)
    for m in range(M):
        idx, _ = oracle.knn(X, Xref[m], 1000)
        np.testing.assert_array_equal(cand[m], idx)


def test_knn_small_batch_on_the_ordered_grid(lagp):
    """On the 2-d grid design (rows in index order, so a location's neighbours
    lie in one or two design segments) with a small batch."""
    w = W.paper_2d(M=5)
    cand = knn_gpu(lagp, w.X, w.Xref, 1000)
    for m in range(w.M):
        idx, _ = oracle.knn(w.X, w.Xref[m], 1000)
        np.testing.assert_array_equal(cand[m], idx)


def test_knn_exact_ties_go_to_lower_index(lagp):
    rng = np.random.default_rng(5)
    X = rng.integers(0, 7, (6000, 3)).astype(np.float64)   # many duplicates and ties
    Xref = rng.integers(0, 7, (20, 3)).astype(np.float64) + 0.5 * (rng.random((20, 3)) < 0.5)
    cand = knn_gpu(lagp, X, Xref, 300)
    for m in range(20):
        idx, _ = oracle.knn(X, Xref[m], 300)
        np.testing.assert_array_equal(cand[m], idx)


# --- FP64 form ---------------------------------------------------------------------

@pytest.mark.parametrize("search", ["exhaustive", "ray"])
def test_fp64_dense_2d_full(lagp, search):
    """The 2-d workload in full: N = 4000, M = 100, n = 30, N' = 500."""
    w = W.dense_2d(M=100)
    g = gpu_run(lagp, w, search, "fp64", nrays=2)
    o = oracle_run(w, search, nrays=2)
    ident, exc = assert_fp64_parity(g, o, w.n0, w.M)
    assert ident >= 0.95 * w.M
    if search == "ray":
        np.testing.assert_array_equal(g["nevals"][:, : w.n - w.n0], o["nevals"][:, : w.n - w.n0])


@pytest.mark.parametrize("case", [
    dict(N=700, p=1, M=9, n0=3, n=12, nc=40, theta=0.01, g=1e-5, nrays=1),
    dict(N=900, p=3, M=11, n0=5, n=5, nc=50, theta=0.1, g=1e-6, nrays=2),        # n = n0
    dict(N=650, p=2, M=7, n0=4, n=20, nc=20, theta=0.05, g=1e-4, nrays=0),       # N' = n
    dict(N=1300, p=5, M=13, n0=1, n=17, nc=300, theta=0.5, g=1e-8, nrays=5),     # n0 = 1
    dict(N=2000, p=16, M=3, n0=6, n=40, nc=600, theta=4.0, g=1e-6, nrays=16),    # max p, rays
])
@pytest.mark.parametrize("search", ["exhaustive", "ray"])
def test_fp64_edge_cases(lagp, case, search):
    c = dict(case)
    nr = c.pop("nrays")
    if search == "ray" and (nr if nr > 0 else c["p"]) > c["nc"] - c["n"]:
        pytest.skip("nrays > N' - n is outside the valid range")
    w = W.small(seed=3, search=search, nrays=nr, **c)
    g = gpu_run(lagp, w, search, "fp64")
    o = oracle_run(w, search)
    ident, _ = assert_fp64_parity(g, o, w.n0, w.M)
    assert ident >= w.M - 1


def test_fp64_max_local_design(lagp):
    """n = 128 (the largest local design) with 16 rays and N' = 2000."""
    w = W.small(N=6000, p=4, M=2, n0=6, n=128, nc=2000, theta=0.3, g=1e-6, seed=4,
                search="ray", nrays=16)
    g = gpu_run(lagp, w, "ray", "fp64")
    o = oracle_run(w, "ray")
    assert_fp64_parity(g, o, w.n0, w.M, max_excused_frac=0.5)


def test_fp64_duplicate_design_ties(lagp):
    w = W.small(N=400, p=2, M=6, n0=3, n=14, nc=60, theta=0.05, g=1e-4, seed=15)
    w.X, w.Y = np.vstack([w.X, w.X]), np.concatenate([w.Y, w.Y])
    w.N = 800
    for search in ("exhaustive", "ray"):
        g = gpu_run(lagp, w, search, "fp64", nrays=2)
        o = oracle_run(w, search, nrays=2)
        ident, _ = assert_fp64_parity(g, o, w.n0, w.M)
        assert ident == w.M


def test_fp64_uneven_sizes(lagp):
    """Per-location n and N' in one launch."""
    w = W.small(N=3000, p=3, M=24, n0=4, n=40, nc=400, theta=0.2, g=1e-6, seed=21)
    rng = np.random.default_rng(1)
    n_arr = rng.integers(6, 41, w.M).astype(np.int32)
    nc_arr = rng.integers(60, 401, w.M).astype(np.int32)
    for search in ("exhaustive", "ray"):
        g = gpu_run(lagp, w, search, "fp64", nrays=3, n_arr=n_arr, nc_arr=nc_arr)
        o = oracle_run(w, search, nrays=3, n_arr=n_arr, nc_arr=nc_arr)
        for m in range(w.M):
            assert np.all(g["selected"][m, n_arr[m]:] == -1)
        ident, _ = assert_fp64_parity(g, o, w.n0, w.M)
        assert ident >= w.M - 1


def test_fp64_singular_update_reports_nan(lagp):
    """g = 0 with duplicated nearest points: the Schur complement is 0; the
    location gets NaN and the status word says so."""
    import torch
    X = np.array([[0.5, 0.5], [0.5, 0.5], [0.1, 0.9], [0.9, 0.1], [0.2, 0.2], [0.8, 0.8]] * 20)
    X = X + np.repeat(np.arange(20)[:, None] * 1e-3, 6, axis=0)
    Y = np.sin(X[:, 0])
    Xref = np.array([[0.5, 0.5], [0.3, 0.7]])
    o = oracle.predict(X, Y, Xref, 3, 8, 40, 0.1, 0.0, "exhaustive")
    assert np.isnan(o["mean"][0]) and o["status"][0] != 0
    L = lagp
    ws = torch.empty(L.laGP_workspace_bytes(len(X), 2, 2, 8, 40, 0, 0, 0), dtype=torch.uint8,
                     device="cuda")
    mean = torch.empty(2, dtype=torch.float64, device="cuda")
    s2 = torch.empty(2, dtype=torch.float64, device="cuda")
    L.laGP_build_and_predict(to_dev(X), to_dev(Y), to_dev(Xref), 3, 8, 40, 0.1, 0.0, 0, 0, 0,
                             mean, s2, ws)
    rc, st = L.laGP_status(ws)
    assert rc == -4 and st & 4
    m = mean.cpu().numpy()
    assert np.isnan(m[0]) and (np.isnan(o["mean"][1]) == np.isnan(m[1]))


def test_host_buffer_entry_matches_device_entry(lagp):
    import torch
    L = lagp
    w = W.small(N=2500, p=3, M=16, n0=4, n=20, nc=200, theta=0.2, g=1e-6, seed=8)
    dev = gpu_run(L, w, "ray", "fp32", nrays=3)
    wsb = L.laGP_host_workspace_bytes(w.N, w.p, w.M, w.n, w.nc, 3, 1, 1)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    mean, s2 = np.zeros(w.M), np.zeros(w.M)
    sel = np.zeros((w.M, w.n), np.int32)
    L.laGP_build_and_predict_host(w.X, w.Y, w.Xref, w.n0, w.n, w.nc, w.theta, w.g, 1, 3, 1,
                                  mean, s2, ws, selected=sel)
    np.testing.assert_array_equal(sel, dev["selected"])
    np.testing.assert_array_equal(mean, dev["mean"])
    np.testing.assert_array_equal(s2, dev["s2"])


# --- 4-d paper-scale workload, sampled ---------------------------------------------

@pytest.fixture(scope="module")
def paper4d():
    return W.paper_scale_4d(M=10000)


_ORACLE_4D = {}


def _oracle_4d(w, search):
    """Oracle results of the 2,000-location 4-d sample, computed once per search."""
    if search not in _ORACLE_4D:
        _ORACLE_4D[search] = oracle_run(w, search, nrays=4)
    return _ORACLE_4D[search]


@pytest.mark.parametrize("search", ["exhaustive", "ray"])
def test_fp64_paper_scale_4d_sample(lagp, paper4d, search):
    w = _sample(paper4d, 48)
    g = gpu_run(lagp, w, search, "fp64", nrays=4)
    o = oracle_run(w, search, nrays=4)
    ident, _ = assert_fp64_parity(g, o, w.n0, w.M)
    assert ident >= 0.9 * w.M


@pytest.mark.xfail(reason="FP32 scoring at cond(K) ~1e7: over all 10,000 locations of the 4-d "
                   "workload the FP32-form ray RMSE measured 1.3% above the FP64 form's",
                   strict=False)
def test_fp32_score_ray_paper_scale_4d_sample(lagp, paper4d):
    """4-d workload (theta = 0.25, cond K_50 up to ~1e7), checked at the FP32
    form's 1% RMSE bar, which it misses at this conditioning."""
    w = _sample(paper4d, 2000)
    g = gpu_run(lagp, w, "ray", "fp32", nrays=4)
    check_fp32_form(w, g, _oracle_4d(w, "ray"), rmse_tol=0.01, max_gap=1e-3)


@pytest.mark.xfail(reason="FP32 scoring at cond(K) ~1e7: over all 10,000 locations of the 4-d "
                   "workload the FP32 exhaustive RMSE measured 14% (CUDA-core) and 18% "
                   "(tensor-core) above the FP64 form's", strict=True)
@pytest.mark.parametrize("precision", ["fp32", "fp32_tc"])
def test_fp32_score_exhaustive_paper_scale_4d_sample(lagp, paper4d, precision):
    """On the 4-d workload (theta = 0.25, g = 1e-6, cond K up to ~1e7) FP32
    scores cannot rank candidates whose v is below ~1e-5: the FP32 correlation
    values carry errors as large as v.  Checked at the 1% bar, which it misses;
    the design checks of check_fp32_form run before the RMSE assertion."""
    w = _sample(paper4d, 2000)
    g = gpu_run(lagp, w, "exhaustive", precision)
    check_fp32_form(w, g, _oracle_4d(w, "exhaustive"), rmse_tol=0.01, max_gap=None)


@pytest.mark.parametrize("search,precision", [("ray", "fp32_promote"),
                                              ("exhaustive", "fp32_promote"),
                                              ("exhaustive", "fp32_tc_promote")])
def test_fp32_promoted_paper_scale_4d_sample(lagp, paper4d, search, precision):
    """The FP32 forms with precision promotion on the 4-d workload: every
    location's smallest binary64 pivot is below LAGP_PROMOTE_PIVOT, so (nearly)
    all are re-solved in binary64; each promoted location carries exactly the
    LAGP_FP64 result, and the RMSE meets the 1% bar."""
    w = _sample(paper4d, 2000)
    g = gpu_run(lagp, w, search, precision, nrays=4, want_promoted=True)
    f = gpu_run(lagp, w, search, "fp64", nrays=4)
    assert g["promoted"] >= 0.99 * w.M, g["promoted"]
    assert same_rows(g, f).sum() >= g["promoted"]
    r, se = rmse_ratio(g["mean"], _oracle_4d(w, search)["mean"], w.Ytrue)
    assert r <= 1.01, (r, se)


@pytest.fixture(scope="module")
def large8d():
    return W.large_8d(M=100_000)


_ORACLE_8D = {}


def oracle_8d(w, search, n, M_or):
    """Oracle results on M_or evenly spaced locations of the 8-d workload,
    computed once per (search, n) and shared by the forms checked against it."""
    key = (search, n, M_or)
    if key not in _ORACLE_8D:
        s = _sample(w, M_or)
        s.n = n
        _ORACLE_8D[key] = (s, oracle_run(s, search, nrays=8))
    return _ORACLE_8D[key]


@pytest.mark.parametrize("search,n,M_or,precision", [
    ("ray", 50, 2000, "fp32"), ("exhaustive", 50, 2000, "fp32"),
    ("exhaustive", 50, 2000, "fp32_tc"), ("exhaustive", 80, 1000, "fp32")])
def test_fp32_score_large_8d_sample(lagp, large8d, search, n, M_or, precision):
    """The FP32-scoring form on its own workload (N = 1e6, p = 8, theta = 1)
    in the bench's launch configuration (all 100,000 locations in one call),
    checked against the oracle on evenly spaced locations: FP64 predictive
    equations on the form's own design, s2 where the designs coincide, and
    departures only at close oracle decisions.  The RMSE bar itself is checked
    over all 100,000 locations below, free of sampling noise.  Exhaustive
    "fp32" runs the incremental CUDA-core scorer, "fp32_tc" the tensor-core
    contraction (n <= 64)."""
    import torch
    w = large8d
    out = lagp.predict(to_dev(w.X), to_dev(w.Y), to_dev(w.Xref), w.n0, n, w.nc, w.theta, w.g,
                       search=search, nrays=8, precision=precision, want_trace=True)
    torch.cuda.synchronize()
    idx = np.linspace(0, w.M - 1, M_or).astype(int)
    g = {k: v.cpu().numpy()[idx] for k, v in out.items()}
    s, o = oracle_8d(w, search, n, M_or)
    check_fp32_form(s, g, o, rmse_tol=None, max_gap=1e-3 if search == "ray" else None,
                    first_step_gap=1e-3)


def golden_oracle_rmse():
    """The oracle's RMSE over all 100,000 locations of the 8-d workload, per
    search, written by tests/golden/make_oracle_rmse_8d.py (oracle only)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_rmse_sinusoid8d.txt")
    if not os.path.exists(path):
        pytest.skip("the oracle's 100,000-location RMSE file has not been written yet")
    out = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            search, rmse, locs, bad = line.split()
            assert int(locs) == 100_000 and int(bad) == 0
            out[search] = float(rmse)
    return out


@pytest.mark.parametrize("search,precision,tol", [
    ("ray", "fp32", 0.01), ("exhaustive", "fp32", 0.01), ("exhaustive", "fp32_tc", 0.01),
    ("ray", "fp64", 1e-12), ("exhaustive", "fp64", 1e-12)])
def test_rmse_over_the_whole_8d_workload(lagp, large8d, search, precision, tol):
    """The FP32 form's accuracy bar on the workload it is quoted on, over all
    100,000 locations (no sampling): the FP32-scoring form's out-of-sample
    RMSE within 1% of the oracle's; the FP64 form, whose designs are the
    oracle's, equal to it up to rounding."""
    import torch
    w = large8d
    rows = golden_oracle_rmse()
    if search not in rows:
        pytest.skip("the oracle's %s RMSE over 100,000 locations has not been written yet" % search)
    want = rows[search]
    out = lagp.predict(to_dev(w.X), to_dev(w.Y), to_dev(w.Xref), w.n0, w.n, w.nc, w.theta, w.g,
                       search=search, nrays=8, precision=precision)
    torch.cuda.synchronize()
    got = float(np.sqrt(np.mean((out["mean"].cpu().numpy() - w.Ytrue) ** 2)))
    assert got <= want * (1 + tol), (got, want, got / want)
    if precision == "fp64":
        assert abs(got - want) <= tol * want, (got, want)


@pytest.mark.parametrize("search,precision", [("ray", "fp32"), ("exhaustive", "fp32"),
                                              ("exhaustive", "fp32_tc")])
def test_promotion_on_the_whole_8d_workload(lagp, large8d, search, precision):
    """On the 8-d workload the local designs stay well conditioned (smallest
    binary64 pivots around 1e-3): precision promotion re-solves at most 0.1% of
    the 100,000 locations, and every other location is bit-identical to the
    form without it."""
    import torch
    w = large8d
    args = (to_dev(w.X), to_dev(w.Y), to_dev(w.Xref), w.n0, w.n, w.nc, w.theta, w.g)
    a = lagp.predict(*args, search=search, nrays=8, precision=precision + "_promote",
                     want_trace=True, want_promoted=True)
    b = lagp.predict(*args, search=search, nrays=8, precision=precision, want_trace=True,
                     want_promoted=True)
    torch.cuda.synchronize()
    assert b["promoted"] == 0
    assert a["promoted"] <= 0.001 * w.M, a["promoted"]
    na = {k: v.cpu().numpy() for k, v in a.items() if k != "promoted"}
    nb = {k: v.cpu().numpy() for k, v in b.items() if k != "promoted"}
    assert (~same_rows(na, nb)).sum() <= a["promoted"]


@pytest.mark.parametrize("search", ["ray", "exhaustive"])
def test_fp64_large_8d_sample(lagp, large8d, search):
    """Plain FP64 form at N = 1e6, p = 8 on 24 locations: bit-identical, for
    both searches."""
    s = _sample(large8d, 24)
    g = gpu_run(lagp, s, search, "fp64", nrays=8)
    o = oracle_run(s, search, nrays=8)
    ident, _ = assert_fp64_parity(g, o, s.n0, s.M)
    assert ident >= s.M - 1
