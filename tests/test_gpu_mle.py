"""Local inference for the lengthscale on the GPU (laGP_mle_predict, through
the C ABI) against the FP64 oracle's predict_mle: on the FP64 form's designs
(bit-identical to the oracle's), the estimate within 1e-8 relative (both stop
at a 1e-10 relative step of the same safeguarded Newton iteration; their sums
run in different orders) and the prediction at it within the kriging error
bound 1e-13 cond(K) plus 1e-7 relative for the estimates' difference; a second stage (one design call per location at its own
estimate) against the oracle's two-stage driver; a bad design index and the
largest design size."""
import numpy as np
import pytest

import oracle
from gpu_helpers import to_dev
from paper_1409_0074_gb300 import workloads as W

pytestmark = pytest.mark.gpu

G, TMIN, TMAX = 1e-6, 1e-3, 2.0


@pytest.fixture(scope="module")
def lagp(cuda):
    from paper_1409_0074_gb300 import build
    build.build()
    from paper_1409_0074_gb300 import lagp as L
    L.load()
    return L


def _cond_bounds(X, Y, sel, x, theta, g):
    from scipy.spatial.distance import cdist
    S, yS = X[sel], Y[sel]
    K = np.exp(-cdist(S, S, "sqeuclidean") / theta) + g * np.eye(len(sel))
    cond = np.linalg.cond(K)
    psi = yS @ np.linalg.solve(K, yS)
    return 1e-13 * cond, psi / len(sel) * 1e-13 * cond


def _design_fp64(L, w, Xref, theta, n, nc):
    import torch
    out = L.predict(to_dev(w.X), to_dev(w.Y), to_dev(Xref), w.n0, n, nc, theta, w.g,
                    search="exhaustive", precision="fp64", want_trace=True)
    torch.cuda.synchronize()
    return out["selected"]


def _check(w, Xref, g_out, o, sel):
    th = g_out["theta"].cpu().numpy()
    mean = g_out["mean"].cpu().numpy()
    s2 = g_out["s2"].cpu().numpy()
    np.testing.assert_allclose(th, o["theta"], rtol=1e-8)
    for m in range(len(Xref)):
        # rounding of the two K^{-1} (1e-13 cond) plus the estimates' allowed
        # 1e-8 relative difference carried into the prediction (1e-7)
        rel, s2_err = _cond_bounds(w.X, w.Y, sel[m], Xref[m], o["theta"][m], w.g)
        mo, so = o["mean"][m], o["s2"][m]
        assert abs(mean[m] - mo) <= rel * max(1.0, abs(mo)) + 1e-7 * abs(mo) + 1e-10, m
        assert abs(s2[m] - so) <= s2_err + 1e-7 * abs(so), m


@pytest.mark.parametrize("name", ["dense_2d", "paper_4d"])
def test_first_stage_matches_the_oracle(lagp, name):
    if name == "dense_2d":
        w = W.dense_2d()
        Xref, n, nc = w.Xref[:40], w.n, w.nc
    else:
        w = W.paper_scale_4d()
        Xref, n, nc = w.Xref[:16], w.n, w.nc
    sel = _design_fp64(lagp, w, Xref, w.theta, n, nc)
    o = oracle.predict_mle(w.X, w.Y, Xref, w.n0, n, nc, w.theta, w.g, TMIN, TMAX, stages=1,
                           nthreads=0)
    np.testing.assert_array_equal(sel.cpu().numpy(), o["selected"])
    g_out = lagp.mle_predict(to_dev(w.X), to_dev(w.Y), to_dev(Xref), sel, w.theta, w.g, TMIN,
                             TMAX)
    _check(w, Xref, g_out, o, o["selected"])
    it = g_out["iters"].cpu().numpy()
    assert (it >= 1).all() and (it <= 200).all()


def test_second_stage_matches_the_oracle(lagp):
    """Stage 2 redesigns at the first-stage estimate.  The designs are driven by
    the oracle's first-stage estimates (the GPU's agree to 1e-8, checked
    here), so that both sides redesign at the same theta bit for bit."""
    w = W.dense_2d()
    Xref = w.Xref[:4]
    import torch
    sel1 = _design_fp64(lagp, w, Xref, w.theta, w.n, w.nc)
    s1 = lagp.mle_predict(to_dev(w.X), to_dev(w.Y), to_dev(Xref), sel1, w.theta, w.g, TMIN,
                          TMAX)
    o1 = oracle.predict_mle(w.X, w.Y, Xref, w.n0, w.n, w.nc, w.theta, w.g, TMIN, TMAX, stages=1)
    np.testing.assert_allclose(s1["theta"].cpu().numpy(), o1["theta"], rtol=1e-8)
    th1 = o1["theta"]
    sel2 = torch.cat([_design_fp64(lagp, w, Xref[m:m + 1], float(th1[m]), w.n, w.nc)
                      for m in range(len(Xref))])
    g2 = {k: [] for k in ("theta", "mean", "s2")}
    for m in range(len(Xref)):
        r = lagp.mle_predict(to_dev(w.X), to_dev(w.Y), to_dev(Xref[m:m + 1]), sel2[m:m + 1],
                             float(th1[m]), w.g, TMIN, TMAX)
        for k in g2:
            g2[k].append(r[k])
    g2 = {k: torch.cat(v) for k, v in g2.items()}
    o = oracle.predict_mle(w.X, w.Y, Xref, w.n0, w.n, w.nc, w.theta, w.g, TMIN, TMAX, stages=2)
    np.testing.assert_array_equal(sel2.cpu().numpy(), o["selected"])
    _check(w, Xref, g2, o, o["selected"])


def test_bad_index_and_largest_design(lagp):
    import torch
    w = W.paper_scale_4d()
    Xref = w.Xref[:3]
    sel = _design_fp64(lagp, w, Xref, w.theta, 64, 500)
    o = oracle.predict_mle(w.X, w.Y, Xref, w.n0, 64, 500, w.theta, w.g, TMIN, TMAX, stages=1)
    r = lagp.mle_predict(to_dev(w.X), to_dev(w.Y), to_dev(Xref), sel, w.theta, w.g, TMIN, TMAX)
    _check(w, Xref, r, o, o["selected"])
    bad = sel.clone()
    bad[1, 5] = w.N          # out of range: that location is NaN, the others unaffected
    M = len(Xref)
    out = [torch.empty(M, dtype=torch.float64, device="cuda") for _ in range(3)]
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    lagp.laGP_mle_predict(to_dev(w.X), to_dev(w.Y), to_dev(Xref), bad, w.theta, w.g, TMIN, TMAX,
                          out[0], out[1], out[2], st)
    torch.cuda.synchronize()
    assert int(st.cpu()[0]) == 4           # LAGP_STATUS_NUMERIC
    th = out[0].cpu().numpy()
    assert np.isnan(th[1]) and np.isfinite(th[[0, 2]]).all()
    np.testing.assert_allclose(th[[0, 2]], o["theta"][[0, 2]], rtol=1e-8)
    # no locations: nothing to do
    lagp.laGP_mle_predict(to_dev(w.X), to_dev(w.Y), to_dev(Xref[:0]), sel[:0], w.theta, w.g,
                          TMIN, TMAX, out[0][:0], out[1][:0], out[2][:0], st)


@pytest.mark.parametrize("name,search", [("dense_2d", "exhaustive"), ("dense_2d", "ray"),
                                         ("paper_2d", "ray")])
def test_one_call_stages_match_the_oracle(lagp, name, search):
    """laGP_build_and_predict_mle: the design, the estimate and, for two
    stages, the redesign at each location's own estimate, all in one call
    (per-location theta inside the design kernels).
    Stage 1 against the oracle's predict_mle: identical designs (FP64 form),
    the estimate to 1e-8.  Stage 2 redesigns at the GPU's own first estimate,
    which differs from the oracle's in the eighth digit -- at these workloads
    a relative change of theta that small already moves most greedy designs
    (the oracle's rounding-noise runs move them with 1 ulp) -- so stage 2 is
    checked against the oracle's design at the GPU's first estimate, location
    by location: identical designs, then the estimate on it started there."""
    w = W.dense_2d() if name == "dense_2d" else W.paper_2d(M=24)
    Xref = w.Xref[:24]
    nr = 1 if name == "paper_2d" else 2
    X, Y, Xr = to_dev(w.X), to_dev(w.Y), to_dev(Xref)
    tmax = 10.0 if name == "paper_2d" else TMAX
    run = lambda stages: lagp.predict_mle(X, Y, Xr, w.n0, w.n, w.nc, w.theta, w.g, TMIN, tmax,
                                          stages=stages, search=search, nrays=nr,
                                          precision="fp64", want_selected=True)
    g1, g2 = run(1), run(2)
    o1 = oracle.predict_mle(w.X, w.Y, Xref, w.n0, w.n, w.nc, w.theta, w.g, TMIN, tmax,
                            search=search, nrays=nr, stages=1, nthreads=0)
    np.testing.assert_array_equal(g1["selected"].cpu().numpy(), o1["selected"])
    th1 = g1["theta"].cpu().numpy()
    np.testing.assert_allclose(th1, o1["theta"], rtol=1e-8)
    sel2 = g2["selected"].cpu().numpy()
    th2, mean2, s22 = (g2[k].cpu().numpy() for k in ("theta", "mean", "s2"))
    for m in range(len(Xref)):
        d = oracle.predict(w.X, w.Y, Xref[m:m + 1], w.n0, w.n, w.nc, float(th1[m]), w.g, search,
                           nrays=nr)
        np.testing.assert_array_equal(sel2[m], d["selected"][0])
        S, yS = w.X[sel2[m]], w.Y[sel2[m]]
        t2, _ = oracle.mle_theta(S, yS, float(th1[m]), w.g, TMIN, tmax)
        assert abs(th2[m] - t2) <= 1e-8 * t2, (m, th2[m], t2)
        rel, s2_err = _cond_bounds(w.X, w.Y, sel2[m], Xref[m], t2, w.g)
        # the prediction at the GPU's estimate against numpy kriging there
        from scipy.spatial.distance import cdist
        K = np.exp(-cdist(S, S, "sqeuclidean") / th2[m]) + w.g * np.eye(len(S))
        k = np.exp(-cdist(S, Xref[m][None], "sqeuclidean") / th2[m])[:, 0]
        mu = k @ np.linalg.solve(K, yS)
        v = (yS @ np.linalg.solve(K, yS)) * ((1 + w.g) - k @ np.linalg.solve(K, k)) / len(S)
        assert abs(mean2[m] - mu) <= rel * max(1.0, abs(mu)) + 1e-10, m
        assert abs(s22[m] - v) <= s2_err + 1e-9 * abs(v), m
