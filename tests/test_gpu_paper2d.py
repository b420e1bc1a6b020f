"""The 2-d experiment of Sec 5.1 on the GPU, through the C ABI: the gridded
design of 40,401 points, one ray per step, n = 50, N' = 1000.

FP64 form: identical designs and predictions to the oracle on a sample of the
99 x 99 predictive grid, for both searches.  FP32-scoring form: its accuracy
bar (RMSE within 1% of the oracle's), missed by the plain form and met
with precision promotion.  Local inference for theta on the
GPU's designs (one stage, as in Table 1) against the oracle's predict_mle."""
import numpy as np
import pytest

import oracle
from gpu_helpers import check_fp32_form, rmse_ratio, to_dev
from paper_1409_0074_gb300 import workloads as W
from test_gpu_parity import assert_fp64_parity, gpu_run, oracle_run, same_rows

pytestmark = pytest.mark.gpu

TMIN, TMAX = 1e-3, 10.0


@pytest.fixture(scope="module")
def lagp(cuda):
    from paper_1409_0074_gb300 import build
    build.build()
    from paper_1409_0074_gb300 import lagp as L
    L.load()
    return L


@pytest.mark.parametrize("search", ["ray", "exhaustive"])
def test_fp64_paper_2d_sample(lagp, search):
    w = W.paper_2d(M=64)
    g = gpu_run(lagp, w, search, "fp64", nrays=1)
    o = oracle_run(w, search, nrays=1)
    ident, _ = assert_fp64_parity(g, o, w.n0, w.M)
    assert ident >= w.M - 2
    if search == "ray":
        np.testing.assert_array_equal(g["nevals"][:, : w.n - w.n0], o["nevals"][:, : w.n - w.n0])


_ORACLE = {}


def _oracle_2d(w, search):
    """Oracle results of the 1,000-location sample, computed once per search."""
    if search not in _ORACLE:
        _ORACLE[search] = oracle_run(w, search, nrays=1)
    return _ORACLE[search]


@pytest.mark.xfail(reason="FP32 scoring on the dense 2-d grid (neighbour correlations above "
                   "0.999 at theta = 0.5): over 1,000 sampled locations the FP32-form RMSE "
                   "measured 1.16x (ray) and 1.96x (exhaustive) the oracle's", strict=True)
@pytest.mark.parametrize("search", ["ray", "exhaustive"])
def test_fp32_paper_2d_sample(lagp, search):
    w = W.paper_2d(M=1000)
    g = gpu_run(lagp, w, search, "fp32", nrays=1)
    check_fp32_form(w, g, _oracle_2d(w, search), rmse_tol=0.01, max_gap=None)


@pytest.mark.parametrize("search", ["ray", "exhaustive"])
def test_fp32_promoted_paper_2d_sample(lagp, search):
    """The FP32 form with precision promotion: the grid's local designs have
    binary64 pivots below LAGP_PROMOTE_PIVOT, so the locations are re-solved in
    binary64, carry the LAGP_FP64 results and meet the 1% bar."""
    w = W.paper_2d(M=1000)
    g = gpu_run(lagp, w, search, "fp32_promote", nrays=1, want_promoted=True)
    f = gpu_run(lagp, w, search, "fp64", nrays=1)
    assert g["promoted"] >= 0.99 * w.M, g["promoted"]
    assert same_rows(g, f).sum() >= g["promoted"]
    r, se = rmse_ratio(g["mean"], _oracle_2d(w, search)["mean"], w.Ytrue)
    assert r <= 1.01, (r, se)


def test_first_stage_theta_on_the_paper_2d_designs(lagp):
    """Stage 1 of Table 1: the GPU's FP64 ray design at theta0, then theta-hat
    on it by laGP_mle_predict, against the oracle's one-stage driver."""
    import torch
    w = W.paper_2d(M=32)
    X, Y, Xr = to_dev(w.X), to_dev(w.Y), to_dev(w.Xref)
    d = lagp.predict(X, Y, Xr, w.n0, w.n, w.nc, w.theta, w.g, search="ray", nrays=1,
                     precision="fp64", want_trace=True)
    torch.cuda.synchronize()
    o = oracle.predict_mle(w.X, w.Y, w.Xref, w.n0, w.n, w.nc, w.theta, w.g, TMIN, TMAX,
                           search="ray", nrays=1, stages=1, nthreads=0)
    np.testing.assert_array_equal(d["selected"].cpu().numpy(), o["selected"])
    r = lagp.mle_predict(X, Y, Xr, d["selected"], w.theta, w.g, TMIN, TMAX)
    np.testing.assert_allclose(r["theta"].cpu().numpy(), o["theta"], rtol=1e-8)
    np.testing.assert_allclose(r["mean"].cpu().numpy(), o["mean"], rtol=1e-6, atol=1e-9)
