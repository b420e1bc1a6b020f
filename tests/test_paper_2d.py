"""The 2-d experiment of Sec 5.1, the one workload the paper specifies in full
(CPU only): the generator against the figure the paper prints for it, the
predictive grid's placement, and the oracle's accuracy on it.

Accuracy is context, not parity: the paper estimates theta locally and its
nugget is not stated, so its RMSE column (0.0008-0.0010 at n = 50) is quoted
beside ours in the design notes, not asserted."""
import os

import numpy as np

import oracle
from paper_1409_0074_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_response_matches_the_printed_mean_only_rmse():
    want = float([l for l in open(os.path.join(GOLDEN, "paper_2d_mean_only_rmse.txt"))
                  if l.strip() and not l.startswith("#")][0])
    w = W.paper_2d()
    assert w.N == 201 * 201 and w.M == 99 * 99 and w.p == 2 and w.nrays == 1
    got = float(np.sqrt(np.mean((w.Y - w.Y.mean()) ** 2)))
    assert abs(got - want) <= 0.5e-4, got


def test_design_and_predictive_grids():
    w = W.paper_2d()
    axis = np.unique(w.X[:, 0])
    assert axis.size == 201 and axis[0] == -2.0 and axis[-1] == 2.0
    np.testing.assert_allclose(np.diff(axis), 0.02, atol=1e-12)
    # every predictive coordinate lies midway between two design coordinates
    for k in range(2):
        d = np.min(np.abs(w.Xref[:, k][:, None] - axis[None, :]), axis=1)
        np.testing.assert_allclose(d, 0.01, atol=1e-9)
    # a sample is a subset of the full predictive grid
    s = W.paper_2d(M=50)
    full = {tuple(r) for r in np.round(w.Xref, 9)}
    assert all(tuple(r) in full for r in np.round(s.Xref, 9))


def test_orderings_of_table_1_with_local_inference_for_theta():
    """On a sample of the predictive grid, with local inference for theta as
    the paper runs it (Sec 5: one stage, the design at theta0 then theta-hat on
    it; two stages, a second design at theta-hat), n = 50: every greedy design
    beats the 50 nearest neighbours, a second stage beats the first for each
    search, and all are far below the mean-only RMSE -- the orderings of
    Table 1 (left)."""
    w = W.paper_2d(M=48)
    rm = lambda r: float(np.sqrt(np.mean((r["mean"] - w.Ytrue) ** 2)))
    run = lambda n0, search, stages: oracle.predict_mle(
        w.X, w.Y, w.Xref, n0, w.n, w.nc, w.theta, w.g, 1e-3, 10.0, search, nrays=1,
        stages=stages, nthreads=0)
    nn = run(w.n, "exhaustive", 1)
    r = {(s, st): run(w.n0, s, st) for s in ("ray", "exhaustive") for st in (1, 2)}
    assert all(np.all(v["status"] == 0) for v in r.values())
    for s in ("ray", "exhaustive"):
        assert rm(r[(s, 2)]) < rm(r[(s, 1)]) < rm(nn)
    assert max(rm(v) for v in r.values()) < 0.001 * 0.2085
