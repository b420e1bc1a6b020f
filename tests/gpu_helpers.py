"""Helpers shared by the GPU parity tests: device copies, sampled workloads and
the checks of the FP32-scoring form against the oracle."""
import numpy as np

from paper_1409_0074_gb300 import workloads as W


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _sample(w, M):
    s = W.Workload(**{k: getattr(w, k) for k in ("name", "N", "p", "M", "n0", "n", "nc",
                                                 "theta", "g", "search", "nrays", "response")})
    s.X, s.Y = w.X, w.Y
    idx = np.linspace(0, w.M - 1, M).astype(int)
    s.Xref, s.Ytrue, s.M = w.Xref[idx], w.Ytrue[idx], M
    return s


def _kriging_on_design(w, sel, m):
    """numpy kriging (Eq. predgp, preds2) on a given local design: the GPU's
    FP64 factor update and predictive equations must reproduce it for
    whatever design its FP32 scores chose."""
    from scipy.spatial.distance import cdist
    sel = sel[sel >= 0]
    S, yS, x = w.X[sel], w.Y[sel], w.Xref[m]
    K = np.exp(-cdist(S, S, "sqeuclidean") / w.theta) + w.g * np.eye(len(sel))
    k = np.exp(-cdist(S, x[None], "sqeuclidean") / w.theta)[:, 0]
    Ki_y = np.linalg.solve(K, yS)
    Ki_k = np.linalg.solve(K, k)
    return k @ Ki_y, (yS @ Ki_y) * ((1 + w.g) - k @ Ki_k) / len(sel), np.linalg.cond(K)


def rmse_ratio(g_mean, o_mean, ytrue):
    """RMSE ratio (GPU / oracle) over paired locations and its standard error
    (delta method on the two mean squared errors)."""
    eg, eo = (g_mean - ytrue) ** 2, (o_mean - ytrue) ** 2
    r2 = eg.mean() / eo.mean()
    se_r2 = np.sqrt(np.var(eg - r2 * eo, ddof=1) / len(eg)) / eo.mean()
    r = np.sqrt(r2)
    return r, se_r2 / (2 * r)


def check_fp32_form(w, g, o, rmse_tol, max_gap, first_step_gap=None):
    # predictive equations on the GPU's own design (FP64 update + predict)
    for m in range(0, w.M, max(1, w.M // 25)):
        mu, s2, cond = _kriging_on_design(w, g["selected"][m], m)
        assert abs(g["mean"][m] - mu) <= 1e-13 * cond * max(1.0, abs(mu)), (m, g["mean"][m], mu)
        assert abs(g["s2"][m] - s2) <= 1e-13 * cond * abs(s2), (m, g["s2"][m], s2)
    # where designs coincide, s2 agrees to 1e-4
    same = np.all(g["selected"] == o["selected"], axis=1)
    if same.any():
        rel = np.abs(g["s2"][same] - o["s2"][same]) / o["s2"][same]
        assert np.all(rel <= 1e-4), rel.max()
    # out-of-sample accuracy: the RMSE ratio over the sampled locations (the
    # point estimate; callers size the sample so that it is a few tenths of a
    # percent from the ratio over the whole workload)
    r, se = rmse_ratio(g["mean"], o["mean"], w.Ytrue)
    if rmse_tol is not None:
        assert r <= 1 + rmse_tol, (r, se)
    # a design first departs from the oracle's only where the oracle's own
    # decision was close (FP32 scores resolve relative gaps of about 1e-4)
    gaps, first = [], []
    for m in range(w.M):
        d = np.nonzero(g["selected"][m] != o["selected"][m])[0]
        if len(d):
            assert d[0] >= w.n0
            gaps.append(o["gap"][m, d[0] - w.n0])
            if d[0] == w.n0:
                first.append(o["gap"][m, 0])
    if max_gap is not None and gaps:
        assert max(gaps) < max_gap, max(gaps)
    # the first greedy step scores against the same well-conditioned K_n0
    if first_step_gap is not None and first:
        assert max(first) < first_step_gap, max(first)
    return r, se, same.mean()
