"""Pins of the oracle's local inference for the lengthscale (Sec 2.1, Eq. gpk;
Sec 5: Newton-like maximisation of the local posterior, second-stage
re-design), each against something other than the oracle's own formulas:
numerical integration over tau^2 of scipy's multivariate normal density,
finite differences of an independent numpy log-likelihood, scipy's bounded
scalar minimiser, a dense grid, numpy kriging, and lengthscale recovery from
data drawn from a GP with a known lengthscale."""
import numpy as np
import pytest

import oracle

scipy = pytest.importorskip("scipy")
from scipy import integrate, optimize, stats  # noqa: E402
from scipy.spatial.distance import cdist  # noqa: E402


def _K(S, theta, g):
    return np.exp(-cdist(S, S, "sqeuclidean") / theta) + g * np.eye(len(S))


def _loglik_np(S, y, theta, g):
    """Eq. gpk written independently: slogdet and a linear solve."""
    n = len(y)
    K = _K(S, theta, g)
    _, logdet = np.linalg.slogdet(K)
    psi = y @ np.linalg.solve(K, y)
    from math import lgamma, log, pi
    return lgamma(n / 2) - n / 2 * log(2 * pi) - 0.5 * logdet - n / 2 * np.log(psi / 2)


def _case(seed, n=18, p=2):
    rng = np.random.default_rng(seed)
    S = rng.random((n, p))
    y = np.sin(4 * S[:, 0] + 1) + 0.5 * np.cos(3 * S[:, -1]) + 0.2 * S.sum(axis=1)
    return S, y


@pytest.mark.parametrize("seed,theta", [(0, 0.08), (1, 0.3), (2, 1.2)])
def test_marginal_likelihood_equals_the_integral_over_tau2(seed, theta):
    """p(y | theta) = int N(y; 0, tau^2 K) (1 / tau^2) dtau^2 (reference prior
    on tau^2): integrate over s = log tau^2 with scipy's density."""
    g = 1e-4
    S, y = _case(seed, n=8)
    K = _K(S, theta, g)

    def f(s):
        return stats.multivariate_normal.logpdf(y, mean=np.zeros(len(y)), cov=np.exp(s) * K)

    grid = np.linspace(-30, 30, 2001)
    fmax = max(f(s) for s in grid)
    val, _ = integrate.quad(lambda s: np.exp(f(s) - fmax), -30, 30, limit=400,
                            points=[grid[np.argmax([f(s) for s in grid])]])
    want = fmax + np.log(val)
    got, _, _ = oracle.loglik(S, y, theta, g)
    assert got == pytest.approx(want, abs=1e-7)


@pytest.mark.parametrize("seed,theta,g", [(0, 0.05, 1e-6), (3, 0.2, 1e-6), (4, 0.9, 1e-3),
                                          (5, 0.02, 1e-2)])
def test_derivatives_match_finite_differences(seed, theta, g):
    S, y = _case(seed)
    v, d1, d2 = oracle.loglik(S, y, theta, g)
    assert v == pytest.approx(_loglik_np(S, y, theta, g), rel=1e-9, abs=1e-9)
    h = 1e-4 * theta
    lp, l0, lm = (_loglik_np(S, y, theta + h, g), _loglik_np(S, y, theta, g),
                  _loglik_np(S, y, theta - h, g))
    assert d1 == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-6 / theta)
    assert d2 == pytest.approx((lp - 2 * l0 + lm) / (h * h), rel=2e-3, abs=1e-3 / theta ** 2)


def _unimodal_on(S, y, g, lo, hi):
    ts = np.geomspace(lo, hi, 400)
    vals = np.array([_loglik_np(S, y, t, g) for t in ts])
    inner = (vals[1:-1] > vals[:-2]) & (vals[1:-1] > vals[2:])
    return inner.sum() <= 1, ts[np.argmax(vals)]


@pytest.mark.parametrize("seed", range(6))
def test_newton_maximiser_matches_scipy_and_a_grid(seed):
    g, lo, hi = 1e-6, 1e-3, 5.0
    S, y = _case(seed)
    uni, t_grid = _unimodal_on(S, y, g, lo, hi)
    if not uni:
        pytest.skip("several local maxima on this range")
    t_hat, iters = oracle.mle_theta(S, y, 0.1, g, lo, hi)
    res = optimize.minimize_scalar(lambda t: -_loglik_np(S, y, t, g), bounds=(lo, hi),
                                   method="bounded", options={"xatol": 1e-12})
    assert t_hat == pytest.approx(res.x, rel=1e-5)
    assert t_hat == pytest.approx(t_grid, rel=0.03)
    _, d1, d2 = oracle.loglik(S, y, t_hat, g)
    if lo * 1.01 < t_hat < hi * 0.99:
        assert abs(d1) * t_hat < 1e-6 and d2 < 0
        # Newton's quadratic convergence: bisection alone needs ~40 halvings
        # of [lo, hi] to reach the 1e-10 relative tolerance
        assert iters <= 15


def test_maximiser_on_a_bound_returns_the_bound():
    g = 1e-6
    S, y = _case(1)
    t_star, _ = oracle.mle_theta(S, y, 0.1, g, 1e-3, 5.0)
    # the range stops short of the maximiser on either side
    t_hi, _ = oracle.mle_theta(S, y, 0.01, g, 1e-3, 0.5 * t_star)
    t_lo, _ = oracle.mle_theta(S, y, 3.0, g, 2.0 * t_star, 5.0)
    assert t_hi == pytest.approx(0.5 * t_star, rel=1e-8)
    assert t_lo == pytest.approx(2.0 * t_star, rel=1e-8)


def test_lengthscale_recovered_from_gp_draws():
    """y drawn from N(0, K_theta*) on 150 points: the estimate lands near theta*."""
    rng = np.random.default_rng(7)
    S = rng.random((150, 2))
    g = 1e-6
    for t_true in (0.05, 0.2):
        K = _K(S, t_true, 1e-8)
        y = np.linalg.cholesky(K) @ rng.standard_normal(len(S))
        t_hat, _ = oracle.mle_theta(S, y, 0.1, g, 1e-3, 5.0)
        assert 0.7 * t_true < t_hat < 1.4 * t_true


def _kriging(S, yS, x, theta, g):
    """mean, s2 and their error bounds: both errors grow with cond(K), and
    1 + g - k^T K^{-1} k cancels (1e-13 cond, as for the other kriging pins)."""
    K = _K(S, theta, g)
    k = np.exp(-((S - x) ** 2).sum(axis=1) / theta)
    a = np.linalg.solve(K, yS)
    b = np.linalg.solve(K, k)
    n = len(yS)
    psi = yS @ a
    cond = np.linalg.cond(K)
    return k @ a, psi * ((1 + g) - k @ b) / n, psi / n * 1e-13 * cond, 1e-13 * cond


@pytest.mark.parametrize("search,stages", [("exhaustive", 1), ("exhaustive", 2), ("ray", 2)])
def test_two_stage_driver(search, stages):
    """The prediction is kriging at the estimate on the returned design; the
    estimate maximises the likelihood of that design; a second stage is the
    greedy design at the first stage's estimate."""
    rng = np.random.default_rng(11)
    N, p = 3000, 2
    X = rng.random((N, p))
    Y = np.sin(2 * np.pi * 1.3 * X[:, 0] + 0.4) + np.cos(2 * np.pi * 0.7 * X[:, 1])
    Xref = 0.05 + 0.9 * rng.random((5, p))
    n0, n, nc, theta0, g, lo, hi = 6, 24, 300, 0.1, 1e-6, 1e-3, 2.0
    out = oracle.predict_mle(X, Y, Xref, n0, n, nc, theta0, g, lo, hi, search=search,
                             nrays=2, stages=stages)
    assert (out["status"] == 0).all()
    one = oracle.predict_mle(X, Y, Xref, n0, n, nc, theta0, g, lo, hi, search=search,
                             nrays=2, stages=1)
    for m in range(len(Xref)):
        sel = out["selected"][m]
        S, yS = X[sel], Y[sel]
        mu, s2, s2_err, rel = _kriging(S, yS, Xref[m], out["theta"][m], g)
        assert abs(out["mean"][m] - mu) <= rel * max(1.0, abs(mu))
        assert abs(out["s2"][m] - s2) <= s2_err + 1e-9 * abs(s2)
        t_ref, _ = oracle.mle_theta(S, yS, one["theta"][m] if stages == 2 else theta0, g, lo, hi)
        assert out["theta"][m] == pytest.approx(t_ref, rel=1e-9)
    if stages == 2:
        # the second-stage design is the greedy design at the first estimate
        for m in range(len(Xref)):
            d = oracle.predict(X, Y, Xref[m:m + 1], n0, n, nc, one["theta"][m], g, search,
                               nrays=2)
            np.testing.assert_array_equal(d["selected"][0], out["selected"][m])
