"""Pins of the pre-scaling oracle (oracle/sep_mle.py, Sec 5.3): the separable
global likelihood against the isotropic C oracle and finite differences, the
BFGS maximiser against a library optimiser and an exact scaling property."""
import math

import numpy as np
import pytest

import oracle
from oracle import sep_mle as SM


def _data(n=60, p=3, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.random((n, p))
    freq = np.array([0.5, 1.2, 2.0, 0.8, 1.6, 0.3, 1.0, 1.4])[:p]
    y = np.sin(2 * np.pi * X @ freq) + 0.3 * np.prod(X, axis=1)
    return X, y


@pytest.mark.parametrize("t", [0.05, 0.3, 1.7])
def test_equal_lengthscales_reduce_to_the_isotropic_likelihood(t):
    """With theta_k = t for every k the separable model is the isotropic one:
    its value equals the C oracle's loglik and its gradient components sum to
    the isotropic derivative (d/dt of l(t, ..., t))."""
    X, y = _data()
    l, gr = SM.sep_loglik(X, y, np.full(3, t), 1e-6)
    li, d1, _ = oracle.loglik(X, y, t, 1e-6)
    assert abs(l - li) <= 1e-9 * max(1.0, abs(li))
    assert abs(gr.sum() - d1) <= 1e-7 * max(1.0, abs(d1))


def test_gradient_matches_central_differences():
    X, y = _data(p=3, seed=2)
    th = np.array([0.2, 0.9, 0.45])
    _, gr = SM.sep_loglik(X, y, th, 1e-6)
    for k in range(3):
        h = 1e-4 * th[k]           # truncation error ~h^2; smaller steps meet rounding in l
        e = np.zeros(3)
        e[k] = h
        fd = (SM.sep_loglik(X, y, th + e, 1e-6)[0] - SM.sep_loglik(X, y, th - e, 1e-6)[0]) / (2 * h)
        assert abs(fd - gr[k]) <= 1e-6 * max(1.0, abs(gr[k])), (k, fd, gr[k])


def test_not_positive_definite_gives_nan():
    X = np.zeros((5, 2))            # coincident rows, no nugget: K singular
    l, gr = SM.sep_loglik(X, np.arange(5.0), np.ones(2), 0.0)
    assert math.isnan(l) and np.all(np.isnan(gr))


def test_bfgs_maximiser_agrees_with_a_library_optimiser():
    """BFGS of reading P2 and scipy's L-BFGS-B (another algorithm) reach the
    same interior maximiser, where the gradient vanishes."""
    from scipy.optimize import minimize
    X, y = _data(n=80, p=3, seed=4)
    th, it, ev, l = SM.sep_mle(X, y, 1e-6, 0.5, 1e-3, 10.0)
    assert 1 < it < 200 and ev >= it

    def f(eta):
        v, gr = SM.sep_loglik(X, y, np.exp(eta), 1e-6)
        return -v, -gr * np.exp(eta)
    r = minimize(f, np.log(np.full(3, 0.5)), jac=True, method="L-BFGS-B",
                 bounds=[(math.log(1e-3), math.log(10.0))] * 3,
                 options=dict(ftol=1e-15, gtol=1e-12, maxiter=1000))
    np.testing.assert_allclose(th, np.exp(r.x), rtol=1e-4)
    assert l >= -r.fun - 1e-9 * abs(r.fun)
    _, gr = SM.sep_loglik(X, y, th, 1e-6)
    assert np.all(np.abs(gr * th) <= 1e-5 * (1 + abs(l)))


def test_lengthscales_scale_with_the_inputs():
    """Multiplying input column k by c multiplies the correlation's
    (x_ak - x_bk)^2 by c^2, so the maximiser's theta_k scales by c^2 exactly
    (the others are unchanged)."""
    X, y = _data(n=70, p=3, seed=6)
    th, *_ = SM.sep_mle(X, y, 1e-6, 0.5, 1e-4, 100.0, tol=1e-11)
    Xs = X.copy()
    Xs[:, 1] *= 3.0
    ts, *_ = SM.sep_mle(Xs, y, 1e-6, th * np.array([1.0, 9.0, 1.0]), 1e-4, 100.0, tol=1e-11)
    np.testing.assert_allclose(ts, th * np.array([1.0, 9.0, 1.0]), rtol=1e-6)


def test_box_bounds_hold():
    """A maximiser outside the box is returned on its face."""
    X, y = _data(n=50, p=2, seed=8)
    th, *_ = SM.sep_mle(X, y, 1e-6, 0.05, 1e-3, 0.06)
    assert np.all(th >= 1e-3 * (1 - 1e-12)) and np.all(th <= 0.06 * (1 + 1e-12))
    assert np.any(np.isclose(th, 0.06, rtol=1e-12))


def test_prescale_is_division_by_root_lengthscales():
    X, _ = _data(n=10, p=3)
    th = np.array([0.25, 4.0, 1.0])
    np.testing.assert_array_equal(SM.prescale(X, th), X / np.array([0.5, 2.0, 1.0]))
