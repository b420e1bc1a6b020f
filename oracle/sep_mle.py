"""Pre-scaled inputs (Sec 5.3, the "rays with pre-scaled inputs" columns of
the borehole subset table): a crude global analysis fits a separable Gaussian
correlation to a random subset of the design by maximum likelihood, and every
input coordinate is then divided by the square root of its global lengthscale
before the local approximation runs on the scaled inputs.

TEST INFRASTRUCTURE ONLY: the test suite and the benchmark's CPU-baseline leg
are its only users; the CUDA product path never imports it.  Plain numpy in
binary64, library routines (Cholesky, triangular solves) as single steps.

Readings (the paper gives the idea, not the fitting details):
  P1  the global model is the separable form of Eq. gpk: K_ab =
      exp(-sum_k (x_ak - x_bk)^2 / theta_k) off the diagonal and 1 + g on it
      (g fixed, as for the local designs), with the reference prior on the
      scale, so that the log likelihood is the local one of readings M1-M2
      with a vector theta; a flat prior on theta over [tmin, tmax]^p.
  P2  the maximiser is BFGS on eta = log theta from eta0 = log theta0: inverse
      curvature H = I at the start; ascent direction d = H grad, scaled down
      so that no coordinate moves more than 2; trial points projected on the
      box; step t = 1, 1/2, 1/4, ... (at most 40 halvings) until the Armijo
      condition l(eta_t) >= l(eta) + 1e-4 grad . (eta_t - eta) holds; the BFGS
      update of H is skipped unless s . y > 1e-12 |s| |y| (y the change of the
      negated gradient); stop when an accepted step (or the first trial)
      moves no coordinate of eta by more than tol, or when no halving is
      accepted, or after maxit iterations.
  P3  the scaled inputs are x_k / sqrt(theta_k) for the design and the
      predictive locations alike; on them the separable global correlation is
      the isotropic one with theta = 1.
"""
import math

import numpy as np


def sep_loglik(S, y, theta, g):
    """Log likelihood of the separable model (reading P1) on the rows S
    (n x p) with responses y, and its gradient in theta:
        l = log Gamma(n/2) - (n/2) log(2 pi) - (1/2) log|K| - (n/2) log(psi / 2),
        psi = y^T K^{-1} y,
        dl/dtheta_k = -(1/2) tr(K^{-1} K_k) - (n/2) psi_k / psi,
        psi_k = -alpha^T K_k alpha,  alpha = K^{-1} y,
        K_k,ab = K_ab (x_ak - x_bk)^2 / theta_k^2 (zero on the diagonal).
    Returns (l, grad); (nan, nan-vector) when K is not positive definite."""
    S = np.asarray(S, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    n, p = S.shape
    D = (S[:, None, :] - S[None, :, :]) ** 2                  # n x n x p
    K = np.exp(-(D / theta).sum(axis=2))
    np.fill_diagonal(K, 1.0 + g)
    try:
        Lc = np.linalg.cholesky(K)
    except np.linalg.LinAlgError:
        return math.nan, np.full(p, math.nan)
    Linv = np.linalg.solve(Lc, np.eye(n))
    Ki = Linv.T @ Linv
    alpha = Ki @ y
    psi = float(y @ alpha)
    logdet = 2.0 * float(np.sum(np.log(np.diag(Lc))))
    l = (math.lgamma(0.5 * n) - 0.5 * n * math.log(2.0 * math.pi) - 0.5 * logdet
         - 0.5 * n * math.log(psi / 2.0))
    grad = np.empty(p)
    for k in range(p):
        Kk = K * D[:, :, k] / theta[k] ** 2
        np.fill_diagonal(Kk, 0.0)
        tr = float(np.sum(Ki * Kk))                          # tr(K^{-1} K_k), both symmetric
        psik = -float(alpha @ Kk @ alpha)
        grad[k] = -0.5 * tr - 0.5 * n * psik / psi
    return l, grad


def sep_mle(S, y, g, theta0, tmin, tmax, tol=1e-9, maxit=200):
    """BFGS maximiser of sep_loglik over [tmin, tmax]^p (reading P2).
    Returns (theta, iterations, likelihood evaluations, l at theta)."""
    S = np.asarray(S, dtype=np.float64)
    p = S.shape[1]
    lo, hi = math.log(tmin), math.log(tmax)
    eta = np.clip(np.log(np.broadcast_to(np.asarray(theta0, dtype=np.float64), (p,))), lo, hi)
    l, gt = sep_loglik(S, y, np.exp(eta), g)
    evals = 1
    gr = gt * np.exp(eta)                                     # gradient in eta
    H = np.eye(p)
    it = 0
    while it < maxit:
        it += 1
        d = H @ gr
        m = float(np.max(np.abs(d)))
        if m > 2.0:
            d = d * (2.0 / m)
        t = 1.0
        accepted = False
        stalled = False
        for _ in range(41):
            eta_t = np.clip(eta + t * d, lo, hi)
            s = eta_t - eta
            if float(np.max(np.abs(s))) <= tol:
                stalled = True
                break
            l_t, gt_t = sep_loglik(S, y, np.exp(eta_t), g)
            evals += 1
            if l_t == l_t and l_t >= l + 1e-4 * float(gr @ s):
                accepted = True
                break
            t *= 0.5
        if not accepted:
            break
        gr_t = gt_t * np.exp(eta_t)
        yv = gr - gr_t
        sy = float(s @ yv)
        if sy > 1e-12 * float(np.linalg.norm(s)) * float(np.linalg.norm(yv)):
            rho = 1.0 / sy
            E = np.eye(p) - rho * np.outer(s, yv)
            H = E @ H @ E.T + rho * np.outer(s, s)
        eta, l, gr = eta_t, l_t, gr_t
        if float(np.max(np.abs(s))) <= tol or stalled:
            break
    return np.exp(eta), it, evals, l


def prescale(X, theta):
    """Inputs divided by the square roots of the global lengthscales (P3)."""
    return np.asarray(X, dtype=np.float64) / np.sqrt(np.asarray(theta, dtype=np.float64))
