"""Seeded synthetic workloads shaped like the paper's experiments.

The paper's benchmark data (borehole, LGBB, Zhou, piston) are not available, so
noise-free synthetic responses on iid uniform designs stand in for them at the
paper's shapes: an 8-d design of N = 1e6 points with n = 50 and N' = 1000
candidates mirrors the borehole runs of Sec 5.3; a dense 2-d design mirrors
Sec 5.1.  The one workload the paper specifies completely, the gridded 2-d
function of Sec 5.1, is paper_2d (no random draws).

This module only draws inputs.  It holds none of the method's arithmetic and is
shared, as input source only, by the tests, the benchmark and the oracle side of
the tests.  One numpy Generator per workload, seed 0, draws in this order:
  1. design X = U[0,1)^(N x p)
  2. response constants a ~ U[0.5, 2)^p, then phi ~ U[0, 2 pi)^p (sinusoid form)
  3. predictive locations Xref = U[0,1)^(M x p)  (2-d form: 0.05 + 0.9 U)
  4. per-location n ~ U{20..100} then N_close ~ U{300..2000}   (uneven form)
"""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class Workload:
    name: str
    N: int
    p: int
    M: int
    n0: int
    n: int
    nc: int
    theta: float
    g: float
    search: str = "ray"
    nrays: int = 0
    response: str = "sinusoid"
    uneven: bool = False
    seed: int = 0
    X: Optional[np.ndarray] = field(default=None, repr=False)
    Y: Optional[np.ndarray] = field(default=None, repr=False)
    Xref: Optional[np.ndarray] = field(default=None, repr=False)
    Ytrue: Optional[np.ndarray] = field(default=None, repr=False)
    n_arr: Optional[np.ndarray] = field(default=None, repr=False)
    nc_arr: Optional[np.ndarray] = field(default=None, repr=False)
    a: Optional[np.ndarray] = field(default=None, repr=False)
    phi: Optional[np.ndarray] = field(default=None, repr=False)

    def true_response(self, X):
        """The workload's noise-free response at the rows of X."""
        if self.response == "2d":
            return _resp_2d(X)
        if self.response == "paper_2d":
            return _resp_paper_2d(X)
        return _resp_sinusoid(X, self.a, self.phi)


def _resp_2d(X):
    x1, x2 = X[:, 0], X[:, 1]
    return np.sin(2 * np.pi * 1.3 * x1 + 0.4) + np.cos(2 * np.pi * 0.7 * x2) + 0.5 * x1 * x2


def _resp_sinusoid(X, a, phi):
    return np.sin(2 * np.pi * a[None, :] * X + phi[None, :]).sum(axis=1) + 0.3 * np.prod(X, axis=1)


def _w_paper(x):
    """w(x) of the 2-d test function of Sec 5.1."""
    return np.exp(-(x - 1.0) ** 2) + np.exp(-0.8 * (x + 1.0) ** 2) - 0.05 * np.sin(8.0 * (x + 0.1))


def _resp_paper_2d(X):
    """f(x1, x2) = -w(x1) w(x2) (Sec 5.1)."""
    return -_w_paper(X[:, 0]) * _w_paper(X[:, 1])


def _grid(axis):
    a, b = np.meshgrid(axis, axis, indexing="ij")
    return np.stack([a.ravel(), b.ravel()], axis=1)


def generate(w: Workload) -> Workload:
    if w.response == "paper_2d":
        # deterministic: the design is the 201 x 201 grid on [-2, 2]^2; the
        # predictive locations a 99 x 99 grid of midpoints between design
        # coordinates (-1.97 + 0.04 k), so that none lies on X_N
        X = _grid(np.linspace(-2.0, 2.0, 201))
        Xref = _grid(-1.97 + 0.04 * np.arange(99))
        if w.M < Xref.shape[0]:
            Xref = Xref[np.random.default_rng(w.seed).choice(Xref.shape[0], w.M,
                                                            replace=False)]
        w.X, w.Y, w.Xref, w.Ytrue = X, _resp_paper_2d(X), Xref, _resp_paper_2d(Xref)
        w.N, w.M = X.shape[0], Xref.shape[0]
        return w
    rng = np.random.default_rng(w.seed)
    X = rng.random((w.N, w.p))
    if w.response == "2d":
        Xref = 0.05 + 0.9 * rng.random((w.M, w.p))
        Y, Yt = _resp_2d(X), _resp_2d(Xref)
    else:
        a = rng.uniform(0.5, 2.0, w.p)
        phi = rng.uniform(0.0, 2 * np.pi, w.p)
        Xref = rng.random((w.M, w.p))
        Y, Yt = _resp_sinusoid(X, a, phi), _resp_sinusoid(Xref, a, phi)
        w.a, w.phi = a, phi
    w.X, w.Y, w.Xref, w.Ytrue = X, Y, Xref, Yt
    if w.uneven:
        w.n_arr = rng.integers(20, 101, w.M).astype(np.int32)
        w.nc_arr = rng.integers(300, 2001, w.M).astype(np.int32)
    return w


def dense_2d(M=100, **kw):
    """2-d design, N = 4000, n0 = 6, n = 30, N' = 500, theta = 0.1, g = 1e-6."""
    return generate(Workload("dense_2d_N4000_n30", N=4000, p=2, M=M, n0=6, n=30, nc=500,
                             theta=0.1, g=1e-6, search=kw.pop("search", "exhaustive"),
                             nrays=kw.pop("nrays", 2), response="2d", **kw))


def paper_scale_4d(M=10000, **kw):
    """4-d design, N = 1e5, n = 50, N' = 1000, theta = 0.25, 4 rays."""
    return generate(Workload("sinusoid_4d_N100000_n50", N=100_000, p=4, M=M, n0=6, n=50,
                             nc=1000, theta=0.25, g=1e-6, search=kw.pop("search", "ray"),
                             nrays=kw.pop("nrays", 4), **kw))


def large_8d(M=100_000, N=1_000_000, **kw):
    """8-d design, N = 1e6, n = 50, N' = 1000, theta = 1, p = 8 rays (the
    borehole-shaped headline workload)."""
    return generate(Workload("sinusoid_8d_N%d_n50" % N, N=N, p=8, M=M, n0=6, n=50, nc=1000,
                             theta=1.0, g=1e-6, search=kw.pop("search", "ray"),
                             nrays=kw.pop("nrays", 8), **kw))


def uneven_8d(M=50_000, N=1_000_000, **kw):
    """8-d design, N = 1e6, per-location n ~ U{20..100}, N' ~ U{300..2000}."""
    return generate(Workload("sinusoid_8d_N%d_uneven" % N, N=N, p=8, M=M, n0=6, n=100,
                             nc=2000, theta=1.0, g=1e-6, search=kw.pop("search", "ray"),
                             nrays=kw.pop("nrays", 8), uneven=True, **kw))


def paper_2d(M=9801, n=50, nc=1000, theta=0.5, g=1e-6, **kw):
    """The 2-d experiment of Sec 5.1: f = -w(x1) w(x2) on the 201 x 201 grid
    over [-2, 2]^2 (N = 40,401), predicted on a 99 x 99 grid (M = 9801; a
    smaller M takes a seeded sample of it), one ray per step.  theta is the
    fixed lengthscale of the design (the start value of local inference for
    theta, which the paper runs on every local design)."""
    return generate(Workload("paper_2d_N40401_n%d" % n, N=40401, p=2, M=M, n0=6, n=n,
                             nc=nc, theta=theta, g=g, search=kw.pop("search", "ray"),
                             nrays=kw.pop("nrays", 1), response="paper_2d", **kw))


def small(N=600, p=2, M=8, n0=4, n=12, nc=60, theta=0.05, g=1e-6, seed=0, search="exhaustive",
          nrays=2, response="sinusoid"):
    """Small seeded case for tests (several tiles, ragged tails)."""
    return generate(Workload("small_%dd_N%d" % (p, N), N=N, p=p, M=M, n0=n0, n=n, nc=nc,
                             theta=theta, g=g, search=search, nrays=nrays, response=response,
                             seed=seed))


def subset(N, n, seed=1):
    """n distinct design rows drawn uniformly without replacement (the random
    subset of the crude global analysis that pre-scales the inputs, Sec 5.3),
    as int32 row indices in draw order."""
    return np.random.default_rng(seed).permutation(N)[:n].astype(np.int32)
