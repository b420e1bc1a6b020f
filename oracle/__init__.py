"""FP64 CPU oracle for local approximate GP prediction (Gramacy & Haaland,
arXiv:1409.0074): kNN candidates, greedy ALC local design by exhaustive search
(Sec 2.2, Eq. alc) or by ray search (Sec 4), and the predictive equations
(Eq. predgp, preds2).

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
benchmark's CPU-baseline leg are its only users.  The CUDA product path never
imports it.  The arithmetic lives in lagp_oracle.c; this module marshals numpy
arrays through ctypes.

Local inference for the lengthscale (Sec 5, Eq. gpk): loglik, mle_theta and
predict_mle, pinned in tests/test_oracle_mle.py.

Every function here is pinned by tests under tests/ against closed forms,
brute force or library routines (numpy, scipy).  The paper prints no worked ray
example, so ray-search designs are pinned piece by piece (round-robin offsets,
segments, Brent minima, snapping) and as whole designs against a replay of
every step from independent parts: a numpy kNN sort, the hand-worked offsets,
ALC as a directly re-solved variance drop, scipy's bounded Brent minimiser and
a brute-force snap (tests/test_oracle_ray_designs.py).
"""
import contextlib
import ctypes as C

import numpy as np

from . import build as _build

_lib = None
_F1 = C.CFUNCTYPE(C.c_double, C.c_double, C.c_void_p)


def lib():
    global _lib
    if _lib is None:
        _lib = _configure(C.CDLL(_build.build()))
    return _lib


@contextlib.contextmanager
def library(path):
    """Route every call of this module to another build of the oracle while
    the block runs (the planted-mistake tests compile altered copies)."""
    global _lib
    saved = _lib
    _lib = _configure(C.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def set_jitter(seed):
    """Rounding-noise probe: with seed != 0 every correlation value is
    multiplied by 1 +- 2^-52 (a counter-based choice per location and call);
    seed 0 switches it off."""
    lib().lagp_oracle_set_jitter(C.c_uint64(int(seed)))


def _configure(L):
    """Declares the C signatures on a loaded oracle library; returns it."""
    dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int32)
    L.lagp_oracle_set_jitter.restype = None
    L.lagp_oracle_set_jitter.argtypes = [C.c_uint64]
    L.lagp_oracle_set_snap_scope.restype = None
    L.lagp_oracle_set_snap_scope.argtypes = [C.c_int]
    L.lagp_oracle_exp.restype = C.c_double
    L.lagp_oracle_exp.argtypes = [C.c_double]
    L.lagp_oracle_sqdist.restype = C.c_double
    L.lagp_oracle_sqdist.argtypes = [dp, dp, C.c_int]
    L.lagp_oracle_knn.restype = C.c_int
    L.lagp_oracle_knn.argtypes = [dp, C.c_int64, C.c_int, dp, C.c_int, ip, dp]
    L.lagp_oracle_update.restype = C.c_double
    L.lagp_oracle_update.argtypes = [dp, C.c_int, C.c_int, dp, C.c_double, dp]
    L.lagp_oracle_alc.restype = C.c_double
    L.lagp_oracle_alc.argtypes = [dp, C.c_int, C.c_int, dp, C.c_int, dp, dp, dp,
                                     C.c_double, C.c_double, dp, dp, dp]
    L.lagp_oracle_brent.restype = C.c_double
    L.lagp_oracle_brent.argtypes = [_F1, C.c_void_p, C.c_double, C.c_double,
                                       C.c_double, C.c_int, dp, C.POINTER(C.c_int), dp]
    L.lagp_oracle_ray_k.restype = C.c_int
    L.lagp_oracle_ray_k.argtypes = [C.c_int, C.c_int]
    L.lagp_oracle_ray_segment.restype = C.c_double
    L.lagp_oracle_ray_segment.argtypes = [dp, dp, dp, dp, C.c_int, dp]
    L.lagp_oracle_bbox.restype = None
    L.lagp_oracle_bbox.argtypes = [dp, C.c_int64, C.c_int, dp, dp]
    L.lagp_oracle_predict.restype = C.c_int
    L.lagp_oracle_predict.argtypes = [
        dp, dp, C.c_int64, C.c_int, dp, C.c_int64, C.c_int, C.c_int, C.c_int,
        ip, ip, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
        dp, dp, ip, dp, ip, ip, C.c_int]
    L.lagp_oracle_loglik.restype = C.c_double
    L.lagp_oracle_loglik.argtypes = [dp, dp, C.c_int, C.c_int, C.c_double, C.c_double,
                                        dp, dp]
    L.lagp_oracle_mle_theta.restype = C.c_double
    L.lagp_oracle_mle_theta.argtypes = [dp, dp, C.c_int, C.c_int, C.c_double,
                                           C.c_double, C.c_double, C.c_double,
                                           C.c_double, C.c_int, C.POINTER(C.c_int)]
    L.lagp_oracle_predict_mle.restype = C.c_int
    L.lagp_oracle_predict_mle.argtypes = [
        dp, dp, C.c_int64, C.c_int, dp, C.c_int64, C.c_int, C.c_int, C.c_int,
        C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int,
        dp, dp, dp, ip, ip, C.c_int]
    return L


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int32))


def exp(x: float) -> float:
    """exp by Cody-Waite reduction and a degree-13 Taylor polynomial."""
    return lib().lagp_oracle_exp(float(x))


def sqdist(a, b) -> float:
    a, pa = _d(a)
    b, pb = _d(b)
    return lib().lagp_oracle_sqdist(pa, pb, a.size)


def knn(X, x, nc):
    """The nc nearest design rows to x: (indices, squared distances), sorted by
    (distance, index) (Sec 2.2)."""
    X, pX = _d(X)
    x, px = _d(x)
    idx, pi = _i(np.zeros(nc, np.int32))
    dist, pd = _d(np.zeros(nc))
    rc = lib().lagp_oracle_knn(pX, X.shape[0], X.shape[1], px, nc, pi, pd)
    if rc != 0:
        raise ValueError("knn: bad arguments")
    return idx, dist


def update(Kinv, kvec, g):
    """One partitioned-inverse step: K_j^{-1} (j x j) and k_j(x_new) ->
    (K_{j+1}^{-1}, v).  Raises when v <= 0."""
    j = len(kvec)
    buf = np.zeros((j + 1, j + 1))
    buf[:j, :j] = Kinv
    buf, pb = _d(buf)
    k, pk = _d(kvec)
    w, pw = _d(np.zeros(max(j, 1)))
    v = lib().lagp_oracle_update(pb, j, j + 1, pk, float(g), pw)
    if not v > 0:
        raise FloatingPointError("update: Schur complement v = %r <= 0" % v)
    return buf, v


def alc(S, Kinv, kx, x, z, theta, g):
    """ALC at z (Eq. alc integrand, reading R3/R4): returns (alc, v, num)."""
    S, pS = _d(np.atleast_2d(S))
    j, p = S.shape
    Kinv, pK = _d(Kinv)
    kx, pkx = _d(kx)
    x, px = _d(x)
    z, pz = _d(z)
    w, pw = _d(np.zeros(max(2 * j, 1)))
    v = C.c_double()
    num = C.c_double()
    a = lib().lagp_oracle_alc(pS, j, p, pK, j, pkx, px, pz, float(theta), float(g), pw,
                              C.byref(v), C.byref(num))
    return a, v.value, num.value


def brent(f, lo=0.0, hi=1.0, tol=2.0 ** -13, max_iter=1000):
    """Brent (1973) fmin of a Python callable on [lo, hi]:
    returns (xmin, fmin, nevals, mingap)."""
    cb = _F1(lambda s, _ctx: float(f(s)))
    xmin = C.c_double()
    ne = C.c_int()
    gap = C.c_double()
    fmin = lib().lagp_oracle_brent(cb, None, lo, hi, tol, max_iter, C.byref(xmin),
                                   C.byref(ne), C.byref(gap))
    return xmin.value, fmin, ne.value, gap.value


def ray_k(j, n0):
    """Round-robin start offset k = t mod floor(sqrt(t)), t = j - n0 + 1 (Sec 4)."""
    return lib().lagp_oracle_ray_k(int(j), int(n0))


def ray_segment(A, x, lo, hi):
    """Segment end E and clip fraction tau for a ray from start A away from x (Sec 4)."""
    A, pA = _d(A)
    x, px = _d(x)
    lo, plo = _d(lo)
    hi, phi = _d(hi)
    E, pE = _d(np.zeros(A.size))
    tau = lib().lagp_oracle_ray_segment(pA, px, plo, phi, A.size, pE)
    return E, tau


def bbox(X):
    X, pX = _d(X)
    p = X.shape[1]
    lo, plo = _d(np.zeros(p))
    hi, phi = _d(np.zeros(p))
    lib().lagp_oracle_bbox(pX, X.shape[0], p, plo, phi)
    return lo, hi


SEARCH = {"exhaustive": 0, "ray": 1}


SNAP = {"candidates": 0, "design": 1}


@contextlib.contextmanager
def _snap_scope(snap):
    lib().lagp_oracle_set_snap_scope(SNAP[snap])
    try:
        yield
    finally:
        lib().lagp_oracle_set_snap_scope(0)


def predict(X, Y, Xref, n0, n, nc, theta, g, search="exhaustive", nrays=0,
            n_arr=None, nc_arr=None, nthreads=1, snap="candidates"):
    """The whole path for every row of Xref.  Returns a dict with mean, s2,
    selected (design indices in selection order, -1 padded), gap (per greedy
    step, smallest relative gap of its decisions), nevals (ALC evaluations per
    ray step), status, and threads (OpenMP threads used).  snap = "design"
    snaps ray steps over all of X_N outside the design (reading R14) instead
    of the unselected candidates."""
    with _snap_scope(snap):
        return _predict(X, Y, Xref, n0, n, nc, theta, g, search, nrays, n_arr, nc_arr, nthreads)


def _predict(X, Y, Xref, n0, n, nc, theta, g, search, nrays, n_arr, nc_arr, nthreads):
    X, pX = _d(X)
    Y, pY = _d(Y)
    Xref, pR = _d(np.atleast_2d(Xref))
    N, p = X.shape
    M = Xref.shape[0]
    n_stride = int(max(n, np.max(n_arr) if n_arr is not None else 0))
    pn = pc = None
    if n_arr is not None:
        n_arr, pn = _i(n_arr)
    if nc_arr is not None:
        nc_arr, pc = _i(nc_arr)
    mean, pm = _d(np.zeros(M))
    s2, ps = _d(np.zeros(M))
    sel, psel = _i(np.zeros((M, n_stride), np.int32))
    gap, pg = _d(np.zeros((M, n_stride)))
    nev, pne = _i(np.zeros((M, n_stride), np.int32))
    st, pst = _i(np.zeros(M, np.int32))
    used = lib().lagp_oracle_predict(pX, pY, N, p, pR, M, n0, n, nc, pn, pc, n_stride,
                                     float(theta), float(g), SEARCH[search], int(nrays),
                                     pm, ps, psel, pg, pne, pst, int(nthreads))
    return dict(mean=mean, s2=s2, selected=sel, gap=gap, nevals=nev, status=st,
                threads=used)


def loglik(S, y, theta, g):
    """log p(y | K_theta) of Eq. gpk on the local design S (n x p) with
    responses y, and its first and second derivatives in theta:
    (value, d/dtheta, d2/dtheta2)."""
    S, pS = _d(np.atleast_2d(S))
    y, py = _d(y)
    n, p = S.shape
    d1, p1 = _d(np.zeros(1))
    d2, p2 = _d(np.zeros(1))
    v = lib().lagp_oracle_loglik(pS, py, n, p, float(theta), float(g), p1, p2)
    return v, float(d1[0]), float(d2[0])


def mle_theta(S, y, theta0, g, tmin, tmax, tol=1e-10, maxit=200):
    """Safeguarded Newton maximiser of loglik over [tmin, tmax] from theta0
    (Sec 5's local inference for the lengthscale).  Returns (theta, iters)."""
    S, pS = _d(np.atleast_2d(S))
    y, py = _d(y)
    n, p = S.shape
    it = C.c_int(0)
    t = lib().lagp_oracle_mle_theta(pS, py, n, p, float(theta0), float(g), float(tmin),
                                    float(tmax), float(tol), int(maxit), C.byref(it))
    return t, it.value


def predict_mle(X, Y, Xref, n0, n, nc, theta0, g, tmin, tmax, search="exhaustive", nrays=0,
                stages=1, nthreads=1, snap="candidates"):
    """Local designs coupled with local inference for theta: `stages` rounds of
    (greedy design at the current theta, then the MLE on that design, starting
    from theta0), and the predictive equations at the last estimate on the last
    design.  Returns a dict with mean, s2, theta, selected, status, threads."""
    X, pX = _d(X)
    Y, pY = _d(Y)
    Xref, pR = _d(np.atleast_2d(Xref))
    N, p = X.shape
    M = Xref.shape[0]
    mean, pm = _d(np.zeros(M))
    s2, ps = _d(np.zeros(M))
    th, pt = _d(np.zeros(M))
    sel, psel = _i(np.zeros((M, n), np.int32))
    st, pst = _i(np.zeros(M, np.int32))
    with _snap_scope(snap):
        used = lib().lagp_oracle_predict_mle(pX, pY, N, p, pR, M, n0, n, nc, float(theta0),
                                             float(g), float(tmin), float(tmax), SEARCH[search],
                                             int(nrays), int(stages), pm, ps, pt, psel, pst,
                                             int(nthreads))
    return dict(mean=mean, s2=s2, theta=th, selected=sel, status=st, threads=used)
