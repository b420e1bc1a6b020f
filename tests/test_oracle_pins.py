"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test names the passage of Gramacy & Haaland (arXiv:1409.0074) it checks and
what fixes the expected value: libm, numpy/scipy/scikit-learn routines, brute
force on tiny inputs, closed forms, metamorphic identities, or the paper's own
rules worked by hand (tests/golden/).  Nugget values are chosen large enough
that dropping g from a formula moves a result past the tolerance.
"""
import math
import os

import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle
from paper_1409_0074_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def kmat(A, B, theta):
    """Isotropic Gaussian correlation via scipy's squared distances (Sec 2.1)."""
    return np.exp(-cdist(np.atleast_2d(A), np.atleast_2d(B), "sqeuclidean") / theta)


def ulps(a, b):
    if a == b:
        return 0
    return abs(a - b) / math.ulp(max(abs(a), abs(b)))


# --- exp ---------------------------------------------------------------------

def test_exp_within_two_ulp_of_libm():
    rng = np.random.default_rng(1)
    xs = np.concatenate([-rng.random(20000) * 708.0, -rng.random(20000) * 5.0,
                         rng.random(2000) * 700.0, [0.0, -1e-300, -0.5, -1.0, -707.9]])
    worst = max(ulps(oracle.exp(float(x)), math.exp(float(x))) for x in xs)
    assert worst <= 2.0
    assert oracle.exp(0.0) == 1.0
    assert oracle.exp(-709.0) == 0.0          # flushed below the normal range
    assert math.isnan(oracle.exp(float("nan")))


# --- kNN (Sec 2.2) -------------------------------------------------------------

@pytest.mark.parametrize("grid", [False, True])
def test_knn_equals_lexicographic_sort(grid):
    rng = np.random.default_rng(2)
    if grid:   # integer grid: many exactly tied distances
        X = rng.integers(0, 6, (1500, 3)).astype(np.float64)
        x = np.array([2.0, 3.0, 1.0])
    else:
        X = rng.random((3000, 4))
        x = rng.random(4)
    d = np.zeros(X.shape[0])
    for k in range(X.shape[1]):
        d = d + (X[:, k] - x[k]) ** 2
    order = np.lexsort((np.arange(X.shape[0]), d))[:300]
    idx, dist = oracle.knn(X, x, 300)
    np.testing.assert_array_equal(idx, order)
    np.testing.assert_array_equal(dist, d[order])


# --- partitioned inverse (Sec 2.2, pieces of Eq. alc) ---------------------------

@pytest.mark.parametrize("theta,g", [(0.02, 1e-3), (0.3, 1e-6)])
def test_update_matches_direct_inverse_every_step(theta, g):
    rng = np.random.default_rng(3)
    S = rng.random((25, 2))
    Kinv = np.zeros((0, 0))
    for j in range(S.shape[0]):
        kvec = np.array([oracle.exp(-(oracle.sqdist(S[i], S[j]) / theta)) for i in range(j)])
        Kinv, v = oracle.update(Kinv, kvec, g)
        K = kmat(S[: j + 1], S[: j + 1], theta) + g * np.eye(j + 1)
        direct = np.linalg.inv(K)
        cond = np.linalg.cond(K)
        err = np.linalg.norm(Kinv - direct) / np.linalg.norm(direct)
        assert err <= 1e-13 * cond + 1e-14, (j, err, cond)
        # v is the Schur complement: det K_{j+1} / det K_j
        if j > 0:
            Kp = K[:j, :j]
            ratio = np.exp(np.linalg.slogdet(K)[1] - np.linalg.slogdet(Kp)[1])
            assert abs(v - ratio) <= 1e-12 * cond * max(1.0, ratio)


# --- ALC (Eq. alc integrand, sign reading R3) ----------------------------------

def _posterior_var(S, z, theta, g):
    """Correlation-scale predictive variance at z given design S, by direct solve."""
    K = kmat(S, S, theta) + g * np.eye(len(S))
    k = kmat(S, z, theta)[:, 0]
    return (1.0 + g) - k @ np.linalg.solve(K, k)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_alc_equals_bruteforce_variance_reduction(p):
    rng = np.random.default_rng(10 + p)
    N, j, theta, g = 50, 6, 0.05 * p, 1e-3
    X = rng.random((N, p))
    x = rng.random(p)
    idx, _ = oracle.knn(X, x, N)
    S = X[idx[:j]]
    K = kmat(S, S, theta) + g * np.eye(j)
    Kinv = np.linalg.inv(K)
    kx = kmat(S, x, theta)[:, 0]
    V0 = _posterior_var(S, x, theta, g)
    for c in idx[j:]:
        z = X[c]
        a, v, num = oracle.alc(S, Kinv, kx, x, z, theta, g)
        bf = V0 - _posterior_var(np.vstack([S, z]), x, theta, g)
        assert a >= 0.0
        assert abs(a - bf) <= 1e-9 * max(1.0, abs(bf)), (c, a, bf)
        assert abs(v - _posterior_var(S, z, theta, g)) <= 1e-10


# --- predictive equations (Eq. predgp, preds2) ---------------------------------

def _sklearn_pred(S, yS, x, theta, g):
    """Mean, correlation-scale variance and psi from scikit-learn's exact GP."""
    from sklearn.gaussian_process import GaussianProcessRegressor
    from sklearn.gaussian_process.kernels import RBF
    gp = GaussianProcessRegressor(kernel=RBF(length_scale=math.sqrt(theta / 2.0)), alpha=g,
                                  optimizer=None, normalize_y=False)
    gp.fit(S, yS)
    mu, sd = gp.predict(np.atleast_2d(x), return_std=True)
    n = len(S)
    K = kmat(S, S, theta) + g * np.eye(n)
    logdet = np.linalg.slogdet(K)[1]
    # log marginal likelihood = -psi/2 - logdet/2 - n/2 log(2 pi)
    psi = -2.0 * (gp.log_marginal_likelihood_value_ + 0.5 * logdet + 0.5 * n * math.log(2 * math.pi))
    return mu[0], sd[0] ** 2 + g, psi


@pytest.mark.parametrize("n", [6, 14])
def test_predict_matches_sklearn_kriging(n):
    pytest.importorskip("sklearn")
    w = W.small(N=400, p=2, M=5, n0=6, n=n, nc=40, theta=0.02, g=1e-2, seed=4)
    r = oracle.predict(w.X, w.Y, w.Xref, w.n0, w.n, w.nc, w.theta, w.g, "exhaustive")
    for m in range(w.M):
        sel = r["selected"][m, :n]
        mu, var, psi = _sklearn_pred(w.X[sel], w.Y[sel], w.Xref[m], w.theta, w.g)
        assert abs(r["mean"][m] - mu) <= 1e-10 * max(1.0, abs(mu))
        assert abs(r["s2"][m] - psi * var / n) <= 1e-9 * abs(psi * var / n)


def test_predict_precision_matrix_form():
    """sigma^2 and mean from the inverse of the joint (n+1)x(n+1) correlation
    matrix of (design, x): the conditional of a Gaussian (Sec 2.1)."""
    w = W.small(N=300, p=3, M=4, n0=5, n=5, nc=20, theta=0.1, g=1e-3, seed=5)
    r = oracle.predict(w.X, w.Y, w.Xref, w.n0, w.n, w.nc, w.theta, w.g, "exhaustive")
    for m in range(w.M):
        sel = r["selected"][m, :5]
        Z = np.vstack([w.X[sel], w.Xref[m]])
        J = kmat(Z, Z, w.theta) + w.g * np.eye(6)
        P = np.linalg.inv(J)
        cond_var = 1.0 / P[5, 5]
        cond_mean = -P[5, :5] @ w.Y[sel] / P[5, 5]
        psi = w.Y[sel] @ np.linalg.solve(J[:5, :5], w.Y[sel])
        assert abs(r["mean"][m] - cond_mean) <= 1e-10 * max(1, abs(cond_mean))
        assert abs(r["s2"][m] - psi * cond_var / 5) <= 1e-9 * psi * cond_var / 5


def test_interpolates_as_nugget_vanishes():
    """At g -> 0 the predictor interpolates the design (Sec 2.1)."""
    gx = np.linspace(0.0, 1.0, 9)
    X = np.array([[a, b] for a in gx for b in gx])
    Y = np.sin(3 * X[:, 0]) + X[:, 1] ** 2
    xs = X[[10, 40, 57]]
    r = oracle.predict(X, Y, xs, 4, 10, 30, 0.01, 1e-10, "exhaustive")
    np.testing.assert_allclose(r["mean"], Y[[10, 40, 57]], rtol=0, atol=1e-7)
    assert np.all(r["s2"] < 1e-8)


# --- greedy local design (Sec 2.2) ---------------------------------------------

def test_exhaustive_greedy_matches_bruteforce_resolves():
    """Each greedy pick minimises the directly re-solved variance V_{j+1}(x)."""
    w = W.small(N=120, p=2, M=3, n0=3, n=10, nc=30, theta=0.02, g=1e-3, seed=6)
    r = oracle.predict(w.X, w.Y, w.Xref, w.n0, w.n, w.nc, w.theta, w.g, "exhaustive")
    for m in range(w.M):
        x = w.Xref[m]
        cand, _ = oracle.knn(w.X, x, w.nc)
        S = list(cand[: w.n0])
        for j in range(w.n0, w.n):
            rest = [c for c in cand if c not in S]
            vals = np.array([_posterior_var(w.X[S + [c]], x, w.theta, w.g) for c in rest])
            order = np.argsort(vals, kind="stable")
            gap = (vals[order[1]] - vals[order[0]]) / max(abs(vals[order[0]]), 1e-300)
            assert gap > 1e-8, "tiny case should have no near-ties"
            S.append(rest[order[0]])
        np.testing.assert_array_equal(r["selected"][m, : w.n], S)


def test_full_candidate_set_gives_knn_kriging():
    """With N' = n every candidate is selected; the final predictor is kriging on
    the n nearest neighbours whatever the order (Sec 2.2)."""
    pytest.importorskip("sklearn")
    w = W.small(N=500, p=2, M=4, n0=3, n=15, nc=15, theta=0.05, g=1e-3, seed=7)
    for search in ("exhaustive", "ray"):
        r = oracle.predict(w.X, w.Y, w.Xref, w.n0, w.n, w.nc, w.theta, w.g, search,
                           nrays=1)
        for m in range(w.M):
            cand, _ = oracle.knn(w.X, w.Xref[m], w.nc)
            assert sorted(r["selected"][m]) == sorted(cand)
            mu, var, psi = _sklearn_pred(w.X[cand], w.Y[cand], w.Xref[m], w.theta, w.g)
            assert abs(r["mean"][m] - mu) <= 1e-9 * max(1, abs(mu))
            assert abs(r["s2"][m] - psi * var / w.n) <= 1e-8 * psi * var / w.n


@pytest.mark.parametrize("search", ["exhaustive", "ray"])
def test_variance_nonincreasing_and_alc_nonnegative(search):
    w = W.small(N=800, p=2, M=3, n0=4, n=16, nc=80, theta=0.05, g=1e-4, seed=8,
                search=search)
    r = oracle.predict(w.X, w.Y, w.Xref, w.n0, w.n, w.nc, w.theta, w.g, search, nrays=2)
    for m in range(w.M):
        sel = r["selected"][m]
        x = w.Xref[m]
        V = [_posterior_var(w.X[sel[:j]], x, w.theta, w.g) for j in range(w.n0, w.n + 1)]
        assert np.all(np.diff(V) <= 1e-12)
        cand, _ = oracle.knn(w.X, x, w.nc)
        S = w.X[sel[:10]]
        K = kmat(S, S, w.theta) + w.g * np.eye(10)
        Kinv, kx = np.linalg.inv(K), kmat(S, x, w.theta)[:, 0]
        for c in cand:
            assert oracle.alc(S, Kinv, kx, x, w.X[c], w.theta, w.g)[0] >= 0.0


@pytest.mark.parametrize("search", ["exhaustive", "ray"])
def test_exact_ties_go_to_the_lower_rank(search):
    """A design holding every point twice makes exact ties in distance, ALC and
    snapping distance; each tie must go to the lower candidate rank, i.e. the
    lower design index (readings R6, R7, R11)."""
    w = W.small(N=300, p=2, M=6, n0=3, n=14, nc=60, theta=0.05, g=1e-4, seed=15)
    X2, Y2 = np.vstack([w.X, w.X]), np.concatenate([w.Y, w.Y])
    r = oracle.predict(X2, Y2, w.Xref, w.n0, w.n, w.nc, w.theta, w.g, search, nrays=2)
    assert np.all(r["status"] == 0)
    for m in range(w.M):
        sel = list(r["selected"][m])
        for pos, i in enumerate(sel):
            twin = i + w.N if i < w.N else i - w.N
            if twin in sel:
                assert sel.index(min(i, twin)) < sel.index(max(i, twin))
            else:
                assert i < w.N, (m, pos, i)


# --- metamorphic identities ----------------------------------------------------

@pytest.mark.parametrize("search", ["exhaustive", "ray"])
def test_scaling_coordinates_by_two_and_theta_by_four_is_exact(search):
    w = W.small(N=700, p=3, M=4, n0=4, n=14, nc=70, theta=0.1, g=1e-5, seed=9)
    a = oracle.predict(w.X, w.Y, w.Xref, w.n0, w.n, w.nc, w.theta, w.g, search, nrays=3)
    b = oracle.predict(2 * w.X, w.Y, 2 * w.Xref, w.n0, w.n, w.nc, 4 * w.theta, w.g, search,
                       nrays=3)
    np.testing.assert_array_equal(a["selected"], b["selected"])
    np.testing.assert_array_equal(a["mean"], b["mean"])
    np.testing.assert_array_equal(a["s2"], b["s2"])


@pytest.mark.parametrize("search", ["exhaustive", "ray"])
def test_permuting_design_rows_permutes_selection(search):
    w = W.small(N=700, p=2, M=4, n0=4, n=14, nc=70, theta=0.05, g=1e-5, seed=10)
    perm = np.random.default_rng(0).permutation(w.N)
    a = oracle.predict(w.X, w.Y, w.Xref, w.n0, w.n, w.nc, w.theta, w.g, search, nrays=2)
    b = oracle.predict(w.X[perm], w.Y[perm], w.Xref, w.n0, w.n, w.nc, w.theta, w.g, search,
                       nrays=2)
    np.testing.assert_array_equal(perm[b["selected"]], a["selected"])
    np.testing.assert_array_equal(a["mean"], b["mean"])
    np.testing.assert_array_equal(a["s2"], b["s2"])


def test_translation_keeps_design_up_to_rounding():
    w = W.small(N=600, p=2, M=5, n0=4, n=12, nc=60, theta=0.05, g=1e-4, seed=11)
    a = oracle.predict(w.X, w.Y, w.Xref, w.n0, w.n, w.nc, w.theta, w.g, "exhaustive")
    b = oracle.predict(w.X + 3.0, w.Y, w.Xref + 3.0, w.n0, w.n, w.nc, w.theta, w.g,
                       "exhaustive")
    same = np.all(a["selected"] == b["selected"], axis=1)
    assert same.sum() >= w.M - 1
    np.testing.assert_allclose(a["mean"][same], b["mean"][same], rtol=1e-8, atol=1e-10)


# --- ray search pieces (Sec 4) -------------------------------------------------

def test_round_robin_offsets_match_hand_table():
    path = os.path.join(GOLDEN, "ray_start_offsets_n0_6.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 44
    for j, k in rows:
        assert oracle.ray_k(int(j), 6) == int(k), (j, k)


def test_ray_segment_hand_cases():
    lo, hi = np.zeros(2), np.ones(2)
    # inside: B = A + 10 (A - x) stays in the box
    E, tau = oracle.ray_segment([0.5, 0.5], [0.48, 0.5], lo, hi)
    assert tau == 1.0 and np.allclose(E, [0.7, 0.5], atol=1e-15)
    # exits through x1 = 1 at a quarter of the way: B = (2.5, 0.5)
    E, tau = oracle.ray_segment([0.5, 0.5], [0.3, 0.5], lo, hi)
    assert abs(tau - 0.25) < 1e-15 and np.allclose(E, [1.0, 0.5], atol=1e-15)
    # diagonal: B - A = (0.5, -0.2); x1 = 1 is reached at tau = 0.2, before
    # x2 = 0 (tau = 0.5), so E = (1.0, 0.06)
    E, tau = oracle.ray_segment([0.9, 0.1], [0.85, 0.12], lo, hi)
    assert abs(tau - 0.2) < 1e-15 and np.allclose(E, [1.0, 0.06], atol=1e-15)
    # the other way round: B - A = (-0.2, 0.5) reaches x2 = 1 at tau = 0.2
    E, tau = oracle.ray_segment([0.1, 0.9], [0.12, 0.85], lo, hi)
    assert abs(tau - 0.2) < 1e-15 and np.allclose(E, [0.06, 1.0], atol=1e-15)
    # start on the boundary, pointing out: zero length
    E, tau = oracle.ray_segment([1.0, 0.5], [0.9, 0.5], lo, hi)
    assert tau == 0.0 and np.array_equal(E, [1.0, 0.5])


def test_ray_segment_is_maximal_inside_box():
    rng = np.random.default_rng(12)
    lo, hi = np.array([-1.0, 0.0, 2.0]), np.array([1.0, 3.0, 2.5])
    for _ in range(200):
        A = lo + (hi - lo) * rng.random(3)
        x = A + 0.2 * rng.standard_normal(3)
        E, tau = oracle.ray_segment(A, x, lo, hi)
        B = A + 10 * (A - x)
        assert np.all(E >= lo - 1e-12) and np.all(E <= hi + 1e-12)
        np.testing.assert_allclose(E, A + tau * (B - A), atol=1e-12)
        if tau < 1.0:   # a step further leaves the box
            Z = A + (tau + 1e-9) * (B - A)
            assert np.any(Z < lo) or np.any(Z > hi)


@pytest.mark.parametrize("f,xstar", [
    (lambda s: (s - 0.3) ** 2, 0.3),
    (lambda s: s ** 3 - s, 1 / math.sqrt(3)),
    (lambda s: math.cos(7 * s), math.pi / 7),
    (lambda s: abs(s - 0.77) + 0.1 * (s - 0.77) ** 2, 0.77),
])
def test_brent_finds_known_minima(f, xstar):
    x, fx, ne, _ = oracle.brent(f)
    assert abs(x - xstar) <= 2.5e-4
    assert fx == f(x)
    assert ne < 60


def test_brent_trajectory_matches_scipy_bounded():
    """scipy's bounded scalar minimiser is an independent implementation of the
    same Brent (1973) method: from the same golden-section start, both must
    evaluate the same sequence of points (up to rounding) and stop together."""
    from scipy.optimize import minimize_scalar
    rng = np.random.default_rng(13)
    for _ in range(40):
        c1, c2, w1, w2 = rng.random(4)
        f = lambda s: -(math.exp(-(s - c1) ** 2 / (0.02 + w1 * 0.1))
                        + 1.5 * math.exp(-(s - c2) ** 2 / (0.02 + w2 * 0.1)))
        ours, theirs = [], []
        x, fx, ne, _ = oracle.brent(lambda s: (ours.append(s), f(s))[1])
        minimize_scalar(lambda s: (theirs.append(s), f(s))[1], bounds=(0, 1),
                        method="bounded", options={"xatol": 2.0 ** -13})
        assert ne == len(ours) == len(theirs)
        np.testing.assert_allclose(ours, theirs, rtol=0, atol=1e-8)
        # a local minimum: no lower value a little to either side
        for dx in (-2e-3, 2e-3):
            if 0 <= x + dx <= 1:
                assert f(x + dx) >= fx - 1e-12


def _oracle_state(w, m, j):
    """Design of the first j oracle selections at location m, rebuilt with the
    oracle's own update so that every value matches its internal state."""
    r = oracle.predict(w.X, w.Y, w.Xref[m:m + 1], w.n0, j, w.nc, w.theta, w.g, "ray",
                       nrays=w.nrays)
    sel = r["selected"][0, :j]
    S = w.X[sel]
    Kinv = np.zeros((0, 0))
    for i in range(j):
        kv = np.array([oracle.exp(-(oracle.sqdist(S[a], S[i]) / w.theta)) for a in range(i)])
        Kinv, _ = oracle.update(Kinv, kv, w.g)
    kx = np.array([oracle.exp(-(oracle.sqdist(S[i], w.Xref[m]) / w.theta)) for i in range(j)])
    return sel, S, Kinv, kx


def test_ray_step_composes_pinned_pieces():
    """One ray step rebuilt from the pinned pieces: round-robin starts, segments,
    Brent on -ALC, the s = 0 check, the best ray, and a brute-force snap with the
    starts forbidden (Sec 4)."""
    w = W.small(N=900, p=2, M=3, n0=4, n=14, nc=90, theta=0.05, g=1e-5, seed=14, nrays=3)
    lo, hi = oracle.bbox(w.X)
    full = oracle.predict(w.X, w.Y, w.Xref, w.n0, w.n, w.nc, w.theta, w.g, "ray", nrays=3)
    for m in range(w.M):
        x = w.Xref[m]
        cand, _ = oracle.knn(w.X, x, w.nc)
        for j in (w.n0, w.n0 + 4, w.n - 1):
            sel, S, Kinv, kx = _oracle_state(w, m, j)
            U = [c for c in cand if c not in set(sel)]
            k0 = oracle.ray_k(j, w.n0)
            starts = [U[(k0 + i) % len(U)] for i in range(w.nrays)]
            best = None
            for i, st in enumerate(starts):
                A = w.X[st]
                E, _ = oracle.ray_segment(A, x, lo, hi)
                pt = lambda s: A + s * (E - A)
                alc = lambda s: oracle.alc(S, Kinv, kx, x, pt(s), w.theta, w.g)[0]
                a0 = alc(0.0)
                s_star, a_star = 0.0, a0
                if oracle.sqdist(A, E) > 0:
                    sb, fb, _, _ = oracle.brent(lambda s: -alc(s))
                    if not a0 >= -fb:
                        s_star, a_star = sb, -fb
                if best is None or a_star > best[0]:
                    best = (a_star, pt(s_star))
            xs = best[1]
            allowed = [c for c in U if c not in starts or np.array_equal(w.X[c], xs)]
            d = [oracle.sqdist(w.X[c], xs) for c in allowed]
            pick = allowed[int(np.argmin(d))]
            assert pick == full["selected"][m, j], (m, j)


# --- qualitative claims of the paper -------------------------------------------

def test_designs_mix_near_neighbours_and_satellites():
    """Local designs hold nearest neighbours and farther 'satellite' points
    (Sec 3, Figure 1); ray designs are qualitatively similar (Sec 4)."""
    w = W.dense_2d(M=20)
    for search in ("exhaustive", "ray"):
        r = oracle.predict(w.X, w.Y, w.Xref, w.n0, w.n, w.nc, w.theta, w.g, search,
                           nrays=2)
        frac_nn = []
        for m in range(w.M):
            cand, _ = oracle.knn(w.X, w.Xref[m], w.n)
            frac_nn.append(np.isin(r["selected"][m], cand).mean())
        frac_nn = np.array(frac_nn)
        assert 0.2 < frac_nn.mean() < 0.95, (search, frac_nn.mean())


def test_greedy_design_beats_nearest_start_and_rays_track_exhaustive():
    w = W.dense_2d(M=40)
    rm = lambda r: float(np.sqrt(np.mean((r["mean"] - w.Ytrue) ** 2)))
    nn = oracle.predict(w.X, w.Y, w.Xref, w.n0, w.n0, w.nc, w.theta, w.g, "exhaustive")
    ex = oracle.predict(w.X, w.Y, w.Xref, w.n0, w.n, w.nc, w.theta, w.g, "exhaustive")
    ry = oracle.predict(w.X, w.Y, w.Xref, w.n0, w.n, w.nc, w.theta, w.g, "ray", nrays=2)
    assert rm(ex) < 0.5 * rm(nn)
    assert rm(ry) < 3.0 * rm(ex)
