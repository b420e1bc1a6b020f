"""Whole ray-search designs of the FP64 oracle against an independent
replay (CPU only).

Sec 4 of Gramacy & Haaland (arXiv:1409.0074) prints no worked ray example, so
the oracle's ray designs are pinned here by rebuilding every greedy step from
parts that share nothing with the oracle's code:
- candidates: a numpy sort of the squared distances by (distance, index);
- ray starts: the round-robin offsets worked by hand in
  tests/golden/ray_start_offsets_n0_6.txt, over the unselected candidates in
  rank order;
- segments: B = A + 10 (A - x), cut where it leaves the design's bounding box;
- ALC(z): the drop in the kriging variance at x when z joins the design,
  by direct solves of the two systems (Eq. alc as a variance reduction);
- the line search: scipy's bounded scalar minimiser (Brent's method) on -ALC
  with the same absolute tolerance 2^-13, then the s = 0 check;
- the snap: the nearest unselected candidate to the best ray's point by brute
  force, the step's other starts excluded, ties to the lower rank.
A design may leave the oracle's only at a step whose decision the oracle logged
as close (relative gap below 1e-6): the two sides round differently.  Five
plausible mistakes planted in altered copies of the oracle each fail the replay.
"""
import os

import numpy as np
import pytest
from scipy.optimize import minimize_scalar
from scipy.spatial.distance import cdist

import oracle
from paper_1409_0074_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NEAR_TIE = 1e-6


def _offsets():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "ray_start_offsets_n0_6.txt"))
            if l.strip() and not l.startswith("#")]
    return {int(j): int(k) for j, k in rows}


def _kmat(A, B, theta):
    return np.exp(-cdist(np.atleast_2d(A), np.atleast_2d(B), "sqeuclidean") / theta)


def _var_at(S, x, theta, g):
    """Correlation-scale kriging variance at x given the design rows S."""
    K = _kmat(S, S, theta) + g * np.eye(len(S))
    k = _kmat(S, x, theta)[:, 0]
    return (1.0 + g) - k @ np.linalg.solve(K, k)


def _segment(A, x, lo, hi):
    """End of the ray from A away from x: A + tau 10 (A - x) with the largest
    tau in [0, 1] that stays inside [lo, hi]."""
    d = 10.0 * (A - x)
    tau = 1.0
    for a, dk, l, h in zip(A, d, lo, hi):
        if dk > 0:
            tau = min(tau, (h - a) / dk)
        elif dk < 0:
            tau = min(tau, (l - a) / dk)
    tau = max(tau, 0.0)
    return A + tau * d


def _replay_ray_design(w, m, offsets, lo, hi):
    x = w.Xref[m]
    d = cdist(w.X, x[None], "sqeuclidean")[:, 0]
    cand = np.lexsort((np.arange(w.N), d))[:w.nc]
    sel = list(cand[:w.n0])
    for j in range(w.n0, w.n):
        S = w.X[sel]
        v0 = _var_at(S, x, w.theta, w.g)
        alc = lambda z: v0 - _var_at(np.vstack([S, z]), x, w.theta, w.g)
        U = [c for c in cand if c not in set(sel)]
        starts = [U[(offsets[j] + i) % len(U)] for i in range(w.nrays)]
        best = None
        for st in starts:
            A = w.X[st]
            E = _segment(A, x, lo, hi)
            pt = lambda s: A + s * (E - A)
            a0 = alc(A)
            s_star, a_star = 0.0, a0
            if np.sum((E - A) ** 2) > 0:
                r = minimize_scalar(lambda s: -alc(pt(s)), bounds=(0.0, 1.0), method="bounded",
                                    options={"xatol": 2.0 ** -13})
                if a0 < -r.fun:
                    s_star, a_star = r.x, -r.fun
            if best is None or a_star > best[0]:
                best = (a_star, pt(s_star))
        xs = best[1]
        allowed = [c for c in U if c not in starts or np.array_equal(w.X[c], xs)]
        pool = allowed if allowed else U
        dist = [np.sum((w.X[c] - xs) ** 2) for c in pool]
        sel.append(pool[int(np.argmin(dist))])
    return np.array(sel)


CASES = [
    (2, 900, 0.05, 1e-5, 3, 21),
    (2, 1600, 0.02, 1e-6, 2, 22),
    (3, 2000, 0.2, 1e-4, 3, 23),
]


def check_ray_designs(p, N, theta, g, nrays, seed):
    w = W.small(N=N, p=p, M=6, n0=6, n=20, nc=120, theta=theta, g=g, seed=seed, nrays=nrays)
    o = oracle.predict(w.X, w.Y, w.Xref, w.n0, w.n, w.nc, w.theta, w.g, "ray", nrays=nrays)
    offsets = _offsets()
    lo, hi = w.X.min(axis=0), w.X.max(axis=0)
    whole = 0
    for m in range(w.M):
        mine = _replay_ray_design(w, m, offsets, lo, hi)
        diff = np.nonzero(mine != o["selected"][m])[0]
        if len(diff) == 0:
            whole += 1
            continue
        first = diff[0]
        assert first >= w.n0
        assert o["gap"][m, first - w.n0] < NEAR_TIE, (m, first, o["gap"][m, first - w.n0])
    # the replay reproduces most designs end to end
    assert whole >= w.M - 1, whole
    return whole


@pytest.mark.parametrize("case", CASES)
def test_whole_ray_designs_match_an_independent_replay(case):
    check_ray_designs(*case)


# Plausible mistakes in the oracle's ray search, each planted in an altered
# copy of the oracle's source; every one must fail the replay above.
MISTAKES = {
    "s = 0 check left out": (
        "if (!(alc0 >= alc_b)) { s_star = sb; alc_star = alc_b; }",
        "{ s_star = sb; alc_star = alc_b; }", 1),
    "round-robin offset off by one": (
        "int r = U[(k0 + i) % nU];", "int r = U[(k0 + i + 1) % nU];", 1),
    "worst ray taken": (
        "if (alcs[i] > alcs[ib]) ib = i;", "if (alcs[i] < alcs[ib]) ib = i;", 1),
    "segment without the factor 10": (
        "10.0 * (A[k] - x[k])", "1.0 * (A[k] - x[k])", 2),
    "the step's starts allowed in the snap": (
        "        if (forbidden) continue;\n        double d = lagp_oracle_sqdist(c, xs, p);",
        "        (void)forbidden;\n        double d = lagp_oracle_sqdist(c, xs, p);", 1),
}


@pytest.mark.parametrize("name", sorted(MISTAKES))
def test_each_planted_ray_mistake_fails_the_replay(name):
    import tempfile
    from oracle import build as oracle_build
    old, new, count = MISTAKES[name]
    src = open(oracle_build.SRC).read()
    assert src.count(old) == count, name
    with tempfile.TemporaryDirectory() as d:
        path = oracle_build.compile_source(src.replace(old, new), d)
        failed = 0
        with oracle.library(path):
            for case in CASES:
                try:
                    check_ray_designs(*case)
                except AssertionError:
                    failed += 1
        assert failed, "planted mistake '%s' passed the ray-design replay" % name
